// exchange_smem.cu -- decimation and cooling/heating exchanges (sections
// III.A and III.B of Hasenbusch & Schaefer) with the configurations of the
// current pair staged in shared memory, for lattices whose configurations fit
// on one SM (float: L <= 16).
//
// One CTA per chain walks the pairs (b, b+1) in increasing beta.  The
// configuration that sits at beta_{i+1} after pair i is the first
// configuration of pair i+1, so it stays on chip: per pair one configuration
// is read from global memory and at most one is written back (the one whose
// temperature is final).  Neighbour gathers of the cooling and heating sweeps,
// the decimated sums and the re-insertion heat bath all read shared memory.
// Global buffers keep their identities: a transformed configuration is written
// into the buffer of the configuration it replaces, and the
// temperature-to-buffer map records where each configuration lives.
#include "kernels.h"
#include "exchange_common.cuh"
#include "pt_device.cuh"
#include "tma.cuh"

namespace ptk {

constexpr int SX_THREADS = 1024;
constexpr int SX_MAX_NT = 512;

struct SxSmem {
    int buf[SX_MAX_NT];
    int lab[SX_MAX_NT];
    int rts[SX_MAX_NT];
    double H[SX_MAX_NT];
    double red[4 * 32];
    int flag;
};

__device__ void sx_load_state(const DevBatch& a, const ChainDesc& cd, int NT, SxSmem& sm) {
    for (int b = threadIdx.x; b < NT; b += blockDim.x) {
        sm.buf[b] = a.bufmap[cd.r0 + b];
        sm.lab[b] = a.label[cd.r0 + b];
        sm.rts[b] = a.rt_state[cd.r0 + b];
        sm.H[b] = a.H[cd.r0 + b];
    }
    __syncthreads();
}

__device__ void sx_store_state(const DevBatch& a, const ChainDesc& cd, int NT, SxSmem& sm, int ch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int top = sm.lab[0], bot = sm.lab[NT - 1];
        if (sm.rts[bot] == 1) sm.rts[bot] = 2;
        if (sm.rts[top] == 2) {
            a.rt_count[ch] += 1;
            sm.rts[top] = 1;
        } else if (sm.rts[top] == 0) {
            sm.rts[top] = 1;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NT; b += blockDim.x) {
        a.bufmap[cd.r0 + b] = sm.buf[b];
        a.label[cd.r0 + b] = sm.lab[b];
        a.rt_state[cd.r0 + b] = sm.rts[b];
        a.H[cd.r0 + b] = sm.H[b];
    }
}

// Copy n elements (a multiple of the 16-byte vector width) between global and
// shared memory with the whole CTA.
template <typename T>
__device__ __forceinline__ void sx_copy(T* __restrict__ dst, const T* __restrict__ src, int n) {
    constexpr int VW = 16 / sizeof(T);
    for (int q = threadIdx.x * VW; q < n; q += blockDim.x * VW) {
        T v[VW];
        ldv<T, VW>(src + q, v);
        stv<T, VW>(dst + q, v);
    }
}

template <typename T>
__device__ __forceinline__ T sx_decim_D(T n, T b1, T b2, T db, T lr) {
    const T R1 = b1 * n, R2 = b2 * n;
    if (R1 >= (T)0.5)
        return db * n - lr + M<T>::log1p_(-M<T>::exp_((T)-2 * R2)) - M<T>::log1p_(-M<T>::exp_((T)-2 * R1));
    return ln_sinhc<T>(R2) - ln_sinhc<T>(R1);
}

// ---------------------------------------------------------------------------
// Cooling/heating (section III.B).  The heated proposal of pair i is
// C^-1 of the configuration at beta_{i+1}, which no earlier pair of the update
// touches: k_heat_pre_smem computes it for every pair of every chain at once (with
// its energy and ln det J_C), and k_exchange_coolheat_smem then walks the
// pairs of each chain in order, cooling the configuration at beta_i (which
// does depend on the earlier decisions) in shared memory.
// ---------------------------------------------------------------------------
constexpr int HP_THREADS = 256;

// One colour of the cooling (COOL) or heating sweep of a configuration held
// in shared memory, over V-site vectors: the sites of colour `col` of `src`
// are transformed into `dst` (dst may equal src), the field coming from the
// other colour of `field`.  Adds ln det J_f to lj and, with ENERGY, -s.S of
// the new spins to e.  JS: the couplings J0, J1 are in shared memory too.
template <typename T, int V, bool COOL, bool ENERGY, bool JS = false>
__device__ __forceinline__ void ch_colour(const SampleDesc& sd, const T* field, const T* src, T* dst,
                                          const float* J0, const float* J1, int col, T eps, T& lj, T& e) {
    const int half = sd.half;
    const T* fo = field + (1 - col) * 3 * half;
    const float* Jown = col ? J1 : J0;
    const float* Joth = col ? J0 : J1;
    for (int h0 = (int)threadIdx.x * V; h0 < half; h0 += (int)blockDim.x * V) {
        const VRow q = vrow<V>(sd, col, h0);
        T S[3][V], s[3][V];
        nbr_field<T, V, JS>(fo, Jown, Joth, half, h0, q.xs, q.hyp, q.hym, q.hzp, q.hzm, q.p, S);
#pragma unroll
        for (int c = 0; c < 3; ++c) ldv<T, V>(src + col * 3 * half + c * half + h0, s[c]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv = {s[0][v], s[1][v], s[2][v]};
            lj += COOL ? cool_site<T>(eps, Sv, sv) : heat_site<T>(eps, Sv, sv);
            if (ENERGY) e -= dot(sv, Sv);
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<T, V>(dst + col * 3 * half + c * half + h0, s[c]);
    }
}

// Heated proposal of pair i (blockIdx.y) of chain blockIdx.x: C^-1 = colour
// 1 then colour 0 of the inverse step on the configuration at beta_{i+1},
// with eps_i.  The configuration and its sample's couplings are staged in
// shared memory (two bulk copies, io_bar counts their bytes; they fit one SM
// wherever the staged walk does): colour 1 then colour 0 are transformed in
// place (each site reads its own spin and neighbours of the other colour,
// which that pass does not change), and the result leaves by one bulk copy
// into the proposal buffer.
constexpr int HS_THREADS = 512;

template <typename T, int V>
__device__ __forceinline__ void heat_pass_smem(const SampleDesc& sd, T* cfg, const float* sJ, T eps, T (&part)[2]) {
    const int half = sd.half;
    T none = (T)0;
    ch_colour<T, V, false, false, true>(sd, cfg, cfg, cfg, sJ, sJ + 3 * half, 1, eps, part[0], none);
    __syncthreads();
    ch_colour<T, V, false, true, true>(sd, cfg, cfg, cfg, sJ, sJ + 3 * half, 0, eps, part[0], part[1]);
}

template <typename T>
__global__ void __launch_bounds__(HS_THREADS, sizeof(T) == 4 ? 2 : 1) k_heat_pre_smem(DevBatch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * 32];
    __shared__ __align__(8) unsigned long long io_bar;
    const int ch = blockIdx.x, i = blockIdx.y;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    if (i + 1 >= sd.NT) return;  // uniform over the block
    const int half = sd.half, n3 = 6 * half;
    const T* src = (const T*)a.spins + a.chain_off[ch] + (long long)a.bufmap[cd.r0 + i + 1] * n3;
    const long long pair = cd.pair_off + i;
    T* out = (T*)a.heat_buf + pair * (6LL * a.max_half);
    T* cfg = reinterpret_cast<T*>(smem_raw);
    float* sJ = reinterpret_cast<float*>(cfg + n3);  // n3 * sizeof(T) is a multiple of 16 B
    if (threadIdx.x == 0) {
        mbar_init(&io_bar, 1);
        fence_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned sb = (unsigned)(n3 * (int)sizeof(T)), jb = (unsigned)n3 * 4u;
        mbar_expect_tx(&io_bar, sb + jb);
        // failure-path test hook: block (0, 0) leaves its copies un-issued, so its wait runs out
        if (!(a.wait_fault && blockIdx.x == 0 && blockIdx.y == 0)) {
            bulk_g2s(cfg, src, sb, &io_bar);
            bulk_g2s(sJ, a.J + sd.J_off, jb, &io_bar);
        }
    }
    const T eps = (T)a.eps[sd.eps_off + i];
    if (__syncthreads_or(!mbar_wait_io(&io_bar, 0u, a, !(a.wait_fault && blockIdx.x == 0 && blockIdx.y == 0)))) {
        // gave up (error word set): no proposal; an infinite energy makes the
        // walk reject the pair (ln A = -inf, or NaN at beta = 0: never accepted)
        if (threadIdx.x == 0) {
            a.heat_H[pair] = __longlong_as_double(0x7FF0000000000000LL);
            a.heat_lnJ[pair] = 0.0;
        }
        return;
    }
    T part[2] = {(T)0, (T)0};  // ln det J_C, energy
    if (sizeof(T) == 4 && sd.vec == 4) heat_pass_smem<T, (sizeof(T) == 4 ? 4 : 2)>(sd, cfg, sJ, eps, part);
    else if (sd.hL % 2 == 0) heat_pass_smem<T, 2>(sd, cfg, sJ, eps, part);
    else heat_pass_smem<T, 1>(sd, cfg, sJ, eps, part);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_s2g(out, cfg, (unsigned)(n3 * (int)sizeof(T)));
        bulk_commit();
    }
    double tot[2];
    block_sum_exact<T, 2>(part, tot, red);
    if (threadIdx.x == 0) {
        a.heat_lnJ[pair] = tot[0];
        a.heat_H[pair] = tot[1];
        bulk_wait_read();
    }
}

// Asynchronous 16-byte global -> shared copies (cp.async, cache-global) of n
// elements by the whole CTA; complete after cp_async_wait_all.
template <typename T>
__device__ __forceinline__ void sx_prefetch(T* dst, const T* src, int n) {
    constexpr int VW = 16 / sizeof(T);
    for (int q = threadIdx.x * VW; q < n; q += blockDim.x * VW) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + q) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The pair walk of one chain.  Slot A holds s1 (the configuration now at
// beta_i), slot F receives f1 = C(s1).  Accept: the heated configuration of
// beta_{i+1} is final at beta_i; it belongs in s1's buffer, and the walk
// only records that (commit[pair] = that buffer; k_heat_commit copies all
// accepted proposals afterwards, in parallel, since no later pair reads a
// configuration whose temperature is final); f1 moves on as the next s1 (to
// be written into s2's buffer).  Reject: s1 is final (written back if it was
// transformed earlier in this update) and s2 moves on as the next s1.  With
// room for a third slot G, s2 is fetched into it asynchronously while s1 is
// cooled, so no pair waits on global memory.  Buffer identities never
// change; only contents, labels and energies do.
template <typename T>
__global__ void __launch_bounds__(SX_THREADS, 1) k_exchange_coolheat_smem(DevBatch a, int three_slots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SxSmem sm;
    __shared__ PairDraws<SX_MAX_NT> pd;
    __shared__ double pHH[SX_MAX_NT], pLJ[SX_MAX_NT], pbeta[SX_MAX_NT];  // per pair / replica
    const int ch = blockIdx.x;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    const int NT = sd.NT, half = sd.half, n3 = 6 * half;
    T* const slots = reinterpret_cast<T*>(smem_raw);
    auto slot = [&](int q) { return slots + (size_t)q * n3; };
    const unsigned long long step = *a.d_step;
    pd.load(a.seed, (uint32_t)cd.s, (uint32_t)cd.copy, step, NT - 1);
    for (int q = (int)threadIdx.x; q < NT; q += (int)blockDim.x) {
        pbeta[q] = a.betas[sd.beta_off + q];
        if (q + 1 < NT) {
            pHH[q] = a.heat_H[cd.pair_off + q];
            pLJ[q] = a.heat_lnJ[cd.pair_off + q];
        }
    }
    sx_load_state(a, cd, NT, sm);  // its barrier also publishes the tables above
    T* pool = (T*)a.spins + a.chain_off[ch];
    const float* J0 = a.J + sd.J_off;
    const float* J1 = a.J + sd.J_off + 3 * half;
    const bool v2 = (sd.hL % 2) == 0;
    int A = 0, F = 1, G = 2;  // slots of s1, of C(s1), of the prefetched s2
    int ownerA = sm.buf[0];   // global buffer of s1
    bool dirtyA = false;
    sx_copy(slot(A), pool + (long long)ownerA * n3, n3);
    __syncthreads();
    for (int i = 0; i + 1 < NT; ++i) {
        const int ownerB = sm.buf[i + 1];
        if (three_slots) sx_prefetch(slot(G), pool + (long long)ownerB * n3, n3);
        const T eps = (T)a.eps[sd.eps_off + i];
        const T* s1 = slot(A);
        T* f1 = slot(F);
        T part[2] = {(T)0, (T)0};  // ln det J_C(s1), energy of C(s1)
        T none = (T)0;
        if (v2) ch_colour<T, 2, true, false>(sd, s1, s1, f1, J0, J1, 0, eps, part[0], none);
        else ch_colour<T, 1, true, false>(sd, s1, s1, f1, J0, J1, 0, eps, part[0], none);
        __syncthreads();
        if (v2) ch_colour<T, 2, true, true>(sd, f1, s1, f1, J0, J1, 1, eps, part[0], part[1]);
        else ch_colour<T, 1, true, true>(sd, f1, s1, f1, J0, J1, 1, eps, part[0], part[1]);
        double tot[2];
        block_sum_exact<T, 2>(part, tot, sm.red);
        const long long pair = cd.pair_off + i;
        if (threadIdx.x == 0) {
            const double LJ1 = tot[0], HC = tot[1];
            const double HH = pHH[i], LJ2 = pLJ[i];
            const double b1 = pbeta[i], b2 = pbeta[i + 1];
            const double lnA = -b2 * HC - b1 * HH + b1 * sm.H[i] + b2 * sm.H[i + 1] + LJ1 - LJ2;
            xlog_write(a, pair, lnA, LJ1, LJ2);
            const bool ok = accept_lnu(lnA, pd.lnu[i]);
            sm.flag = ok;
            a.heat_commit[pair] = ok ? ownerA : -1;
            if (ok) {
                pd.acc[i] = 1;
                sm.H[i] = HH;
                sm.H[i + 1] = HC;
                const int t = sm.lab[i]; sm.lab[i] = sm.lab[i + 1]; sm.lab[i + 1] = t;
            }
        }
        __syncthreads();
        if (sm.flag) {
            // C^-1(s2) is final at beta_i (committed later); C(s1) moves on
            const int t = A; A = F; F = t;
            dirtyA = true;
        } else {
            // s1 is final at beta_i; s2 moves on
            if (dirtyA) sx_copy(pool + (long long)ownerA * n3, slot(A), n3);
            if (three_slots) {
                const int t = A; A = G; G = t;
            } else {
                sx_copy(slot(F), pool + (long long)ownerB * n3, n3);
                const int t = A; A = F; F = t;
            }
            dirtyA = false;
        }
        ownerA = ownerB;
        if (three_slots) cp_async_wait_all();
        __syncthreads();
    }
    if (dirtyA) sx_copy(pool + (long long)ownerA * n3, slot(A), n3);
    sx_store_state(a, cd, NT, sm, ch);
    pd.store(a.prop + cd.pair_off, a.acc + cd.pair_off, NT - 1);
}

// Accepted heated proposals into the buffers the walk recorded: block
// (chain, pair), commit[pair] >= 0 names the chain's buffer.
template <typename T>
__global__ void __launch_bounds__(HP_THREADS) k_heat_commit(DevBatch a) {
    const int ch = blockIdx.x, i = blockIdx.y;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    if (i + 1 >= sd.NT) return;
    const long long pair = cd.pair_off + i;
    const int target = a.heat_commit[pair];
    if (target < 0) return;
    const int n3 = 6 * sd.half;
    sx_copy((T*)a.spins + a.chain_off[ch] + (long long)target * n3,
            (const T*)a.heat_buf + pair * (6LL * a.max_half), n3);
}

// ---------------------------------------------------------------------------
// Decimation: slots hold s1 (at beta_i) and s2 (at beta_{i+1}).  Accept: the
// kept colours change temperature, the decimated colour of both is redrawn
// at the new beta; s2 is then final at beta_i (written back), s1 moves on to
// beta_{i+1}.  Reject: s1 is final (written back if re-inserted earlier), s2
// moves on.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SX_THREADS, 1) k_exchange_decimation_smem(DevBatch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SxSmem sm;
    __shared__ DecimPairs<T, SX_MAX_NT> dp;
    __shared__ PairDraws<SX_MAX_NT> pd;
    const int ch = blockIdx.x;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    const int NT = sd.NT, half = sd.half, n3 = 6 * half;
    T* const slots = reinterpret_cast<T*>(smem_raw);
    auto slot = [&](int q) { return slots + (size_t)q * n3; };
    const unsigned long long step = *a.d_step;
    dp.load(a.betas + sd.beta_off, NT);  // both visible after sx_load_state's barrier
    pd.load(a.seed, (uint32_t)cd.s, (uint32_t)cd.copy, step, NT - 1);
    sx_load_state(a, cd, NT, sm);
    T* pool = (T*)a.spins + a.chain_off[ch];
    const uint4 wd = rng_words(a.seed, (uint32_t)cd.s, 0u, (uint32_t)cd.copy, step, 3u);
    const int d0 = (int)(wd.x & 1u);
    int A = 0;
    int ownerA = sm.buf[0];
    bool dirtyA = false;
    sx_copy(slot(A), pool + (long long)ownerA * n3, n3);
    for (int i = 0; i + 1 < NT; ++i) {
        const int B = 1 - A;
        const int ownerB = sm.buf[i + 1];
        sx_copy(slot(B), pool + (long long)ownerB * n3, n3);
        __syncthreads();
        const int d = (d0 + i) & 1;
        const T b1t = dp.b[i], b2t = dp.b[i + 1], dbt = dp.db[i], lr = dp.lr[i];
        const float* Jd = a.J + sd.J_off + d * 3 * half;
        const float* Jk = a.J + sd.J_off + (1 - d) * 3 * half;
        T* c1 = slot(A);
        T* c2 = slot(B);
        T part[1] = {(T)0};
        for (int h = threadIdx.x; h < half; h += blockDim.x) {
            const Site st = site_of(sd, d, h);
            const V3<T> S1 = local_field<T>(st, half, c1 + (1 - d) * 3 * half, Jd, Jk);
            const V3<T> S2 = local_field<T>(st, half, c2 + (1 - d) * 3 * half, Jd, Jk);
            const T na = M<T>::sqrt_(dot(S1, S1)), nb = M<T>::sqrt_(dot(S2, S2));
            part[0] += sx_decim_D<T>(na, b1t, b2t, dbt, lr) - sx_decim_D<T>(nb, b1t, b2t, dbt, lr);
        }
        double tot1[1];
        block_sum_exact<T, 1>(part, tot1, sm.red);
        const double lnA = tot1[0];
        if (threadIdx.x == 0) {
            xlog_write(a, cd.pair_off + i, lnA, 0.0, 0.0);
            const bool ok = accept_lnu(lnA, pd.lnu[i]);
            sm.flag = ok;
            if (ok) {
                pd.acc[i] = 1;
                sm.buf[i] = ownerB;
                sm.buf[i + 1] = ownerA;
                const int t = sm.lab[i]; sm.lab[i] = sm.lab[i + 1]; sm.lab[i + 1] = t;
            }
        }
        __syncthreads();
        if (sm.flag) {
            // c2 now at b1 (replica id of index i), c1 at b2 (index i+1)
            T e12[2] = {(T)0, (T)0};
            const uint32_t id1 = (uint32_t)(cd.copy * NT + i), id2 = id1 + 1u;
            for (int h = threadIdx.x; h < half; h += blockDim.x) {
                const Site st = site_of(sd, d, h);
                const V3<T> Sa = local_field<T>(st, half, c2 + (1 - d) * 3 * half, Jd, Jk);
                const uint4 w1 = rng_words(a.seed, (uint32_t)cd.s, (uint32_t)st.x, id1, step, 2u);
                const V3<T> sa = hb_site<T>(b1t, Sa, w1.x, w1.y);
                st3(c2 + d * 3 * half, half, h, sa);
                e12[0] -= dot(sa, Sa);
                const V3<T> Sb = local_field<T>(st, half, c1 + (1 - d) * 3 * half, Jd, Jk);
                const uint4 w2 = rng_words(a.seed, (uint32_t)cd.s, (uint32_t)st.x, id2, step, 2u);
                const V3<T> sb = hb_site<T>(b2t, Sb, w2.x, w2.y);
                st3(c1 + d * 3 * half, half, h, sb);
                e12[1] -= dot(sb, Sb);
            }
            double E[2];
            block_sum_exact<T, 2>(e12, E, sm.red);
            if (threadIdx.x == 0) {
                sm.H[i] = E[0];
                sm.H[i + 1] = E[1];
            }
            __syncthreads();
            sx_copy(pool + (long long)ownerB * n3, c2, n3);  // final at b1
            // c1 stays in slot A, now at b2, owned by its own buffer, modified
            dirtyA = true;
        } else {
            if (dirtyA) sx_copy(pool + (long long)ownerA * n3, c1, n3);
            A = B;
            ownerA = ownerB;
            dirtyA = false;
        }
        __syncthreads();
    }
    if (dirtyA) sx_copy(pool + (long long)ownerA * n3, slot(A), n3);
    sx_store_state(a, cd, NT, sm, ch);
    pd.store(a.prop + cd.pair_off, a.acc + cd.pair_off, NT - 1);
}

// Two slots of one configuration each (s1 and its transform, or the pair).
size_t exchange_smem_bytes(int mode, int half, bool fp64) { return (size_t)2 * 6 * half * (fp64 ? 8 : 4); }

// A third slot for the cooling/heating walk's prefetch where it fits beside
// the static tables (about 30 KB) in a CTA's 227 KB.
static bool coolheat_three_slots(int half, bool fp64) {
    return (size_t)3 * 6 * half * (fp64 ? 8 : 4) <= 192 * 1024;
}

bool exchange_smem_supported(int mode, int max_half, bool fp64) {
    // dynamic slots plus about 30 KB of static per-chain tables within the 227 KB of a CTA
    return (mode == 1 || mode == 2) && exchange_smem_bytes(mode, max_half, fp64) <= 196 * 1024;
}

cudaError_t launch_exchange_smem(const DevBatch& b, bool fp64, int mode, int max_half, cudaStream_t st) {
    const size_t smem = exchange_smem_bytes(mode, max_half, fp64);
    cudaError_t e;
    if (mode == 2) {
        if (!b.heat_buf) return cudaErrorInvalidValue;  // the engine allocates it whenever this path exists
        const dim3 grid_pre((unsigned)b.n_chains, (unsigned)(b.max_NT - 1), 1);
        const int three = coolheat_three_slots(max_half, fp64) ? 1 : 0;
        const size_t smem_w = three ? smem / 2 * 3 : smem;
        // configuration and couplings of the largest sample: 6 half (size of T + 4) bytes,
        // within one CTA wherever two configurations fit the walk's slots
        const size_t smem_pre = (size_t)6 * max_half * ((fp64 ? 8 : 4) + 4);
        if (fp64) {
            e = ensure_smem((const void*)k_heat_pre_smem<double>, smem_pre);
            if (e != cudaSuccess) return e;
            k_heat_pre_smem<double><<<grid_pre, HS_THREADS, smem_pre, st>>>(b);
            e = ensure_smem((const void*)k_exchange_coolheat_smem<double>, smem_w);
            if (e != cudaSuccess) return e;
            k_exchange_coolheat_smem<double><<<b.n_chains, SX_THREADS, smem_w, st>>>(b, three);
            k_heat_commit<double><<<grid_pre, HP_THREADS, 0, st>>>(b);
        } else {
            e = ensure_smem((const void*)k_heat_pre_smem<float>, smem_pre);
            if (e != cudaSuccess) return e;
            k_heat_pre_smem<float><<<grid_pre, HS_THREADS, smem_pre, st>>>(b);
            e = ensure_smem((const void*)k_exchange_coolheat_smem<float>, smem_w);
            if (e != cudaSuccess) return e;
            k_exchange_coolheat_smem<float><<<b.n_chains, SX_THREADS, smem_w, st>>>(b, three);
            k_heat_commit<float><<<grid_pre, HP_THREADS, 0, st>>>(b);
        }
    } else {
        if (fp64) {
            e = ensure_smem((const void*)k_exchange_decimation_smem<double>, smem);
            if (e != cudaSuccess) return e;
            k_exchange_decimation_smem<double><<<b.n_chains, SX_THREADS, smem, st>>>(b);
        } else {
            e = ensure_smem((const void*)k_exchange_decimation_smem<float>, smem);
            if (e != cudaSuccess) return e;
            k_exchange_decimation_smem<float><<<b.n_chains, SX_THREADS, smem, st>>>(b);
        }
    }
    return cudaGetLastError();
}

}  // namespace ptk
