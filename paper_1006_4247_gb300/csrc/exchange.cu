// exchange.cu -- tempering updates of Hasenbusch & Schaefer: the standard
// swap (section I, Eq. 1), the decimation swap (section III.A, Eq. aswap,
// appendix A) and the cooling/heating swap (section III.B).
//
// The pairs (b, b+1) of a chain are visited in increasing beta, each seeing
// the result of the previous one, so a chain is sequential in b.  The lattice
// work of a pair (decimated sums and re-insertion, cooling and heating
// sweeps) is spread over a thread-block cluster: every CTA of the cluster
// owns a contiguous slice of the sites of each colour and keeps its own copy
// of the chain's small state (temperature-to-buffer map, labels, energies,
// round-trip states) in shared memory.  Per pair each CTA reduces its partial
// sums, publishes them in its shared memory, and after the hardware cluster
// barrier reads every CTA's partials through distributed shared memory and
// adds them in rank order.  All CTAs therefore hold bit-identical sums, draw
// the same Philox uniform and take the same decision; there is no broadcast
// and no spin-wait.  Spins are exchanged through global memory (L2), made
// visible across the cluster by a fence before each cluster barrier.
#include <cooperative_groups.h>

#include "kernels.h"
#include "exchange_common.cuh"
#include "pt_device.cuh"

namespace cg = cooperative_groups;

namespace ptk {

constexpr int MAX_NT = 512;
constexpr int EX_THREADS = 512;
constexpr int HPX_THREADS = 256;  // k_decim_pre
constexpr int MAX_SUMS = 4;

struct ChainSmem {
    int buf[MAX_NT];
    int lab[MAX_NT];
    int rts[MAX_NT];
    double H[MAX_NT];
    double red[MAX_SUMS * 32];
    double slot[2][MAX_SUMS];  // published partials (double-buffered)
    double sum[MAX_SUMS];      // cluster totals, in rank order
    int flag2[2];              // decision of pair i in flag2[i & 1] (the decimation walk)
    int free0, free1;
};

__device__ void load_chain(const DevBatch& a, const ChainDesc& cd, int NT, ChainSmem& sm, int ch) {
    for (int b = threadIdx.x; b < NT; b += blockDim.x) {
        sm.buf[b] = a.bufmap[cd.r0 + b];
        sm.lab[b] = a.label[cd.r0 + b];
        sm.rts[b] = a.rt_state[cd.r0 + b];
        sm.H[b] = a.H[cd.r0 + b];
    }
    if (threadIdx.x == 0) {
        sm.free0 = a.freebuf[ch].x;
        sm.free1 = a.freebuf[ch].y;
    }
    __syncthreads();
}

// Round trips (section IV.B): a configuration that was at b = 0, then at
// b = NT-1, completes a trip when it is back at b = 0.
__device__ void roundtrip_update(ChainSmem& sm, int NT, long long* count) {
    const int top = sm.lab[0], bot = sm.lab[NT - 1];
    if (sm.rts[bot] == 1) sm.rts[bot] = 2;
    if (sm.rts[top] == 2) {
        *count += 1;
        sm.rts[top] = 1;
    } else if (sm.rts[top] == 0) {
        sm.rts[top] = 1;
    }
}

__device__ void store_chain(const DevBatch& a, const ChainDesc& cd, int NT, ChainSmem& sm, int ch) {
    __syncthreads();
    if (threadIdx.x == 0) roundtrip_update(sm, NT, &a.rt_count[ch]);
    __syncthreads();
    for (int b = threadIdx.x; b < NT; b += blockDim.x) {
        a.bufmap[cd.r0 + b] = sm.buf[b];
        a.label[cd.r0 + b] = sm.lab[b];
        a.rt_state[cd.r0 + b] = sm.rts[b];
        a.H[cd.r0 + b] = sm.H[b];
    }
    if (threadIdx.x == 0) a.freebuf[ch] = make_int2(sm.free0, sm.free1);
}

// Sum NV per-thread values over the CTA, then over the cluster in rank order;
// the totals land in sm.sum[] of every CTA.  Global writes made before the
// call are visible to the whole cluster after it.  `pub` counts publications
// (uniform over the cluster) and selects the slot.
template <typename T, int NV>
__device__ void cluster_sum(cg::cluster_group& cl, ChainSmem& sm, const T (&v)[NV], int& pub) {
    double tot[NV];
    block_sum_exact<T, NV>(v, tot, sm.red);
    const int slot = pub & 1;
    ++pub;
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) sm.slot[slot][k] = tot[k];
    __threadfence();
    cl.sync();
    if (threadIdx.x == 0) {
        const int n = (int)cl.num_blocks();
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += cl.map_shared_rank(&sm.slot[slot][0], r)[k];
            sm.sum[k] = s;
        }
    }
    __syncthreads();
}

// Contiguous slice [lo, hi) of n items for CTA `rank` of `cs`.
__device__ __forceinline__ void slice(int n, int rank, int cs, int& lo, int& hi) {
    lo = (int)(((long long)n * rank) / cs);
    hi = (int)(((long long)n * (rank + 1)) / cs);
}

// ---------------------------------------------------------------------------
// Standard swap: Delta = (b_{i+1} - b_i)(H_{i+1} - H_i) in double.  No
// lattice work: one warp per chain.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_exchange_plain(DevBatch a) {
    __shared__ ChainSmem sm;
    __shared__ PairDraws<MAX_NT> pd;
    const int ch = blockIdx.x;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    const int NT = sd.NT;
    pd.load(a.seed, (uint32_t)cd.s, (uint32_t)cd.copy, *a.d_step, NT - 1);
    load_chain(a, cd, NT, sm, ch);  // its barrier also publishes pd
    if (threadIdx.x == 0) {
        const double* beta = a.betas + sd.beta_off;
        for (int i = 0; i + 1 < NT; ++i) {
            const double lnA = (beta[i + 1] - beta[i]) * (sm.H[i + 1] - sm.H[i]);
            a.prop[cd.pair_off + i] += 1;
            xlog_write(a, cd.pair_off + i, lnA, 0.0, 0.0);
            if (accept_lnu(lnA, pd.lnu[i])) {
                a.acc[cd.pair_off + i] += 1;
                int t = sm.buf[i]; sm.buf[i] = sm.buf[i + 1]; sm.buf[i + 1] = t;
                t = sm.lab[i]; sm.lab[i] = sm.lab[i + 1]; sm.lab[i + 1] = t;
                const double th = sm.H[i]; sm.H[i] = sm.H[i + 1]; sm.H[i + 1] = th;
            }
        }
    }
    store_chain(a, cd, NT, sm, ch);
}

// D(n) = ln I(b2 n) - ln I(b1 n) for |S| = n.  With
// ln(sinh R / R) = R - ln(2R) + ln(1 - e^{-2R}) (appendix A) the large parts
// reduce to (b2 - b1) n - ln(b2/b1), which keeps float accuracy; below
// R = 1/2 the difference is taken directly.
template <typename T>
__device__ __forceinline__ T decim_D(T n, T b1, T b2, T db, T lr) {
    const T R1 = b1 * n, R2 = b2 * n;
    if (R1 >= (T)0.5)
        return db * n - lr + M<T>::log1p_(-M<T>::exp_((T)-2 * R2)) - M<T>::log1p_(-M<T>::exp_((T)-2 * R1));
    return ln_sinhc<T>(R2) - ln_sinhc<T>(R1);
}

// ---------------------------------------------------------------------------
// Decimation swap.  For pair i the decimated colour is d = (d0 + i) mod 2
// (d0 from purpose 3).  ln A = sum over decimated x of
// ln I(b2 S1) - ln I(b1 S1) + ln I(b1 S2) - ln I(b2 S2), S from the kept
// colour; per-site terms in T, sums in double.  On acceptance the buffers
// swap temperatures and the decimated colour of both is redrawn by heat bath
// at its new beta (purpose 2), which also yields the new energies.
// ---------------------------------------------------------------------------
template <typename T, int V>
__device__ __forceinline__ void decimation_chain(const DevBatch& a, cg::cluster_group& cl, ChainSmem& sm,
                                                 const DecimPairs<T, MAX_NT>& dp, PairDraws<MAX_NT>& pd,
                                                 const ChainDesc& cd, const SampleDesc& sd, int ch, int cs,
                                                 int rank);

template <typename T>
__global__ void __launch_bounds__(EX_THREADS, 2) k_exchange_decimation(DevBatch a) {
    __shared__ ChainSmem sm;
    __shared__ DecimPairs<T, MAX_NT> dp;
    __shared__ PairDraws<MAX_NT> pd;
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int ch = blockIdx.x / cs;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    const int NT = sd.NT, half = sd.half;
    dp.load(a.betas + sd.beta_off, NT);  // both visible after load_chain's barrier
    pd.load(a.seed, (uint32_t)cd.s, (uint32_t)cd.copy, *a.d_step, NT - 1);
    load_chain(a, cd, NT, sm, ch);
    if (sd.vec == 4) decimation_chain<T, (sizeof(T) == 4 ? 4 : 2)>(a, cl, sm, dp, pd, cd, sd, ch, cs, rank);
    else if (sd.vec == 2) decimation_chain<T, 2>(a, cl, sm, dp, pd, cd, sd, ch, cs, rank);
    else decimation_chain<T, 1>(a, cl, sm, dp, pd, cd, sd, ch, cs, rank);
    if (rank == 0) {
        store_chain(a, cd, NT, sm, ch);
        __syncthreads();  // thread 0's per-pair counts
        pd.store(a.prop + cd.pair_off, a.acc + cd.pair_off, NT - 1);
    }
    cl.sync();  // no CTA leaves while others may still read its shared memory
}

// Sum over the V-site vectors [lo, hi) of colour d (this thread's share) of
// D(|S|) = ln I(b2 |S|) - ln I(b1 |S|), S the field of config c's other colour.
template <typename T, int V>
__device__ __forceinline__ T decim_sum(const SampleDesc& sd, const T* c, const float* Jd, const float* Jk, int d,
                                       int lo, int hi, int tid, int nth, T b1t, T b2t, T dbt, T lr) {
    const int half = sd.half;
    T part = (T)0;
    for (int h0 = lo + tid * V; h0 < hi; h0 += nth * V) {
        const VRow q = vrow<V>(sd, d, h0);
        T S[3][V];
        nbr_field<T, V>(c + (1 - d) * 3 * half, Jd, Jk, half, h0, q.xs, q.hyp, q.hym, q.hzp, q.hzm, q.p, S);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T n = M<T>::sqrt_(S[0][v] * S[0][v] + S[1][v] * S[1][v] + S[2][v] * S[2][v]);
            part += decim_D<T>(n, b1t, b2t, dbt, lr);
        }
    }
    return part;
}

// The two halves of every pair's ln A that do not depend on the walk:
// T1 = sum over the decimated colour d_i of D(|S|) for the configuration at
// beta_i as the update found it, T2 the same for the one at beta_{i+1}
// (ln A = T1 - T2 when pair i-1 left beta_i's configuration alone, which
// pair i-1 does unless it accepted).  Block (chain, pair); stored in
// decim_pre[2 pair], [2 pair + 1].
template <typename T>
__global__ void __launch_bounds__(HPX_THREADS) k_decim_pre(DevBatch a) {
    __shared__ double red[2 * 32];
    const int ch = blockIdx.x, i = blockIdx.y;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    if (i + 1 >= sd.NT) return;  // uniform over the block
    const int half = sd.half, n3 = 6 * half;
    const uint4 wd = rng_words(a.seed, (uint32_t)cd.s, 0u, (uint32_t)cd.copy, *a.d_step, 3u);
    const int d = (int)((wd.x & 1u) + (uint32_t)i) & 1;
    const T* pool = (const T*)a.spins + a.chain_off[ch];
    const T* c1 = pool + (long long)a.bufmap[cd.r0 + i] * n3;
    const T* c2 = pool + (long long)a.bufmap[cd.r0 + i + 1] * n3;
    const float* Jd = a.J + sd.J_off + d * 3 * half;
    const float* Jk = a.J + sd.J_off + (1 - d) * 3 * half;
    // the walk's per-pair constants (DecimPairs), for this pair only, formed
    // in double by lane 0 of each warp and broadcast
    T k4[4] = {(T)0, (T)0, (T)0, (T)0};
    if ((threadIdx.x & 31u) == 0u) {
        const double b1 = a.betas[sd.beta_off + i], b2 = a.betas[sd.beta_off + i + 1];
        k4[0] = (T)b1;
        k4[1] = (T)b2;
        k4[2] = (T)(b2 - b1);
        k4[3] = b1 > 0.0 ? (T)log(b2 / b1) : (T)0;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) k4[m] = __shfl_sync(0xFFFFFFFFu, k4[m], 0);
    const T b1t = k4[0], b2t = k4[1], dbt = k4[2], lr = k4[3];
    T part[2];
    const int tid = (int)threadIdx.x, nth = (int)blockDim.x;
    constexpr int V4 = sizeof(T) == 4 ? 4 : 2;  // 16-byte rows
    if (sd.vec == 4) {
        part[0] = decim_sum<T, V4>(sd, c1, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
        part[1] = decim_sum<T, V4>(sd, c2, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
    } else if (sd.vec >= 2) {
        part[0] = decim_sum<T, 2>(sd, c1, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
        part[1] = decim_sum<T, 2>(sd, c2, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
    } else {
        part[0] = decim_sum<T, 1>(sd, c1, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
        part[1] = decim_sum<T, 1>(sd, c2, Jd, Jk, d, 0, half, tid, nth, b1t, b2t, dbt, lr);
    }
    double tot[2];
    block_sum_exact<T, 2>(part, tot, red);
    if (threadIdx.x == 0) {
        a.decim_pre[2 * (cd.pair_off + i)] = tot[0];
        a.decim_pre[2 * (cd.pair_off + i) + 1] = tot[1];
    }
}

// The pair walk of one chain; this CTA handles its slice of the V-site
// vectors (16-byte loads of the neighbour rows).  ln A of pair i is
// T1 - T2 (k_decim_pre) unless pair i-1 accepted: then the configuration now
// at beta_i is the one re-inserted at the end of pair i-1, whose kept colour
// (d_{i-1}) changed, and its T1 is summed right after the re-insertion.  A
// rejected pair therefore needs no lattice work and no cluster-wide step: all
// CTAs read the same T1, T2 and take the same decision.
template <typename T, int V>
__device__ __forceinline__ void decimation_chain(const DevBatch& a, cg::cluster_group& cl, ChainSmem& sm,
                                                 const DecimPairs<T, MAX_NT>& dp, PairDraws<MAX_NT>& pd,
                                                 const ChainDesc& cd, const SampleDesc& sd, int ch, int cs,
                                                 int rank) {
    const int NT = sd.NT, half = sd.half;
    int lo, hi;
    slice(half / V, rank, cs, lo, hi);  // in vectors
    lo *= V;
    hi *= V;
    int pub = 0;
    const unsigned long long step = *a.d_step;
    T* pool = (T*)a.spins + a.chain_off[ch];
    const double* pre = a.decim_pre + 2LL * cd.pair_off;
    const uint4 wd = rng_words(a.seed, (uint32_t)cd.s, 0u, (uint32_t)cd.copy, step, 3u);
    const int d0 = (int)(wd.x & 1u);
    bool fresh = true;  // the configuration at beta_i is the one the update started with
    double T1cur = 0.0;
    for (int i = 0; i + 1 < NT; ++i) {
        const int d = (d0 + i) & 1;
        const T b1t = dp.b[i], b2t = dp.b[i + 1];
        const float* Jd = a.J + sd.J_off + d * 3 * half;
        const float* Jk = a.J + sd.J_off + (1 - d) * 3 * half;
        if (threadIdx.x == 0) {
            const double lnA = (fresh ? pre[2 * i] : T1cur) - pre[2 * i + 1];
            if (rank == 0) xlog_write(a, cd.pair_off + i, lnA, 0.0, 0.0);
            const bool ok = accept_lnu(lnA, pd.lnu[i]);
            // by pair parity: after a rejection no barrier separates this
            // write from other warps' read of the previous pair's decision
            sm.flag2[i & 1] = ok;
            if (ok) {
                pd.acc[i] = 1;
                int t = sm.buf[i]; sm.buf[i] = sm.buf[i + 1]; sm.buf[i + 1] = t;
                t = sm.lab[i]; sm.lab[i] = sm.lab[i + 1]; sm.lab[i + 1] = t;
            }
        }
        __syncthreads();
        const bool accepted = sm.flag2[i & 1] != 0;
        fresh = !accepted;
        if (accepted) {
            T e[2] = {(T)0, (T)0};
            T* n1 = pool + (long long)sm.buf[i] * (6LL * half);      // now at b1
            T* n2 = pool + (long long)sm.buf[i + 1] * (6LL * half);  // now at b2
            const uint32_t id1 = (uint32_t)(cd.copy * NT + i), id2 = id1 + 1u;
            for (int h0 = lo + (int)threadIdx.x * V; h0 < hi; h0 += (int)blockDim.x * V) {
                const VRow q = vrow<V>(sd, d, h0);
#pragma unroll
                for (int which = 0; which < 2; ++which) {
                    T* nb_ = which ? n2 : n1;
                    const T bt = which ? b2t : b1t;
                    const uint32_t id = which ? id2 : id1;
                    T S[3][V];
                    nbr_field<T, V>(nb_ + (1 - d) * 3 * half, Jd, Jk, half, h0, q.xs, q.hyp, q.hym, q.hzp, q.hzm,
                                    q.p, S);
                    T out[3][V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
                        const uint32_t x = (uint32_t)(2 * (q.ih0 + v) + q.p + sd.L * q.row);
                        const uint4 w = rng_words(a.seed, (uint32_t)cd.s, x, id, step, 2u);
                        const V3<T> sv = hb_site<T>(bt, Sv, w.x, w.y);
                        out[0][v] = sv.x; out[1][v] = sv.y; out[2][v] = sv.z;
                        e[which] -= dot(sv, Sv);
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) stv<T, V>(nb_ + d * 3 * half + c * half + h0, out[c]);
                }
            }
            cluster_sum<T, 2>(cl, sm, e, pub);  // also makes the re-inserted spins visible to the cluster
            if (threadIdx.x == 0) {
                sm.H[i] = sm.sum[0];
                sm.H[i + 1] = sm.sum[1];
            }
            if (i + 2 < NT) {
                // T1 of pair i+1: its decimated colour is 1 - d, the kept colour d was just redrawn
                const int dn = 1 - d;
                const float* Jdn = a.J + sd.J_off + dn * 3 * half;
                const float* Jkn = a.J + sd.J_off + d * 3 * half;
                T part[1] = {decim_sum<T, V>(sd, n2, Jdn, Jkn, dn, lo, hi, (int)threadIdx.x, (int)blockDim.x,
                                             dp.b[i + 1], dp.b[i + 2], dp.db[i + 1], dp.lr[i + 1])};
                cluster_sum<T, 1>(cl, sm, part, pub);
                T1cur = sm.sum[0];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Cooling/heating swap of pair (b1 < b2) with configurations s1 (at b1) and
// s2 (at b2): s1 is cooled (colour 0 then colour 1) into scratch buffer f1
// and proposed at b2; s2 is heated (colour 1 then colour 0, each the inverse
// step) into scratch buffer f2 and proposed at b1.  The map is an
// involution, so
//   ln A = -b2 H[C s1] - b1 H[C^-1 s2] + b1 H[s1] + b2 H[s2]
//          + ln det J_C(s1) - ln det J_C(C^-1 s2).
// On acceptance the scratch buffers take the two temperatures and the old
// buffers become scratch; nothing is copied.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(EX_THREADS) k_exchange_coolheat(DevBatch a) {
    __shared__ ChainSmem sm;
    __shared__ PairDraws<MAX_NT> pd;
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int ch = blockIdx.x / cs;
    const ChainDesc cd = a.chains[ch];
    const SampleDesc& sd = a.samples[cd.s];
    const int NT = sd.NT, half = sd.half;
    pd.load(a.seed, (uint32_t)cd.s, (uint32_t)cd.copy, *a.d_step, NT - 1);
    load_chain(a, cd, NT, sm, ch);  // its barrier also publishes pd
    int lo, hi;
    slice(half, rank, cs, lo, hi);
    int pub = 0;
    const double* beta = a.betas + sd.beta_off;
    T* pool = (T*)a.spins + a.chain_off[ch];
    const float* J0 = a.J + sd.J_off;
    const float* J1 = a.J + sd.J_off + 3 * half;
    const long long rep = 6LL * half;
    for (int i = 0; i + 1 < NT; ++i) {
        const double b1 = beta[i], b2 = beta[i + 1];
        const T eps = (T)a.eps[sd.eps_off + i];
        const T* s1 = pool + (long long)sm.buf[i] * rep;
        const T* s2 = pool + (long long)sm.buf[i + 1] * rep;
        T* f1 = pool + (long long)sm.free0 * rep;
        T* f2 = pool + (long long)sm.free1 * rep;
        // ln J_C(s1), ln J_C(C^-1 s2), H[C s1], H[C^-1 s2] (threads may hold
        // many sites: two-sum accumulation, v + vc)
        T v[4] = {(T)0, (T)0, (T)0, (T)0}, vc[4] = {(T)0, (T)0, (T)0, (T)0};
        // phase 1: cool colour 0 of s1 (neighbours: s1 colour 1);
        //          heat colour 1 of s2 (neighbours: s2 colour 0)
        for (int h = lo + (int)threadIdx.x; h < hi; h += blockDim.x) {
            const Site st0 = site_of(sd, 0, h);
            const V3<T> S = local_field<T>(st0, half, s1 + 3 * half, J0, J1);
            V3<T> s = ld3(s1, half, h);
            acc_add(v[0], vc[0], cool_site<T>(eps, S, s));
            st3(f1, half, h, s);
            const Site st1 = site_of(sd, 1, h);
            const V3<T> S2 = local_field<T>(st1, half, s2, J1, J0);
            V3<T> u = ld3(s2 + 3 * half, half, h);
            acc_add(v[1], vc[1], heat_site<T>(eps, S2, u));
            st3(f2 + 3 * half, half, h, u);
        }
        __threadfence();
        cl.sync();
        // phase 2: cool colour 1 of s1 (neighbours: cooled colour 0 in f1);
        //          heat colour 0 of s2 (neighbours: heated colour 1 in f2)
        for (int h = lo + (int)threadIdx.x; h < hi; h += blockDim.x) {
            const Site st1 = site_of(sd, 1, h);
            const V3<T> S = local_field<T>(st1, half, f1, J1, J0);
            V3<T> s = ld3(s1 + 3 * half, half, h);
            acc_add(v[0], vc[0], cool_site<T>(eps, S, s));
            st3(f1 + 3 * half, half, h, s);
            acc_add(v[2], vc[2], -dot(s, S));
            const Site st0 = site_of(sd, 0, h);
            const V3<T> S2 = local_field<T>(st0, half, f2 + 3 * half, J0, J1);
            V3<T> u = ld3(s2, half, h);
            acc_add(v[1], vc[1], heat_site<T>(eps, S2, u));
            st3(f2, half, h, u);
            acc_add(v[3], vc[3], -dot(u, S2));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += vc[k];
        cluster_sum<T, 4>(cl, sm, v, pub);
        if (threadIdx.x == 0) {
            const double LJ1 = sm.sum[0], LJ2 = sm.sum[1], HC = sm.sum[2], HH = sm.sum[3];
            const double lnA = -b2 * HC - b1 * HH + b1 * sm.H[i] + b2 * sm.H[i + 1] + LJ1 - LJ2;
            const bool ok = accept_lnu(lnA, pd.lnu[i]);
            if (rank == 0) {
                a.prop[cd.pair_off + i] += 1;
                if (ok) a.acc[cd.pair_off + i] += 1;
                xlog_write(a, cd.pair_off + i, lnA, LJ1, LJ2);
            }
            if (ok) {
                const int o1 = sm.buf[i], o2 = sm.buf[i + 1];
                sm.buf[i] = sm.free1;      // C^-1(s2) at b1
                sm.buf[i + 1] = sm.free0;  // C(s1) at b2
                sm.free0 = o1;
                sm.free1 = o2;
                sm.H[i] = HH;
                sm.H[i + 1] = HC;
                const int t = sm.lab[i]; sm.lab[i] = sm.lab[i + 1]; sm.lab[i + 1] = t;
            }
        }
        __syncthreads();
    }
    if (rank == 0) store_chain(a, cd, NT, sm, ch);
    cl.sync();  // no CTA leaves while others may still read its shared memory
}

// Cluster size per chain: enough CTAs to cover the SMs at least once, a
// power of two <= 8, and at least 64 sites of each colour per CTA.
static int cluster_size(const DevBatch& b) {
    int cs = 1;
    while (cs < 8 && b.n_chains * cs < b.n_sm && b.min_half / (2 * cs) >= 64) cs *= 2;
    return cs;
}

template <typename K>
static cudaError_t launch_cluster(K kernel, const DevBatch& b, int cs, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.n_chains * cs);
    cfg.blockDim = dim3(EX_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, b);
}

int exchange_launch_count(const DevBatch& b, bool fp64, int mode) {
    // the staged cooling/heating: heating pre-pass, walk, commit of the accepted proposals
    if (mode == 2 && b.exchange_impl != 1 && exchange_smem_supported(mode, b.max_half, fp64)) return 3;
    // the cluster decimation walk runs after the pre-pass of its sums
    if (mode == 1 && !(b.exchange_impl != 1 && exchange_smem_supported(mode, b.max_half, fp64))) return 2;
    return 1;
}

cudaError_t launch_exchange(const DevBatch& b, bool fp64, int mode, cudaStream_t st) {
    if (mode == 0) {
        k_exchange_plain<<<b.n_chains, 32, 0, st>>>(b);
        return cudaGetLastError();
    }
    if (b.exchange_impl != 1 && exchange_smem_supported(mode, b.max_half, fp64))
        return launch_exchange_smem(b, fp64, mode, b.max_half, st);
    const int cs = b.exchange_cluster > 0 ? b.exchange_cluster : cluster_size(b);
    cudaError_t e;
    if (mode == 1) {
        const dim3 grid_pairs((unsigned)b.n_chains, (unsigned)(b.max_NT - 1), 1);
        if (fp64) k_decim_pre<double><<<grid_pairs, HPX_THREADS, 0, st>>>(b);
        else k_decim_pre<float><<<grid_pairs, HPX_THREADS, 0, st>>>(b);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = fp64 ? launch_cluster(k_exchange_decimation<double>, b, cs, st)
                 : launch_cluster(k_exchange_decimation<float>, b, cs, st);
    }
    else
        e = fp64 ? launch_cluster(k_exchange_coolheat<double>, b, cs, st)
                 : launch_cluster(k_exchange_coolheat<float>, b, cs, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace ptk
