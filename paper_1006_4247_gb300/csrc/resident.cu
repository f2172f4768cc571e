// resident.cu -- whole update block (n_hb heat-bath + n_or overrelaxation
// sweeps, section III.C / section IV of Hasenbusch & Schaefer) of one replica
// inside one CTA, with the replica held in shared memory.
//
// For small lattices a replica fits on chip (L = 16: 4096 sites x 12 B =
// 48 KB in float), so instead of 2 (n_hb + n_or) passes over HBM the block is
// read once (TMA bulk copies), all half sweeps run out of shared memory with a
// CTA barrier between colours, and the result is written once (one bulk copy).  The energy of the final
// configuration is reduced during the last half sweep (every bond has exactly
// one colour-1 end) and written straight to H[r].
//
// Thread mapping inside a half sweep is the one of the streaming kernel
// (V = 4 consecutive sites of one row per thread, aligned float4 shared-memory
// loads, +-x neighbours from the same vector shifted by one plus one wrapped
// element).  The sample's couplings (12 B per site) are staged in shared
// memory beside the replica, so no half sweep waits on L2: L = 16 takes
// 48 + 48 KB, two CTAs of 512 threads per SM.
#include <cooperative_groups.h>

#include "kernels.h"
#include "pt_device.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace ptk {

constexpr int RES_THREADS = 512;

// ENERGY (compile time, only the block's last half sweep) also returns the
// thread's share of H in the spin precision: a few sites per thread, so at
// most a few float terms meet before the block adds the shares exactly
// (block_sum_exact).
template <typename T, int V, int KIND, bool ENERGY>
__device__ __forceinline__ T res_halfsweep(T* __restrict__ sm, const float* __restrict__ J, const SampleDesc& sd,
                                           int color, T beta, unsigned long long seed, uint32_t sample,
                                           uint32_t rep_id, unsigned long long step) {
    const int half = sd.half, hL = sd.hL, L = sd.L;
    T* own = sm + color * 3 * half;
    const T* oth = sm + (1 - color) * 3 * half;
    const float* Jown = J + color * 3 * half;
    const float* Joth = J + (1 - color) * 3 * half;
    T e = (T)0;
    for (int h0 = (int)threadIdx.x * V; h0 < half; h0 += RES_THREADS * V) {
        const int row = (int)fdiv((uint32_t)h0, sd.div_hL);
        const int ih0 = h0 - row * hL;
        const int k = (int)fdiv((uint32_t)row, sd.div_L);
        const int j = row - k * L;
        const int p = (j + k + color) & 1;
        const int rb = row * hL;
        const int xs = p ? rb + ((ih0 + V == hL) ? 0 : ih0 + V) : rb + ((ih0 == 0) ? hL - 1 : ih0 - 1);
        const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
        const int kp = (k + 1 == L) ? 0 : k + 1, km = (k == 0) ? L - 1 : k - 1;
        const int hyp = ih0 + hL * (jp + L * k), hym = ih0 + hL * (jm + L * k);
        const int hzp = ih0 + hL * (j + L * kp), hzm = ih0 + hL * (j + L * km);

        T S[3][V];
        nbr_field<T, V, true>(oth, Jown, Joth, half, h0, xs, hyp, hym, hzp, hzm, p, S);

        T s[3][V];
        if (KIND == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ldv<T, V>(own + c * half + h0, s[c]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv;
            if (KIND == 1) {
                const int x = 2 * (ih0 + v) + p + L * row;
                const uint4 w = rng_words(seed, sample, (uint32_t)x, rep_id, step, 0u);
                sv = hb_site<T>(beta, Sv, w.x, w.y);
            } else {
                sv = {s[0][v], s[1][v], s[2][v]};
                or_site(Sv, sv);
            }
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
            if (ENERGY) e -= dot(sv, Sv);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<T, V>(own + c * half + h0, s[c]);
    }
    return e;
}

// Row indices of a thread's vector h0 (the same for both colours except the
// checkerboard offset and the wrapped x neighbour).
struct VecIdx {
    int h0, xs0, xs1, hyp, hym, hzp, hzm, p0;
};

// Source lanes of the wrapped x neighbour when a warp holds whole rows of
// n = hL / V vectors: the next vector's lane (p = 1) or the previous one's
// (p = 0), wrapping within the row.
template <int V>
__device__ __forceinline__ void xs_lanes(int hL, int ih0, int& right, int& left) {
    const int lane = (int)(threadIdx.x & 31u), n = hL / V, m = ih0 / V;  // m: vector index in the row
    right = (m == n - 1) ? lane - (n - 1) : lane + 1;
    left = (m == 0) ? lane + (n - 1) : lane - 1;
}

template <int V>
__device__ __forceinline__ VecIdx vec_idx(const SampleDesc& sd, int h0, bool xshfl) {
    const int hL = sd.hL, L = sd.L;
    VecIdx q;
    q.h0 = h0;
    const int row = (int)fdiv((uint32_t)h0, sd.div_hL);
    const int ih0 = h0 - row * hL;
    const int k = (int)fdiv((uint32_t)row, sd.div_L);
    const int j = row - k * L;
    q.p0 = (j + k) & 1;
    const int rb = row * hL;
    int left = rb + ((ih0 == 0) ? hL - 1 : ih0 - 1), right = rb + ((ih0 + V == hL) ? 0 : ih0 + V);
    if (xshfl) xs_lanes<V>(hL, ih0, right, left);  // lanes instead of indices
    q.xs0 = q.p0 ? right : left;   // colour 0: p = p0
    q.xs1 = q.p0 ? left : right;   // colour 1: p = 1 - p0
    const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
    const int kp = (k + 1 == L) ? 0 : k + 1, km = (k == 0) ? L - 1 : k - 1;
    q.hyp = ih0 + hL * (jp + L * k);
    q.hym = ih0 + hL * (jm + L * k);
    q.hzp = ih0 + hL * (j + L * kp);
    q.hzm = ih0 + hL * (j + L * km);
    return q;
}

// Overrelaxation half sweep when every thread owns at most one vector of a
// colour (half <= threads * V): the indices come precomputed.
template <typename T, int V, bool ENERGY, bool XSHFL>
__device__ __forceinline__ T res_or_one(T* __restrict__ sm, const float* __restrict__ J, int half, int color,
                                        const VecIdx& q) {
    T e = (T)0;
    if (q.h0 < half) {
        T* own = sm + color * 3 * half;
        const T* oth = sm + (1 - color) * 3 * half;
        const float* Jown = J + color * 3 * half;
        const float* Joth = J + (1 - color) * 3 * half;
        const int p = q.p0 ^ color;
        const int xs = color ? q.xs1 : q.xs0;
        T S[3][V];
        nbr_field<T, V, true, XSHFL>(oth, Jown, Joth, half, q.h0, xs, q.hyp, q.hym, q.hzp, q.hzm, p, S);
        T s[3][V];
#pragma unroll
        for (int c = 0; c < 3; ++c) ldv<T, V>(own + c * half + q.h0, s[c]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv = {s[0][v], s[1][v], s[2][v]};
            or_site(Sv, sv);
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
            if (ENERGY) e -= dot(sv, Sv);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<T, V>(own + c * half + q.h0, s[c]);
    }
    return e;
}

// The sweep block of one replica (the CTA's replica is held in `sm`).  Heat-
// bath half sweeps run on the same V-site vectors as the overrelaxation ones
// (vector loads, row indices once per vector; the draws and arithmetic per
// site are unchanged).
template <typename T, int V>
__device__ __forceinline__ T res_block(T* sm, const float* J, const DevBatch& a, const SampleDesc& sd,
                                       const int4& rd, int n_hb, int n_or) {
    const T beta = (T)a.betas[sd.beta_off + rd.z];
    const unsigned long long step0 = *a.d_step;
    const int total = 2 * (n_hb + n_or);
    T e = (T)0;
    int kstep = 0;
    for (int hb = 0; hb < n_hb; ++hb)
        for (int c = 0; c < 2; ++c, ++kstep) {
            const unsigned long long st = step0 + (unsigned long long)kstep;
            if (kstep == total - 1)
                e = res_halfsweep<T, V, 1, true>(sm, J, sd, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w, st);
            else
                res_halfsweep<T, V, 1, false>(sm, J, sd, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w, st);
            __syncthreads();
        }
    if (sd.half <= RES_THREADS * V) {
        // whole rows per warp and every lane active: wrapped x neighbours by shuffle
        const bool xsh = (32 % (sd.hL / V) == 0) && ((sd.half / V) % 32 == 0);
        const VecIdx q = vec_idx<V>(sd, (int)threadIdx.x * V, xsh);
        for (int o = 0; o < n_or; ++o)
            for (int c = 0; c < 2; ++c, ++kstep) {
                if (xsh) {
                    if (kstep == total - 1) e = res_or_one<T, V, true, true>(sm, J, sd.half, c, q);
                    else res_or_one<T, V, false, true>(sm, J, sd.half, c, q);
                } else {
                    if (kstep == total - 1) e = res_or_one<T, V, true, false>(sm, J, sd.half, c, q);
                    else res_or_one<T, V, false, false>(sm, J, sd.half, c, q);
                }
                __syncthreads();
            }
        return e;
    }
    for (int o = 0; o < n_or; ++o)
        for (int c = 0; c < 2; ++c, ++kstep) {
            if (kstep == total - 1)
                e = res_halfsweep<T, V, 0, true>(sm, J, sd, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w, 0ull);
            else
                res_halfsweep<T, V, 0, false>(sm, J, sd, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w, 0ull);
            __syncthreads();
        }
    return e;
}

// One CTA per replica of a resident sample (a.res_reps).  The sample's row
// width decides the vector width (4 or 2 sites per thread in float, 2 in
// double); the overrelaxation count is per sample when a.nor_s is given.
template <typename T>
__global__ void __launch_bounds__(RES_THREADS, 2) k_resident(DevBatch a, int n_hb, int n_or) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[32];
    __shared__ __align__(8) unsigned long long io_bar;
    const int r = a.res_reps[a.rcl_begin[0] + (int)blockIdx.x];
    const int4 rd = a.reps[r];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    const int n3 = 6 * half;  // elements of one replica
    const int nor = a.nor_s ? a.nor_s[rd.x] : n_or;
    T* g = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[r] * (long long)n3;
    // couplings after the spins (6 half floats; n3 * sizeof(T) is a multiple of 16 B)
    float* sJ = reinterpret_cast<float*>(sm + n3);
    const float* gJ = a.J + sd.J_off;
    // The replica and its sample's couplings arrive by two bulk copies (one
    // thread issues them; io_bar counts their bytes).  A block that starts
    // with a heat-bath half sweep (colour 0) does not read colour 0's spins:
    // that half sweep draws every one of them afresh.
    const int skip = n_hb > 0 ? 3 * half : 0;
    if (threadIdx.x == 0) {
        mbar_init(&io_bar, 1);
        fence_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned sbytes = (unsigned)((n3 - skip) * (int)sizeof(T)), jbytes = (unsigned)n3 * 4u;
        mbar_expect_tx(&io_bar, sbytes + jbytes);
        // failure-path test hook: CTA 0 leaves its copies un-issued, so its wait runs out
        if (!(a.wait_fault && blockIdx.x == 0)) {
            bulk_g2s(sm + skip, g + skip, sbytes, &io_bar);
            bulk_g2s(sJ, gJ, jbytes, &io_bar);
        }
    }
    // a wait that gave up leaves the replica in global memory as it was
    if (__syncthreads_or(!mbar_wait_io(&io_bar, 0u, a, !(a.wait_fault && blockIdx.x == 0)))) return;
    T e[1];
    if (sizeof(T) == 4 && sd.vec == 4) e[0] = res_block<T, (sizeof(T) == 4 ? 4 : 2)>(sm, sJ, a, sd, rd, n_hb, nor);
    else e[0] = res_block<T, 2>(sm, sJ, a, sd, rd, n_hb, nor);
    // the final replica leaves by one bulk copy, after every thread's writes
    // are made visible to the copy engine (res_block ends with a CTA barrier,
    // the fence and the barrier below order the last half sweep's stores)
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_s2g(g, sm, (unsigned)(n3 * (int)sizeof(T)));
        bulk_commit();
    }
    double H[1];
    block_sum_exact<T, 1>(e, H, red);
    if (threadIdx.x == 0) {
        a.H[r] = H[0];
        bulk_wait_read();  // the shared memory stays until the copy has read it
    }
}

// ---------------------------------------------------------------------------
// Cluster-resident block: a replica too large for one SM (L = 24, 32 in
// float) is split over a cluster of CS CTAs, CTA `rank` holding the z planes
// [rank Lz, (rank + 1) Lz), Lz = L / CS, of both colours and their
// couplings in shared memory ([colour][component][hl], hl = half / CS, the
// same layout as the global colour-split arrays restricted to the slab).
// Neighbours in the planes just outside the slab are read from the adjacent
// CTAs' shared memory (distributed shared memory); a cluster barrier
// separates the half sweeps.  Every CTA executes the same sequence of
// barriers, so no CTA waits on a condition only another one can change.
// ---------------------------------------------------------------------------
constexpr int CL_THREADS = 1024;      // wide clusters: one CTA per SM
constexpr int CL_THREADS_NARROW = 512; // narrow clusters: two CTAs per SM (slab <= 110 KB)

// Neighbour field of V sites of a slab row; the z+ row may live in the next
// CTA (othP) and the z- row with its couplings in the previous one (othM,
// JothM); all pointers address [component][hl] arrays of the other colour.
template <typename T, int V, bool XSHFL = false>
__device__ __forceinline__ void nbr_field_cl(const T* oth, const float* Jown, const float* Joth, int hl, int h0,
                                             int xs, int hyp, int hym, const T* othP, int hzp, const T* othM,
                                             const float* JothM, int hzm, int p, T (&S)[3][V]) {
    {   // +-x: the same row of the other colour, shifted by one (plus xs: an index, or with XSHFL a lane)
        float jp[V], jm[V];
        ldv<float, V>(Jown + h0, jp);
        {
            float jx[V];
            ldv<float, V>(Joth + h0, jx);
            const float jxs = XSHFL ? __shfl_sync(0xFFFFFFFFu, jx[V - 1], xs) : Joth[xs];
#pragma unroll
            for (int v = 0; v < V; ++v) jm[v] = p ? jx[v] : (v == 0 ? jxs : jx[v - 1]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T* o = oth + c * hl;
            T O[V];
            ldv<T, V>(o + h0, O);
            const T os = XSHFL ? __shfl_sync(0xFFFFFFFFu, p ? O[0] : O[V - 1], xs) : o[xs];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T xp = p ? (v == V - 1 ? os : O[v + 1]) : O[v];
                const T xm = p ? O[v] : (v == 0 ? os : O[v - 1]);
                S[c][v] = (T)jp[v] * xp + (T)jm[v] * xm;
            }
        }
    }
    const float* jsrc[4] = {Jown + hl + h0, Joth + hl + hym, Jown + 2 * hl + h0, JothM + 2 * hl + hzm};
    const T* nsrc[4] = {oth + hyp, oth + hym, othP + hzp, othM + hzm};
#pragma unroll
    for (int dir = 0; dir < 4; ++dir) {
        float jd[V];
        ldv<float, V>(jsrc[dir], jd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T n[V];
            ldv<T, V>(nsrc[dir] + c * hl, n);
#pragma unroll
            for (int v = 0; v < V; ++v) S[c][v] += (T)jd[v] * n[v];
        }
    }
}

struct Slab {
    int hl, Lz, k0, rank, cs;  // sites per colour, planes, first plane, CTA rank, cluster size
};

template <typename T, int NTH, int V, int KIND, bool ENERGY>
__device__ __forceinline__ T cl_halfsweep(cg::cluster_group& cl, T* __restrict__ sm, const float* __restrict__ J,
                                          const SampleDesc& sd, const Slab& sb, int color, T beta,
                                          unsigned long long seed, uint32_t sample, uint32_t rep_id,
                                          unsigned long long step) {
    const int hl = sb.hl, hL = sd.hL, L = sd.L;
    T* own = sm + color * 3 * hl;
    const T* oth = sm + (1 - color) * 3 * hl;
    const float* Jown = J + color * 3 * hl;
    const float* Joth = J + (1 - color) * 3 * hl;
    T e = (T)0;
    for (int h0 = (int)threadIdx.x * V; h0 < hl; h0 += NTH * V) {
        const int row = (int)fdiv((uint32_t)h0, sd.div_hL);  // slab row j + L kl
        const int ih0 = h0 - row * hL;
        const int kl = (int)fdiv((uint32_t)row, sd.div_L);
        const int j = row - kl * L;
        const int p = (j + sb.k0 + kl + color) & 1;
        const int rb = row * hL;
        const int xs = p ? rb + ((ih0 + V == hL) ? 0 : ih0 + V) : rb + ((ih0 == 0) ? hL - 1 : ih0 - 1);
        const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
        const int hyp = ih0 + hL * (jp + L * kl), hym = ih0 + hL * (jm + L * kl);
        const bool topz = kl + 1 == sb.Lz, botz = kl == 0;  // uniform over a warp (one plane)
        const T* othP = oth;
        if (topz) othP = cl.map_shared_rank(const_cast<T*>(oth), sb.rank + 1 == sb.cs ? 0 : sb.rank + 1);
        const int hzp = ih0 + hL * (j + L * (topz ? 0 : kl + 1));
        const T* othM = oth;
        const float* JothM = Joth;
        if (botz) {
            const int rm = sb.rank == 0 ? sb.cs - 1 : sb.rank - 1;
            othM = cl.map_shared_rank(const_cast<T*>(oth), rm);
            JothM = cl.map_shared_rank(const_cast<float*>(Joth), rm);
        }
        const int hzm = ih0 + hL * (j + L * (botz ? sb.Lz - 1 : kl - 1));

        T S[3][V];
        nbr_field_cl<T, V>(oth, Jown, Joth, hl, h0, xs, hyp, hym, othP, hzp, othM, JothM, hzm, p, S);
        T s[3][V];
        if (KIND == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ldv<T, V>(own + c * hl + h0, s[c]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv;
            if (KIND == 1) {
                const int x = 2 * (ih0 + v) + p + L * (row + L * sb.k0);
                const uint4 w = rng_words(seed, sample, (uint32_t)x, rep_id, step, 0u);
                sv = hb_site<T>(beta, Sv, w.x, w.y);
            } else {
                sv = {s[0][v], s[1][v], s[2][v]};
                or_site(Sv, sv);
            }
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
            if (ENERGY) e -= dot(sv, Sv);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<T, V>(own + c * hl + h0, s[c]);
    }
    return e;
}

// Indices of a thread's slab vector, computed once per launch when every
// thread owns at most one vector of a colour (hl <= threads * V).
struct VecIdxCl {
    int h0, xs0, xs1, hyp, hym, hzp, hzm, pz;  // pz: bit 0 p of colour 0, bit 1 z+ remote, bit 2 z- remote
};

template <int V>
__device__ __forceinline__ VecIdxCl vec_idx_cl(const SampleDesc& sd, const Slab& sb, int h0, bool xshfl) {
    const int hL = sd.hL, L = sd.L;
    VecIdxCl q;
    q.h0 = h0;
    const int row = (int)fdiv((uint32_t)h0, sd.div_hL);
    const int ih0 = h0 - row * hL;
    const int kl = (int)fdiv((uint32_t)row, sd.div_L);
    const int j = row - kl * L;
    const int p0 = (j + sb.k0 + kl) & 1;
    const int rb = row * hL;
    int left = rb + ((ih0 == 0) ? hL - 1 : ih0 - 1), right = rb + ((ih0 + V == hL) ? 0 : ih0 + V);
    if (xshfl) xs_lanes<V>(hL, ih0, right, left);  // lanes instead of indices
    q.xs0 = p0 ? right : left;
    q.xs1 = p0 ? left : right;
    const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
    q.hyp = ih0 + hL * (jp + L * kl);
    q.hym = ih0 + hL * (jm + L * kl);
    const bool topz = kl + 1 == sb.Lz, botz = kl == 0;
    q.hzp = ih0 + hL * (j + L * (topz ? 0 : kl + 1));
    q.hzm = ih0 + hL * (j + L * (botz ? sb.Lz - 1 : kl - 1));
    q.pz = p0 | (topz ? 2 : 0) | (botz ? 4 : 0);
    return q;
}

// Overrelaxation half sweep of the slab with precomputed indices; the
// neighbour CTAs' arrays are mapped only by the warps of the boundary planes
// (a warp's vectors lie in one plane, so the branch is uniform).
template <typename T, int V, bool ENERGY, bool XSHFL>
__device__ __forceinline__ T cl_or_one(cg::cluster_group& cl, T* __restrict__ sm, const float* __restrict__ J,
                                       int hl, int rank, int cs, int color, const VecIdxCl& q) {
    T e = (T)0;
    if (q.h0 < hl) {
        T* own = sm + color * 3 * hl;
        const T* oth = sm + (1 - color) * 3 * hl;
        const float* Jown = J + color * 3 * hl;
        const float* Joth = J + (1 - color) * 3 * hl;
        const int p = (q.pz & 1) ^ color;
        const int xs = color ? q.xs1 : q.xs0;
        const T* othP = oth;
        if (q.pz & 2) othP = cl.map_shared_rank(const_cast<T*>(oth), rank + 1 == cs ? 0 : rank + 1);
        const T* othM = oth;
        const float* JothM = Joth;
        if (q.pz & 4) {
            const int rm = rank == 0 ? cs - 1 : rank - 1;
            othM = cl.map_shared_rank(const_cast<T*>(oth), rm);
            JothM = cl.map_shared_rank(const_cast<float*>(Joth), rm);
        }
        T S[3][V];
        nbr_field_cl<T, V, XSHFL>(oth, Jown, Joth, hl, q.h0, xs, q.hyp, q.hym, othP, q.hzp, othM, JothM, q.hzm, p,
                                  S);
        T s[3][V];
#pragma unroll
        for (int c = 0; c < 3; ++c) ldv<T, V>(own + c * hl + q.h0, s[c]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv = {s[0][v], s[1][v], s[2][v]};
            or_site(Sv, sv);
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
            if (ENERGY) e -= dot(sv, Sv);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<T, V>(own + c * hl + q.h0, s[c]);
    }
    return e;
}

// The heat-bath half sweeps of the cluster block run one site per thread: on
// the overrelaxation path's vectors they are cheaper themselves but raise the
// kernel's register demand, and the overrelaxation sweeps then spill.
template <typename T, int NTH, int V>
__device__ __forceinline__ T cl_block(cg::cluster_group& cl, T* sm, const float* J, const DevBatch& a,
                                      const SampleDesc& sd, const Slab& sb, const int4& rd, int n_hb, int n_or) {
    const T beta = (T)a.betas[sd.beta_off + rd.z];
    const unsigned long long step0 = *a.d_step;
    const int total = 2 * (n_hb + n_or);
    T e = (T)0;
    int kstep = 0;
    for (int hb = 0; hb < n_hb; ++hb)
        for (int c = 0; c < 2; ++c, ++kstep) {
            const unsigned long long st = step0 + (unsigned long long)kstep;
            if (kstep == total - 1)
                e = cl_halfsweep<T, NTH, 1, 1, true>(cl, sm, J, sd, sb, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w,
                                                st);
            else
                cl_halfsweep<T, NTH, 1, 1, false>(cl, sm, J, sd, sb, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w,
                                             st);
            cl.sync();
        }
    if (sb.hl <= NTH * V) {
        const bool xsh = (32 % (sd.hL / V) == 0) && ((sb.hl / V) % 32 == 0);
        const VecIdxCl q = vec_idx_cl<V>(sd, sb, (int)threadIdx.x * V, xsh);
        for (int o = 0; o < n_or; ++o)
            for (int c = 0; c < 2; ++c, ++kstep) {
                if (xsh) {
                    if (kstep == total - 1) e = cl_or_one<T, V, true, true>(cl, sm, J, sb.hl, sb.rank, sb.cs, c, q);
                    else cl_or_one<T, V, false, true>(cl, sm, J, sb.hl, sb.rank, sb.cs, c, q);
                } else {
                    if (kstep == total - 1) e = cl_or_one<T, V, true, false>(cl, sm, J, sb.hl, sb.rank, sb.cs, c, q);
                    else cl_or_one<T, V, false, false>(cl, sm, J, sb.hl, sb.rank, sb.cs, c, q);
                }
                cl.sync();
            }
        return e;
    }
    for (int o = 0; o < n_or; ++o)
        for (int c = 0; c < 2; ++c, ++kstep) {
            if (kstep == total - 1)
                e = cl_halfsweep<T, NTH, V, 0, true>(cl, sm, J, sd, sb, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w,
                                                0ull);
            else
                cl_halfsweep<T, NTH, V, 0, false>(cl, sm, J, sd, sb, c, beta, a.seed, (uint32_t)rd.x, (uint32_t)rd.w,
                                             0ull);
            cl.sync();
        }
    return e;
}

// One cluster per replica of the group that starts at res_reps[begin]; NTH
// threads per CTA (1024: one CTA per SM; 512: two CTAs of different
// clusters share an SM, so one's barrier waits overlap the other's work).
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH, 1024 / NTH) k_resident_cl(DevBatch a, int n_hb, int n_or, int begin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ double cta_total;
    __shared__ int cta_failed;
    __shared__ __align__(8) unsigned long long io_bar;
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int r = a.res_reps[begin + (int)blockIdx.x / cs];
    const int4 rd = a.reps[r];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    Slab sb;
    sb.hl = half / cs;
    sb.Lz = sd.L / cs;
    sb.k0 = rank * sb.Lz;
    sb.rank = rank;
    sb.cs = cs;
    const int hl = sb.hl, n3 = 6 * hl;
    T* sm = reinterpret_cast<T*>(smem_raw);
    float* sJ = reinterpret_cast<float*>(sm + n3);  // n3 * sizeof(T) is a multiple of 16 B
    const int nor = a.nor_s ? a.nor_s[rd.x] : n_or;
    // this CTA's slab: 6 contiguous runs of hl elements (colour, component)
    // of the replica and of the couplings, fetched by bulk copies issued by
    // one thread (io_bar counts their bytes); colour 0's spin runs are not
    // read when the block starts with a heat-bath half sweep, which draws
    // them afresh
    T* g = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[r] * (6LL * half);
    const float* gJ = a.J + sd.J_off;
    if (threadIdx.x == 0) {
        mbar_init(&io_bar, 1);
        fence_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int run0 = n_hb > 0 ? 3 : 0;
        const unsigned sb = (unsigned)(hl * (int)sizeof(T)), jb = (unsigned)hl * 4u;
        mbar_expect_tx(&io_bar, (unsigned)(6 - run0) * sb + 6u * jb);
        // failure-path test hook: the first CTA of the launch leaves its copies
        // un-issued, so its wait runs out
        if (!(a.wait_fault && blockIdx.x == 0)) {
            for (int run = run0; run < 6; ++run)
                bulk_g2s(sm + run * hl, g + (long long)run * half + rank * hl, sb, &io_bar);
            for (int run = 0; run < 6; ++run)
                bulk_g2s(sJ + run * hl, gJ + (long long)run * half + rank * hl, jb, &io_bar);
        }
    }
    const int failed = __syncthreads_or(!mbar_wait_io(&io_bar, 0u, a, !(a.wait_fault && blockIdx.x == 0)));
    if (threadIdx.x == 0) cta_failed = failed;
    cl.sync();  // every slab loaded (or given up) before any neighbour reads it
    // a wait that gave up anywhere in the cluster: every CTA of it sees the
    // same flags and skips the block, leaving the replica in global memory as
    // it was (one more barrier: no CTA leaves while another reads its flag)
    int any_failed = 0;
    for (int q = 0; q < cs; ++q) any_failed |= *cl.map_shared_rank(&cta_failed, q);
    if (any_failed) {
        cl.sync();
        return;
    }
    T e[1];
    if (sizeof(T) == 4 && sd.vec == 4)
        e[0] = cl_block<T, NTH, (sizeof(T) == 4 ? 4 : 2)>(cl, sm, sJ, a, sd, sb, rd, n_hb, nor);
    else e[0] = cl_block<T, NTH, 2>(cl, sm, sJ, a, sd, sb, rd, n_hb, nor);
    // the last barrier of the block has passed: the slab is final; it leaves
    // by bulk copies after the fence makes every thread's writes visible to
    // the copy engine
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int run = 0; run < 6; ++run)
            bulk_s2g(g + (long long)run * half + rank * hl, sm + run * hl, (unsigned)(hl * (int)sizeof(T)));
        bulk_commit();
    }
    double tot[1];
    block_sum_exact<T, 1>(e, tot, red);
    if (threadIdx.x == 0) cta_total = tot[0];
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double H = 0.0;
        for (int q = 0; q < cs; ++q) H += *cl.map_shared_rank(&cta_total, q);
        a.H[r] = H;
    }
    if (threadIdx.x == 0) bulk_wait_read();  // the slab stays until its copies have read it
    cl.sync();  // no CTA leaves while rank 0 reads its total
}

// One replica (6 half elements of T) and its sample's couplings (6 half floats).
size_t resident_smem_bytes(int half, bool fp64) { return (size_t)6 * half * ((fp64 ? 8 : 4) + 4); }

bool resident_supported(const SampleDesc& sd, bool fp64, int vec) {
    // 16- or 8-byte rows (vec 4 or 2; double only 2), 16-byte aligned
    // coupling blocks (6 half a multiple of 4), and at most 200 KB per CTA
    // (two CTAs per SM up to 112 KB, e.g. L = 16 in float; one above, e.g.
    // L = 16 in double, where the autotuner weighs it against streaming)
    if (vec != 4 && vec != 2) return false;
    if (fp64 && vec != 2) return false;
    if ((6 * sd.half) % 4 != 0) return false;
    return sd.hL % vec == 0 && resident_smem_bytes(sd.half, fp64) <= 200 * 1024;
}

int resident_cluster(const SampleDesc& sd, bool fp64, int vec) {
    if (resident_supported(sd, fp64, vec)) return 1;
    if (vec != 4 && vec != 2) return 0;
    if (fp64 && vec != 2) return 0;
    if (sd.hL % vec) return 0;
    for (int cs : {2, 4, 8}) {
        if (sd.L % cs) continue;
        const int hl = sd.half / cs;  // hL L (L / cs) sites: a multiple of vec
        if (hl % 4 != 0) continue;    // 16-byte aligned runs for the slab copies
        if (resident_smem_bytes(hl, fp64) <= 200 * 1024) return cs;
    }
    return 0;
}

int resident_cluster_narrow(const SampleDesc& sd, bool fp64, int vec) {
    if (resident_supported(sd, fp64, vec)) return 0;  // one CTA per replica already fits
    if (vec != 4 && vec != 2) return 0;
    if (fp64 && vec != 2) return 0;
    if (sd.hL % vec) return 0;
    for (int cs : {2, 4, 8}) {
        if (sd.L % cs) continue;
        const int hl = sd.half / cs;
        if (hl % 4 != 0) continue;
        if (resident_smem_bytes(hl, fp64) <= 110 * 1024) return cs;  // two CTAs per SM
    }
    return 0;
}

int resident_group(int cs, bool narrow) {
    const int lg = cs == 1 ? 0 : cs == 2 ? 1 : cs == 4 ? 2 : 3;
    return lg == 0 ? 0 : lg + (narrow ? 3 : 0);
}

int resident_launch_count(const DevBatch& b) {
    int n = 0;
    for (int g = 0; g < RES_GROUPS; ++g) n += b.rcl_count[g] > 0;
    return n;
}

template <typename T, int NTH>
static cudaError_t launch_cl(const DevBatch& b, int g, int n_hb, int n_or, cudaStream_t st) {
    const int cs = 1 << ((g - 1) % 3 + 1);
    const size_t smem = resident_smem_bytes(b.rcl_half[g] / cs, sizeof(T) == 8);
    cudaError_t e = ensure_smem((const void*)k_resident_cl<T, NTH>, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(b.rcl_count[g] * cs), 1, 1);
    cfg.blockDim = dim3(NTH, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_resident_cl<T, NTH>, b, n_hb, n_or, b.rcl_begin[g]);
}

cudaError_t launch_resident(const DevBatch& b, bool fp64, int n_hb, int n_or, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (b.rcl_count[0] > 0) {
        const size_t smem = resident_smem_bytes(b.rcl_half[0], fp64);
        if (fp64) {
            e = ensure_smem((const void*)k_resident<double>, smem);
            if (e != cudaSuccess) return e;
            k_resident<double><<<b.rcl_count[0], RES_THREADS, smem, st>>>(b, n_hb, n_or);
        } else {
            e = ensure_smem((const void*)k_resident<float>, smem);
            if (e != cudaSuccess) return e;
            k_resident<float><<<b.rcl_count[0], RES_THREADS, smem, st>>>(b, n_hb, n_or);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int g = 1; g < RES_GROUPS; ++g) {
        if (b.rcl_count[g] == 0) continue;
        if (g <= 3)
            e = fp64 ? launch_cl<double, CL_THREADS>(b, g, n_hb, n_or, st)
                     : launch_cl<float, CL_THREADS>(b, g, n_hb, n_or, st);
        else
            e = fp64 ? launch_cl<double, CL_THREADS_NARROW>(b, g, n_hb, n_or, st)
                     : launch_cl<float, CL_THREADS_NARROW>(b, g, n_hb, n_or, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ptk
