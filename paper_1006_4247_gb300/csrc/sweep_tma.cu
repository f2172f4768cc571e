// sweep_tma.cu -- streaming overrelaxation half sweep (section III.C of
// Hasenbusch & Schaefer) with the checkerboard slab and its halo staged in
// shared memory by the Tensor Memory Accelerator (cp.async.bulk).
//
// Work item = (sample, block of P consecutive z planes, group of replicas of
// that sample).  A persistent CTA takes items in turn:
//   * the item's couplings (own-colour forward couplings of the P planes and
//     the other colour's couplings needed as backward bonds, P + 1 planes for
//     z) are read once into shared memory and serve every replica of the
//     group (all replicas of a sample share J);
//   * for each replica, one thread issues bulk copies of the own-colour
//     planes k0 .. k0+P-1 and the other-colour planes k0-1 .. k0+P (the +-z
//     halo, split where it wraps around the periodic lattice) into one of
//     TMA_STAGES stages, completing on the stage's mbarrier; while the CTA
//     updates replica i, the copies of the next TMA_STAGES - 1 replicas are in
//     flight;
//   * the updated spins go straight from registers to global memory with
//     16-byte stores.
// Every mbarrier wait is bounded.  If a wait gives up, the kernel records the
// stage in the batch's error word, waits (bounded again) for its own copies
// and returns; the host reports PT_ERR_TIMEOUT.
#include "kernels.h"
#include "pt_device.cuh"
#include "tma.cuh"

namespace ptk {

constexpr int TMA_THREADS = 256;
constexpr int TMA_V = 4;
constexpr int TMA_STAGES = 4;  // replicas in flight per CTA (one CTA per SM)

// Issue the copies of replica r into a stage: own colour planes [k0, k0+P),
// other colour planes k0-1 .. k0+P in stage slots 0 .. P+1.
__device__ void tma_issue(const DevBatch& a, const SampleDesc& sd, int r, int color, int k0, int P, int plane,
                          float* st_own, float* st_oth, unsigned long long* bar) {
    const int half = sd.half, L = sd.L;
    const int4 rd = a.reps[r];
    const float* base = (const float*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[r] * (6LL * half);
    const float* own = base + color * 3 * half;
    const float* oth = base + (1 - color) * 3 * half;
    const unsigned pb = (unsigned)plane * 4u;
    const unsigned bytes = 3u * (unsigned)P * pb + 3u * (unsigned)(P + 2) * pb;
    mbar_expect_tx(bar, bytes);
    for (int c = 0; c < 3; ++c) {
        bulk_g2s(st_own + (size_t)c * P * plane, own + (size_t)c * half + (size_t)k0 * plane, (unsigned)P * pb, bar);
        float* d = st_oth + (size_t)c * (P + 2) * plane;
        const float* o = oth + (size_t)c * half;
        if (k0 >= 1 && k0 + P <= L - 1) {
            bulk_g2s(d, o + (size_t)(k0 - 1) * plane, (unsigned)(P + 2) * pb, bar);
        } else {
            const int lo = (k0 - 1 + L) % L, hi = (k0 + P) % L;
            bulk_g2s(d, o + (size_t)lo * plane, pb, bar);
            bulk_g2s(d + plane, o + (size_t)k0 * plane, (unsigned)P * pb, bar);
            bulk_g2s(d + (size_t)(P + 1) * plane, o + (size_t)hi * plane, pb, bar);
        }
    }
}

__global__ void __launch_bounds__(TMA_THREADS, 1) k_or_tma(DevBatch a, const int4* __restrict__ items, int n_items,
                                                           int color) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[TMA_STAGES];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        for (int q = 0; q < TMA_STAGES; ++q) mbar_init(&bar[q], 1);
        s_abort = 0;
        fence_async_smem();
    }
    __syncthreads();
    unsigned phase_bits = 0u;  // bit q: parity of the phase stage q waits for
    unsigned inflight = 0u;    // thread 0: bit q set while stage q has copies not yet waited for
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int4 it = items[item];  // (sample, k0, first replica, replica count)
        const SampleDesc& sd = a.samples[it.x];
        const int half = sd.half, hL = sd.hL, L = sd.L;
        const int plane = hL * L;
        const int P = sd.tma_planes;
        const int k0 = it.y;
        const int Pp = P * plane;
        float* Jsm = reinterpret_cast<float*>(smem_raw);                 // 6 P planes + 1
        float* stage0 = Jsm + (size_t)6 * Pp + plane;
        const int stage_elems = 3 * Pp + 3 * (P + 2) * plane;
        auto stage = [&](int q) { return stage0 + (size_t)q * stage_elems; };
        // couplings of the item: own forward (3 x P planes), other colour
        // x and y forward at the same planes, z forward at planes k0-1 .. k0+P-1
        {
            const float* Jown = a.J + sd.J_off + color * 3 * half;
            const float* Joth = a.J + sd.J_off + (1 - color) * 3 * half;
            for (int q = threadIdx.x * 4; q < Pp; q += TMA_THREADS * 4) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v[4];
                    ldv_nc<float, 4>(Jown + (size_t)c * half + (size_t)k0 * plane + q, v);
                    stv<float, 4>(Jsm + (size_t)c * Pp + q, v);
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float v[4];
                    ldv_nc<float, 4>(Joth + (size_t)c * half + (size_t)k0 * plane + q, v);
                    stv<float, 4>(Jsm + (size_t)(3 + c) * Pp + q, v);
                }
            }
            float* Jz = Jsm + (size_t)5 * Pp;
            for (int q = threadIdx.x * 4; q < Pp + plane; q += TMA_THREADS * 4) {
                const int slot = q / plane, w = q - slot * plane;
                const int kk = (k0 - 1 + slot + L) % L;
                float v[4];
                ldv_nc<float, 4>(Joth + (size_t)2 * half + (size_t)kk * plane + w, v);
                stv<float, 4>(Jz + q, v);
            }
        }
        // prologue: the first TMA_STAGES - 1 replicas (the issuing thread also
        // orders the CTA's earlier shared-memory reads before the copies)
        if (threadIdx.x == 0 && !s_abort) {
            fence_async_smem();
            for (int q = 0; q < TMA_STAGES - 1 && q < it.w; ++q) {
                // failure-path test hook: CTA 0 leaves its first stage
                // un-issued, so the wait for it runs out
                if (a.wait_fault && blockIdx.x == 0 && item == 0 && q == 0) continue;
                tma_issue(a, sd, it.z + q, color, k0, P, plane, stage(q), stage(q) + 3 * Pp, &bar[q]);
                inflight |= 1u << q;
            }
        }
        __syncthreads();
        for (int i = 0; i < it.w; ++i) {
            const int st = i % TMA_STAGES;
            const int ahead = i + TMA_STAGES - 1;  // its stage was read in iteration i - 1
            if (ahead < it.w && threadIdx.x == 0 && !s_abort) {
                const int sa = ahead % TMA_STAGES;
                fence_async_smem();
                tma_issue(a, sd, it.z + ahead, color, k0, P, plane, stage(sa), stage(sa) + 3 * Pp, &bar[sa]);
                inflight |= 1u << sa;
            }
            if (mbar_wait_bounded(&bar[st], (phase_bits >> st) & 1u, a.wait_limit)) {
                phase_bits ^= 1u << st;
                inflight &= ~(1u << st);
            } else {
                atomicOr(a.err, 1);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
            const int r = it.z + i;
            const int4 rd = a.reps[r];
            float* gown = (float*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[r] * (6LL * half) +
                          color * 3 * half;
            const float* sown = stage(st);
            const float* soth = stage(st) + 3 * Pp;
            const int ostr = (P + 2) * plane;
            for (int hl = threadIdx.x * TMA_V; hl < Pp; hl += TMA_THREADS * TMA_V) {
                const int h0 = k0 * plane + hl;
                const int row = (int)fdiv((uint32_t)h0, sd.div_hL);
                const int ih0 = h0 - row * hL;
                const int k = (int)fdiv((uint32_t)row, sd.div_L);
                const int j = row - k * L;
                const int q = k - k0;
                const int p = (j + k + color) & 1;
                const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
                const int oc = (q + 1) * plane + j * hL;  // row (j, k) of the other colour in the stage
                const int xs = p ? oc + ((ih0 + TMA_V == hL) ? 0 : ih0 + TMA_V) : oc + ((ih0 == 0) ? hL - 1 : ih0 - 1);
                const int o0 = oc + ih0;
                const int oyp = (q + 1) * plane + jp * hL + ih0, oym = (q + 1) * plane + jm * hL + ih0;
                const int ozp = (q + 2) * plane + j * hL + ih0, ozm = q * plane + j * hL + ih0;
                const int jl = q * plane + j * hL + ih0;            // own-plane index in J / own stage
                const int jxs = q * plane + j * hL + (xs - oc);     // wrapped x neighbour in J planes
                const int jym = q * plane + jm * hL + ih0;
                float S[3][TMA_V];
                {
                    float jp4[TMA_V], jm4[TMA_V], jx[TMA_V];
                    ldv<float, TMA_V>(Jsm + jl, jp4);
                    ldv<float, TMA_V>(Jsm + 3 * Pp + jl, jx);
                    const float jxsv = Jsm[3 * Pp + jxs];
#pragma unroll
                    for (int v = 0; v < TMA_V; ++v) jm4[v] = p ? jx[v] : (v == 0 ? jxsv : jx[v - 1]);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float* o = soth + c * ostr;
                        float O[TMA_V];
                        ldv<float, TMA_V>(o + o0, O);
                        const float os = o[xs];
#pragma unroll
                        for (int v = 0; v < TMA_V; ++v) {
                            const float xp = p ? (v == TMA_V - 1 ? os : O[v + 1]) : O[v];
                            const float xm = p ? O[v] : (v == 0 ? os : O[v - 1]);
                            S[c][v] = jp4[v] * xp + jm4[v] * xm;
                        }
                    }
                }
                const float* jsrc[4] = {Jsm + Pp + jl, Jsm + 4 * Pp + jym, Jsm + 2 * Pp + jl, Jsm + 5 * Pp + jl};
                const int nrow[4] = {oyp, oym, ozp, ozm};
#pragma unroll
                for (int dir = 0; dir < 4; ++dir) {
                    float jd[TMA_V];
                    ldv<float, TMA_V>(jsrc[dir], jd);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float n[TMA_V];
                        ldv<float, TMA_V>(soth + c * ostr + nrow[dir], n);
#pragma unroll
                        for (int v = 0; v < TMA_V; ++v) S[c][v] += jd[v] * n[v];
                    }
                }
                float s[3][TMA_V];
#pragma unroll
                for (int c = 0; c < 3; ++c) ldv<float, TMA_V>(sown + c * Pp + hl, s[c]);
#pragma unroll
                for (int v = 0; v < TMA_V; ++v) {
                    const V3<float> Sv = {S[0][v], S[1][v], S[2][v]};
                    V3<float> sv = {s[0][v], s[1][v], s[2][v]};
                    or_site(Sv, sv);
                    s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) stv<float, TMA_V>(gown + (size_t)c * half + h0, s[c]);
            }
            __syncthreads();  // stage st free for the copies issued in iteration i + 1
        }
        if (s_abort) break;
        __syncthreads();  // J region free for the next item
    }
    if (s_abort && threadIdx.x == 0) {
        // give the copies this CTA still has in flight a bounded chance to
        // land before its shared memory is released (at least the default
        // limit, however short the data waits were set)
        const unsigned long long drain = a.wait_limit > WAIT_LIMIT_DEFAULT ? a.wait_limit : WAIT_LIMIT_DEFAULT;
        for (int st = 0; st < TMA_STAGES; ++st)
            if ((inflight >> st) & 1u) mbar_wait_bounded(&bar[st], (phase_bits >> st) & 1u, drain);
    }
}

bool tma_supported(const SampleDesc& sd, bool fp64) { return !fp64 && sd.L % 8 == 0 && sd.tma_planes > 0; }

// Planes per item: the largest divisor P of L with P * plane <= 1024 sites.
int tma_planes_for(int L) {
    const int plane = (L / 2) * L;
    int best = 0;
    for (int P = 1; P <= L; ++P)
        if (L % P == 0 && P * plane <= 1024) best = P;
    return best;
}

size_t tma_smem_bytes(int P, int plane) {
    const size_t J = (size_t)6 * P * plane + plane;
    const size_t stage = (size_t)3 * P * plane + (size_t)3 * (P + 2) * plane;
    return (J + TMA_STAGES * stage) * sizeof(float);
}

cudaError_t launch_or_tma(const DevBatch& b, int color, cudaStream_t st) {
    if (b.n_tma_items == 0) return cudaSuccess;
    const size_t smem = b.tma_smem;
    cudaError_t e = ensure_smem((const void*)k_or_tma, smem);
    if (e != cudaSuccess) return e;
    const int grid = b.n_tma_items < b.n_sm ? b.n_tma_items : b.n_sm;
    k_or_tma<<<grid, TMA_THREADS, smem, st>>>(b, b.tma_items, b.n_tma_items, color);
    return cudaGetLastError();
}

}  // namespace ptk
