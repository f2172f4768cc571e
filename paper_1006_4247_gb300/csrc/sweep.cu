// sweep.cu -- checkerboard half sweeps (heat bath and overrelaxation,
// section III.C of Hasenbusch & Schaefer), the energy reduction, initial
// spins and the overlap reduction (section II).
//
// Half sweep: one thread updates V consecutive sites (ih0 .. ih0+V-1) of one
// row (j, k) of one colour of one replica; a block is a tile of 256 V
// consecutive sites (h) of one replica.  Along a row the checkerboard offset
// p = (j + k + colour) & 1 is fixed, so the +-x neighbours of the V sites are
// the aligned vector of the other colour at the same h shifted by one place,
// plus one element that wraps around the row; the +-y and +-z neighbours and
// all couplings are aligned vectors.  Per update that is about 7 memory
// instructions instead of 27, all of them unit-stride across the warp.
// Heat bath reads only the neighbours (24 B per update in float), the
// overrelaxation also the old spin (36 B).
#include "kernels.h"
#include "pt_device.cuh"

namespace ptk {

// KIND 0: overrelaxation, 1: heat bath, 2: energy only (colour 0, no store).
// Tiles: tile_begin + blockIdx.x indexes `tidx` (the streaming subset) when
// it is given, else vtiles directly.
template <typename T, int V, int KIND, bool ENERGY>
__global__ void __launch_bounds__(TILE, KIND == 1 ? 5 : 6) k_sweep(DevBatch a, const int* __restrict__ tidx, int tile_begin,
                                                int color, int step_k, int or_index) {
    __shared__ double sh[32];
    const int t = tidx ? tidx[tile_begin + (int)blockIdx.x] : tile_begin + (int)blockIdx.x;
    const int2 tl = a.vtiles[t];
    const int4 rd = a.reps[tl.x];
    if (or_index >= 0 && a.nor_s && or_index >= a.nor_s[rd.x]) return;  // uniform per block
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half, hL = sd.hL, L = sd.L;
    const int h0 = tl.y + (int)threadIdx.x * V;
    T e[1] = {(T)0};  // this thread's V sites of H (energy launches)
    if (h0 < half) {
        T* base = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[tl.x] * (6LL * half);
        T* own = base + color * 3 * half;
        const T* oth = base + (1 - color) * 3 * half;
        const float* Jown = a.J + sd.J_off + color * 3 * half;
        const float* Joth = a.J + sd.J_off + (1 - color) * 3 * half;
        const int row = (int)fdiv((uint32_t)h0, sd.div_hL);
        const int ih0 = h0 - row * hL;
        const int k = (int)fdiv((uint32_t)row, sd.div_L);
        const int j = row - k * L;
        const int p = (j + k + color) & 1;
        const int rb = row * hL;
        // index of the wrapped x neighbour: p = 0 -> left of ih0, p = 1 -> right of ih0+V-1
        const int xs = p ? rb + ((ih0 + V == hL) ? 0 : ih0 + V) : rb + ((ih0 == 0) ? hL - 1 : ih0 - 1);
        const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
        const int kp = (k + 1 == L) ? 0 : k + 1, km = (k == 0) ? L - 1 : k - 1;
        const int hyp = ih0 + hL * (jp + L * k), hym = ih0 + hL * (jm + L * k);
        const int hzp = ih0 + hL * (j + L * kp), hzm = ih0 + hL * (j + L * km);

        T S[3][V];
        nbr_field<T, V>(oth, Jown, Joth, half, h0, xs, hyp, hym, hzp, hzm, p, S);

        T s[3][V];
        if (KIND != 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ldv<T, V>(own + c * half + h0, s[c]);
        }
        const T beta = (KIND == 1) ? (T)a.betas[sd.beta_off + rd.z] : (T)0;
        const unsigned long long step = (KIND == 1) ? *a.d_step + (unsigned long long)step_k : 0ull;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const V3<T> Sv = {S[0][v], S[1][v], S[2][v]};
            V3<T> sv;
            if (KIND == 1) {
                const int x = 2 * (ih0 + v) + p + L * row;
                const uint4 w = rng_words(a.seed, (uint32_t)rd.x, (uint32_t)x, (uint32_t)rd.w, step, 0u);
                sv = hb_site<T>(beta, Sv, w.x, w.y);
            } else {
                sv = {s[0][v], s[1][v], s[2][v]};
                if (KIND == 0) or_site(Sv, sv);
            }
            s[0][v] = sv.x; s[1][v] = sv.y; s[2][v] = sv.z;
            if (ENERGY || KIND == 2) e[0] -= dot(sv, Sv);
        }
        if (KIND != 2) {
#pragma unroll
            for (int c = 0; c < 3; ++c) stv<T, V>(own + c * half + h0, s[c]);
        }
    }
    if (ENERGY || KIND == 2) {
        double tot[1];
        block_sum_exact<T, 1>(e, tot, sh);
        if (threadIdx.x == 0) a.part[t] = tot[0];
    }
}

// H[r] = sum of the tile partials of replica r, in tile order (replicas of
// resident samples are skipped unless `all`).
__global__ void k_energy_finalize(DevBatch a, int all) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_reps) return;
    const int4 rd = a.reps[r];
    const SampleDesc& sd = a.samples[rd.x];
    if (!all && sd.resident) return;
    const int t0 = sd.tile0 + (r - sd.r0) * sd.tiles_per_rep;
    double H = 0.0;
    for (int k = 0; k < sd.tiles_per_rep; ++k) H += a.part[t0 + k];
    a.H[r] = H;
}

// Initial spins: uniform on the sphere from Philox purpose 4
// (z = (w0 >> 8) 2^-23 - 1, phi = 2 pi (w1 >> 8) 2^-24), or all (1, 0, 0).
// Grid: (replica, colour); threads stride over the sites of the colour.
template <typename T>
__global__ void __launch_bounds__(TILE) k_init_spins(DevBatch a, int ordered) {
    const int r = blockIdx.x, color = blockIdx.y;
    const int4 rd = a.reps[r];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    T* own = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[r] * (6LL * half) + color * 3 * half;
    for (int h = threadIdx.x; h < half; h += blockDim.x) {
        V3<T> s;
        if (ordered) {
            s.x = (T)1; s.y = (T)0; s.z = (T)0;
        } else {
            const Site st = site_of(sd, color, h);
            const uint4 w = rng_words(a.seed, (uint32_t)rd.x, (uint32_t)st.x, (uint32_t)rd.w, 0ull, 4u);
            const T z = (T)(w.x >> 8) * (T)0x1p-23 - (T)1;
            const T phi = (T)2 * M<T>::pi * ((T)(w.y >> 8) * (T)0x1p-24);
            const T rho = M<T>::sqrt_((T)1 - z * z);
            T sp, cp;
            M<T>::sincos_(phi, &sp, &cp);
            s.x = rho * cp; s.y = rho * sp; s.z = z;
        }
        st3(own, half, h, s);
    }
}

__global__ void k_advance_step(unsigned long long* d_step, int by) { *d_step += (unsigned long long)by; }

// Overlap Q_ab = sum_x s0_a,x s1_b,x between copy 0 and copy 1 at the same
// beta index (Eq. over) and chi = (1/N) sum_ab Q_ab^2.  One block per
// (sample, beta index); each thread reads 16-byte vectors of consecutive sites
// (a vector never straddles the two colours: half is a multiple of 4) and
// accumulates them in T in chunks of at most 32 sites; the chunk sums are
// added in T with compensation (Knuth's two-sum), which keeps the thread's
// total as accurate as a double sum rounded to T without work on GB300's slow
// FP64 pipe; warp shuffles and one shared-memory pass finish the nine sums
// in a fixed order.
template <typename T>
__global__ void __launch_bounds__(TILE) k_overlap(DevBatch a) {
    __shared__ double sh[9 * 32];
    const int q = blockIdx.x;  // beta_off(s) + b over all samples
    const int s = a.q_sample[q];
    const SampleDesc& sd = a.samples[s];
    const int b = q - sd.beta_off;
    const int half = sd.half;
    const int r0 = sd.r0 + b, r1 = sd.r0 + sd.NT + b;
    const T* b0 = (const T*)a.spins + a.chain_off[sd.chain0] + (long long)a.bufmap[r0] * (6LL * half);
    const T* b1 = (const T*)a.spins + a.chain_off[sd.chain0 + 1] + (long long)a.bufmap[r1] * (6LL * half);
    T hi[9], lo[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) hi[n] = lo[n] = (T)0;
    constexpr int V = 16 / sizeof(T);
    constexpr int CH = 32 / V;  // vectors per chunk of 32 sites
    const int N = 2 * half, NV = N / V;
    for (int base = 0; base < NV; base += CH * TILE) {
        T part[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) part[n] = (T)0;
        const int end = min(NV, base + CH * TILE);
        // two vectors of each copy in flight per thread (12 16-byte loads);
        // the additions into part keep their order
#pragma unroll 2
        for (int xv = base + (int)threadIdx.x; xv < end; xv += TILE) {
            const int x = xv * V;
            const int c = x >= half ? 1 : 0;
            const int h = x - c * half;
            const T* p0 = b0 + c * 3 * half + h;
            const T* p1 = b1 + c * 3 * half + h;
            T u0[3][V], u1[3][V];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ldv_nc<T, V>(p0 + k * half, u0[k]);
                ldv_nc<T, V>(p1 + k * half, u1[k]);
            }
#pragma unroll
            for (int n = 0; n < 9; ++n)
#pragma unroll
                for (int v = 0; v < V; ++v) part[n] += u0[n / 3][v] * u1[n % 3][v];
        }
#pragma unroll
        for (int n = 0; n < 9; ++n) {
            const T sum = hi[n] + part[n];
            const T bb = sum - hi[n];
            lo[n] += (hi[n] - (sum - bb)) + (part[n] - bb);
            hi[n] = sum;
        }
    }
    // the thread totals enter the warp tree in T, the warp sums are added in
    // double (the precision policy of all reductions)
    T tp[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) tp[n] = hi[n] + lo[n];
    double tot[9];
    block_sum_multi<T, 9>(tp, tot, sh);
    if (threadIdx.x == 0) {
        double chi = 0.0;
#pragma unroll
        for (int n = 0; n < 9; ++n) {
            a.Q[(long long)q * 9 + n] = tot[n];
            chi += tot[n] * tot[n];
        }
        a.chi[q] = chi / (double)N;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int V>
static void sweep_tv(const DevBatch& b, const int* tidx, int kind, bool energy, int color, int step_k,
                     int or_index, int begin, int count, cudaStream_t st) {
    if (count == 0) return;
    dim3 grid(count), block(TILE);
    if (kind == 1) {
        if (energy) k_sweep<T, V, 1, true><<<grid, block, 0, st>>>(b, tidx, begin, color, step_k, or_index);
        else k_sweep<T, V, 1, false><<<grid, block, 0, st>>>(b, tidx, begin, color, step_k, or_index);
    } else if (kind == 0) {
        if (energy) k_sweep<T, V, 0, true><<<grid, block, 0, st>>>(b, tidx, begin, color, step_k, or_index);
        else k_sweep<T, V, 0, false><<<grid, block, 0, st>>>(b, tidx, begin, color, step_k, or_index);
    } else {
        k_sweep<T, V, 2, false><<<grid, block, 0, st>>>(b, tidx, begin, 0, 0, -1);
    }
}

// One launch per vector-width class present in the tile set.
static cudaError_t sweep_all(const DevBatch& b, bool fp64, bool streaming_only, int kind, bool energy, int color,
                             int step_k, int or_index, cudaStream_t st) {
    for (int cls = 0; cls < 3; ++cls) {
        const int begin = streaming_only ? b.sclass_begin[cls] : b.vclass_begin[cls];
        const int count = streaming_only ? b.sclass_count[cls] : b.vclass_count[cls];
        if (count == 0) continue;
        const int* tidx = streaming_only ? b.stiles : nullptr;  // NULL stiles: subset == whole list
        const int V = b.vclass_width[cls];
        if (fp64) {
            if (V == 2) sweep_tv<double, 2>(b, tidx, kind, energy, color, step_k, or_index, begin, count, st);
            else sweep_tv<double, 1>(b, tidx, kind, energy, color, step_k, or_index, begin, count, st);
        } else {
            if (V == 4) sweep_tv<float, 4>(b, tidx, kind, energy, color, step_k, or_index, begin, count, st);
            else if (V == 2) sweep_tv<float, 2>(b, tidx, kind, energy, color, step_k, or_index, begin, count, st);
            else sweep_tv<float, 1>(b, tidx, kind, energy, color, step_k, or_index, begin, count, st);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int sweep_stream_launch_count(const DevBatch& b) {
    int n = 0;
    for (int cls = 0; cls < 3; ++cls) n += b.sclass_count[cls] > 0;
    return n;
}

int energy_launch_count(const DevBatch& b, bool all) {
    int n = 0;
    for (int cls = 0; cls < 3; ++cls) n += (all ? b.vclass_count[cls] : b.sclass_count[cls]) > 0;
    return n;
}

cudaError_t launch_halfsweep(const DevBatch& b, bool fp64, int kind, bool energy, int color, int step_k,
                             int or_index, cudaStream_t st) {
    return sweep_all(b, fp64, true, kind, energy, color, step_k, or_index, st);
}

cudaError_t launch_energy(const DevBatch& b, bool fp64, bool all, cudaStream_t st) {
    return sweep_all(b, fp64, !all, 2, false, 0, 0, -1, st);
}

cudaError_t launch_energy_finalize(const DevBatch& b, bool all, cudaStream_t st) {
    k_energy_finalize<<<(b.n_reps + 127) / 128, 128, 0, st>>>(b, all ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(const DevBatch& b, bool fp64, int ordered, cudaStream_t st) {
    dim3 grid(b.n_reps, 2);
    if (fp64) k_init_spins<double><<<grid, TILE, 0, st>>>(b, ordered);
    else k_init_spins<float><<<grid, TILE, 0, st>>>(b, ordered);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(const DevBatch& b, int by, cudaStream_t st) {
    k_advance_step<<<1, 1, 0, st>>>(b.d_step, by);
    return cudaGetLastError();
}

cudaError_t launch_overlap(const DevBatch& b, bool fp64, cudaStream_t st) {
    if (fp64) k_overlap<double><<<b.n_q, TILE, 0, st>>>(b);
    else k_overlap<float><<<b.n_q, TILE, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace ptk
