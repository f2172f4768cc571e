// sweep.cu -- checkerboard half sweeps (heat bath and overrelaxation,
// section III.C of Hasenbusch & Schaefer), the energy reduction, initial
// spins and the overlap reduction (section II).
//
// One thread updates one site of one colour of one replica; a block is a
// tile of 256 consecutive sites (h) of one replica, so all loads and stores of
// a warp are unit-stride in the colour-split layout.  The HB kernel reads only
// the neighbours and writes the site (24 B per update in float); OR also reads
// the old spin (36 B).
#include "kernels.h"
#include "pt_device.cuh"

namespace ptk {

template <typename T, int KIND, bool ENERGY>
__global__ void __launch_bounds__(TILE) k_halfsweep(DevBatch a, int color, int step_k) {
    __shared__ double sh[32];
    const int2 tl = a.tiles[blockIdx.x];
    const int4 rd = a.reps[tl.x];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    const int h = tl.y + (int)threadIdx.x;
    T* base = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[tl.x] * (6LL * half);
    T* own = base + color * 3 * half;
    const T* oth = base + (1 - color) * 3 * half;
    const float* Jown = a.J + sd.J_off + color * 3 * half;
    const float* Joth = a.J + sd.J_off + (1 - color) * 3 * half;
    double e = 0.0;
    if (h < half) {
        const Site st = site_of(sd, color, h);
        const V3<T> S = local_field<T>(st, half, oth, Jown, Joth);
        V3<T> s;
        if (KIND == 1) {
            const T beta = (T)a.betas[sd.beta_off + rd.z];
            const unsigned long long step = *a.d_step + (unsigned long long)step_k;
            const uint4 w = rng_words(a.seed, (uint32_t)rd.x, (uint32_t)st.x, (uint32_t)rd.w, step, 0u);
            s = hb_site<T>(beta, S, w.x, w.y);
        } else {
            s = ld3(own, half, h);
            or_site(S, s);
        }
        st3(own, half, h, s);
        if (ENERGY) e = -(double)dot(s, S);
    }
    if (ENERGY) {
        const double tot = block_sum(e, sh);
        if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
    }
}

// H = - sum over colour-0 sites of s_x . S_x (every bond has one colour-0 end).
template <typename T>
__global__ void __launch_bounds__(TILE) k_energy(DevBatch a) {
    __shared__ double sh[32];
    const int2 tl = a.tiles[blockIdx.x];
    const int4 rd = a.reps[tl.x];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    const int h = tl.y + (int)threadIdx.x;
    const T* base = (const T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[tl.x] * (6LL * half);
    double e = 0.0;
    if (h < half) {
        const Site st = site_of(sd, 0, h);
        const V3<T> S = local_field<T>(st, half, base + 3 * half, a.J + sd.J_off, a.J + sd.J_off + 3 * half);
        const V3<T> s = ld3(base, half, h);
        e = -(double)dot(s, S);
    }
    const double tot = block_sum(e, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

// H[r] = sum of the tile partials of replica r, in tile order.
__global__ void k_energy_finalize(DevBatch a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_reps) return;
    const int4 rd = a.reps[r];
    const SampleDesc& sd = a.samples[rd.x];
    const int t0 = sd.tile0 + (r - sd.r0) * sd.tiles_per_rep;
    double H = 0.0;
    for (int k = 0; k < sd.tiles_per_rep; ++k) H += a.part[t0 + k];
    a.H[r] = H;
}

// Initial spins: uniform on the sphere from Philox purpose 4
// (z = (w0 >> 8) 2^-23 - 1, phi = 2 pi (w1 >> 8) 2^-24), or all (1, 0, 0).
template <typename T>
__global__ void __launch_bounds__(TILE) k_init_spins(DevBatch a, int ordered) {
    const int color = blockIdx.y;
    const int2 tl = a.tiles[blockIdx.x];
    const int4 rd = a.reps[tl.x];
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    const int h = tl.y + (int)threadIdx.x;
    if (h >= half) return;
    T* base = (T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[tl.x] * (6LL * half);
    T* own = base + color * 3 * half;
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

__global__ void k_advance_step(unsigned long long* d_step, int by) { *d_step += (unsigned long long)by; }

// Overlap Q_ab = sum_x s0_a,x s1_b,x between copy 0 and copy 1 at the same
// beta index (Eq. over).  Grid: (tiles, colour); tiles of copy-1 replicas exit.
template <typename T>
__global__ void __launch_bounds__(TILE) k_overlap(DevBatch a) {
    __shared__ double sh[32];
    const int color = blockIdx.y;
    const int2 tl = a.tiles[blockIdx.x];
    const int4 rd = a.reps[tl.x];
    const ChainDesc cd = a.chains[rd.y];
    if (cd.copy != 0) return;
    const SampleDesc& sd = a.samples[rd.x];
    const int half = sd.half;
    const int r1 = tl.x + sd.NT;  // same beta index in copy 1
    const int h = tl.y + (int)threadIdx.x;
    const T* b0 = (const T*)a.spins + a.chain_off[rd.y] + (long long)a.bufmap[tl.x] * (6LL * half) + color * 3 * half;
    const T* b1 = (const T*)a.spins + a.chain_off[rd.y + 1] + (long long)a.bufmap[r1] * (6LL * half) + color * 3 * half;
    V3<T> s0 = {(T)0, (T)0, (T)0}, s1 = {(T)0, (T)0, (T)0};
    if (h < half) {
        s0 = ld3(b0, half, h);
        s1 = ld3(b1, half, h);
    }
    const T u0[3] = {s0.x, s0.y, s0.z};
    const T u1[3] = {s1.x, s1.y, s1.z};
    double* out = a.part9 + ((long long)blockIdx.x * 2 + color) * 9;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
        const double v = block_sum((double)(u0[n / 3] * u1[n % 3]), sh);
        if (threadIdx.x == 0) out[n] = v;
    }
}

// Q[beta_off + b][9] and chi = (1/N) sum Q^2 from the tile partials.
__global__ void k_overlap_finalize(DevBatch a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_reps) return;
    const int4 rd = a.reps[r];
    const ChainDesc cd = a.chains[rd.y];
    if (cd.copy != 0) return;
    const SampleDesc& sd = a.samples[rd.x];
    const int t0 = sd.tile0 + (r - sd.r0) * sd.tiles_per_rep;
    const int q = sd.beta_off + rd.z;
    double chi = 0.0;
    for (int n = 0; n < 9; ++n) {
        double v = 0.0;
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < sd.tiles_per_rep; ++k) v += a.part9[((long long)(t0 + k) * 2 + c) * 9 + n];
        a.Q[(long long)q * 9 + n] = v;
        chi += v * v;
    }
    a.chi[q] = chi / (2.0 * (double)sd.half);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t halfsweep_t(const DevBatch& b, int kind, bool energy, int color, int step_k,
                               cudaStream_t st) {
    dim3 grid(b.n_tiles), block(TILE);
    if (kind == 1) {
        if (energy) k_halfsweep<T, 1, true><<<grid, block, 0, st>>>(b, color, step_k);
        else k_halfsweep<T, 1, false><<<grid, block, 0, st>>>(b, color, step_k);
    } else {
        if (energy) k_halfsweep<T, 0, true><<<grid, block, 0, st>>>(b, color, step_k);
        else k_halfsweep<T, 0, false><<<grid, block, 0, st>>>(b, color, step_k);
    }
    return cudaGetLastError();
}

cudaError_t launch_halfsweep(const DevBatch& b, bool fp64, int kind, bool energy, int color,
                             int step_k, cudaStream_t st) {
    return fp64 ? halfsweep_t<double>(b, kind, energy, color, step_k, st)
                : halfsweep_t<float>(b, kind, energy, color, step_k, st);
}

cudaError_t launch_energy(const DevBatch& b, bool fp64, cudaStream_t st) {
    if (fp64) k_energy<double><<<b.n_tiles, TILE, 0, st>>>(b);
    else k_energy<float><<<b.n_tiles, TILE, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_energy_finalize(const DevBatch& b, cudaStream_t st) {
    k_energy_finalize<<<(b.n_reps + 127) / 128, 128, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(const DevBatch& b, bool fp64, int ordered, cudaStream_t st) {
    dim3 grid(b.n_tiles, 2);
    if (fp64) k_init_spins<double><<<grid, TILE, 0, st>>>(b, ordered);
    else k_init_spins<float><<<grid, TILE, 0, st>>>(b, ordered);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(const DevBatch& b, int by, cudaStream_t st) {
    k_advance_step<<<1, 1, 0, st>>>(b.d_step, by);
    return cudaGetLastError();
}

cudaError_t launch_overlap(const DevBatch& b, bool fp64, cudaStream_t st) {
    dim3 grid(b.n_tiles, 2);
    if (fp64) k_overlap<double><<<grid, TILE, 0, st>>>(b);
    else k_overlap<float><<<grid, TILE, 0, st>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_overlap_finalize<<<(b.n_reps + 127) / 128, 128, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace ptk
