// noalloc.cu -- energy reduction over caller-owned device buffers that
// allocates nothing (pt_energy_noalloc in include/pt.h).
//
// Some callers cannot call cudaMalloc: code embedded in another framework
// whose memory pool must account for every device byte (a library that
// allocates behind its back breaks the budget), and latency-critical loops
// that forbid allocation after start-up because cudaMalloc may synchronise
// the device and has no bounded latency.  For them this variant of the
// engine's energy reduction keeps its per-block partial sums in a fixed
// file-scope device array instead of engine-owned scratch.
//
// The array holds kMaxPartials doubles (512 KiB).  Every GPU that loads this
// library keeps it until the process exits.  Every call writes each partial
// it later reads, so nothing has to start at zero, but all calls share the
// one array: calls that overlap on the GPU (different streams, or different
// host threads on the same device) race and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/pt.h"
#include "kernels.h"

namespace {

constexpr int kMaxPartials = 65536;
constexpr int kThreads = 256;
constexpr int kSitesPerBlock = 2048;  // 8 sites per thread
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxPartials];

// Device address of g_partials per device (host code may not use the symbol
// itself as an address), looked up once per device with that device current.
double* g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Block b handles configuration b / bpc, sites [(b % bpc) * kSitesPerBlock, ...):
// partial = - sum over its sites x and mu of J[mu][x] s_x . s_{x + e_mu}.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_energy_partials(const T* __restrict__ spins,
                                                              const float* __restrict__ J, int L,
                                                              int bpc, double* __restrict__ part) {
    __shared__ double sh[kThreads / 32];
    const int cfg = blockIdx.x / bpc, blk = blockIdx.x % bpc;
    const int N = L * L * L;
    const T* s = spins + (long long)cfg * 3 * N;
    double e = 0.0;
    const int end = min(N, (blk + 1) * kSitesPerBlock);
    for (int x = blk * kSitesPerBlock + (int)threadIdx.x; x < end; x += kThreads) {
        const int i = x % L, j = (x / L) % L, k = x / (L * L);
        const int nb[3] = {(i + 1 == L ? 0 : i + 1) + L * (j + L * k),
                           i + L * ((j + 1 == L ? 0 : j + 1) + L * k),
                           i + L * (j + L * (k + 1 == L ? 0 : k + 1))};
        const T sx = s[3 * x], sy = s[3 * x + 1], sz = s[3 * x + 2];
        T acc = (T)0;
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const T* t = s + 3 * nb[mu];
            acc += (T)J[(long long)mu * N + x] * (sx * t[0] + sy * t[1] + sz * t[2]);
        }
        e -= (double)acc;
    }
    e = warp_sum_d(e);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// energy[c] = sum of the partials of configuration c, in block order.
__global__ void k_energy_partials_finalize(const double* __restrict__ part, int n_configs, int bpc,
                                           double* __restrict__ energy) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_configs) return;
    double H = 0.0;
    for (int b = 0; b < bpc; ++b) H += part[(long long)c * bpc + b];
    energy[c] = H;
}

pt_status nerr(pt_status st, const char* msg) {
    ptk::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" pt_status pt_energy_noalloc(const void* d_spins, int precision, int L, int n_configs,
                                       const float* d_couplings, double* d_energy, void* stream) {
    char buf[256];
    if (precision != PT_FP32 && precision != PT_FP64) return nerr(PT_ERR_ARG, "pt_energy_noalloc: bad precision");
    if (L < 2 || L > 512) return nerr(PT_ERR_ARG, "pt_energy_noalloc: L must be in [2, 512]");
    if (n_configs < 0) return nerr(PT_ERR_ARG, "pt_energy_noalloc: n_configs < 0");
    if (n_configs == 0) return PT_OK;
    if (!d_spins || !d_couplings || !d_energy) return nerr(PT_ERR_ARG, "pt_energy_noalloc: NULL pointer");
    const long long N = (long long)L * L * L;
    const long long bpc = (N + kSitesPerBlock - 1) / kSitesPerBlock;
    if ((long long)n_configs * bpc > kMaxPartials) {
        snprintf(buf, sizeof buf,
                 "pt_energy_noalloc: %d configurations of L = %d need %lld partial sums; the fixed scratch "
                 "holds %d (at most %lld configurations of this size per call)",
                 n_configs, L, (long long)n_configs * bpc, kMaxPartials, (long long)kMaxPartials / bpc);
        return nerr(PT_ERR_ARG, buf);
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return nerr(PT_ERR_CUDA, cudaGetErrorString(ce));
    if (dev < 0 || dev >= kMaxDevices) return nerr(PT_ERR_ARG, "pt_energy_noalloc: device index too large");
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void* p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_partials);
            if (ce != cudaSuccess) {
                snprintf(buf, sizeof buf, "pt_energy_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(ce));
                return nerr(PT_ERR_CUDA, buf);
            }
            g_partials_addr[dev] = static_cast<double*>(p);
        }
        part = g_partials_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)((long long)n_configs * bpc);
    if (precision == PT_FP64)
        k_energy_partials<double><<<blocks, kThreads, 0, st>>>((const double*)d_spins, d_couplings, L, (int)bpc, part);
    else
        k_energy_partials<float><<<blocks, kThreads, 0, st>>>((const float*)d_spins, d_couplings, L, (int)bpc, part);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) {
        k_energy_partials_finalize<<<(n_configs + 127) / 128, 128, 0, st>>>(part, n_configs, (int)bpc, d_energy);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        snprintf(buf, sizeof buf, "pt_energy_noalloc: launch failed: %s", cudaGetErrorString(ce));
        return nerr(PT_ERR_CUDA, buf);
    }
    return PT_OK;
}
