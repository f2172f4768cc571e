// probe.cu -- measured throughput of the SM's shared-memory data path, the
// unit that bounds the resident sweep blocks (every half sweep of a resident
// replica runs out of shared memory), so that their roofline is taken against
// a number measured on the device instead of a datasheet figure
// (pt_smem_bandwidth in include/pt.h).  Not a step of the method.
//
// Every SM runs two CTAs of 512 threads; each thread streams 16-byte loads
// over a 32 KB shared array in an order that is free of bank conflicts (the
// 32 lanes of a warp read 512 consecutive bytes, four full wavefronts) and
// adds them up so that the loads cannot be dropped.  Bytes / elapsed time on
// the stream's CUDA events give the device's rate; clock64 and the global
// timer around the loop give the SM clock the CTAs ran at and the bytes per
// clock per SM.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "../../include/pt.h"
#include "kernels.h"

namespace {

constexpr int kThreads = 512;
constexpr int kBufF4 = 2048;  // float4 elements: 32 KB per CTA

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kThreads, 2) k_smem_stream(int iters, float* sink, unsigned long long* clk) {
    __shared__ float4 buf[kBufF4];
    for (int q = (int)threadIdx.x; q < kBufF4; q += kThreads)
        buf[q] = make_float4((float)q, (float)(q & 7), 1.0f, 0.5f);
    __syncthreads();
    const unsigned long long c0 = clock64(), g0 = global_ns();
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    for (int it = 0; it < iters; ++it) {
        const int i0 = ((int)threadIdx.x + it * 64) & (kBufF4 - 1);
        const int i1 = (i0 + kBufF4 / 2) & (kBufF4 - 1);
        const float4 v = buf[i0], w = buf[i1];
        a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
        b.x += w.x; b.y += w.y; b.z += w.z; b.w += w.w;
    }
    __syncthreads();
    const unsigned long long c1 = clock64(), g1 = global_ns();
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = g1 - g0;
    }
    const float s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
    if (s == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = s;  // never true for these values
}

pt_status perr(pt_status st, const char* what, cudaError_t ce) {
    char buf[256];
    snprintf(buf, sizeof buf, "pt_smem_bandwidth: %s: %s", what, cudaGetErrorString(ce));
    ptk::set_last_error(buf);
    return st;
}

}  // namespace

extern "C" pt_status pt_smem_bandwidth(void* stream, double* bytes_per_s, double* bytes_per_clock_sm,
                                       double* sm_mhz) {
    int dev = 0, nsm = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return perr(PT_ERR_CUDA, "device query", ce);
    const int blocks = 2 * nsm, iters = 8192;
    cudaStream_t st = (cudaStream_t)stream;
    float* sink = nullptr;
    unsigned long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pt_status out = PT_OK;
    double best = 0.0, best_bpc = 0.0, best_mhz = 0.0;
    std::vector<unsigned long long> h((size_t)2 * blocks);
    do {
        if ((ce = cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * kThreads)) != cudaSuccess ||
            (ce = cudaMalloc((void**)&clk, sizeof(unsigned long long) * 2 * (size_t)blocks)) != cudaSuccess) {
            out = perr(PT_ERR_NOMEM, "cudaMalloc", ce);
            break;
        }
        if ((ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess) {
            out = perr(PT_ERR_CUDA, "cudaEventCreate", ce);
            break;
        }
        for (int rep = 0; rep < 4 && out == PT_OK; ++rep) {  // the first launch is a warm-up
            cudaEventRecord(e0, st);
            k_smem_stream<<<blocks, kThreads, 0, st>>>(iters, sink, clk);
            cudaEventRecord(e1, st);
            if ((ce = cudaGetLastError()) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess) {
                out = perr(PT_ERR_CUDA, "probe launch", ce);
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if ((ce = cudaMemcpy(h.data(), clk, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost)) !=
                cudaSuccess) {
                out = perr(PT_ERR_CUDA, "cudaMemcpy", ce);
                break;
            }
            if (rep == 0 || ms <= 0.f) continue;
            const double bytes = (double)blocks * kThreads * iters * 2.0 * 16.0;
            const double rate = bytes / (ms * 1e-3);
            unsigned long long cmax = 0;
            double mhz = 0.0;
            for (int b = 0; b < blocks; ++b) {
                cmax = h[2 * b] > cmax ? h[2 * b] : cmax;
                if (h[2 * b + 1] > 0) mhz += (double)h[2 * b] / (double)h[2 * b + 1] * 1e3;
            }
            if (rate > best) {
                best = rate;
                best_bpc = cmax > 0 ? bytes / ((double)nsm * (double)cmax) : 0.0;
                best_mhz = mhz / blocks;
            }
        }
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (out != PT_OK) return out;
    if (bytes_per_s) *bytes_per_s = best;
    if (bytes_per_clock_sm) *bytes_per_clock_sm = best_bpc;
    if (sm_mhz) *sm_mhz = best_mhz;
    return PT_OK;
}
