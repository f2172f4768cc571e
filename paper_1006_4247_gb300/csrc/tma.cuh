// tma.cuh -- the Tensor Memory Accelerator's bulk copies between global and
// shared memory (cp.async.bulk) and the shared-memory barriers (mbarrier)
// that count their bytes, as used by the engine's kernels.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace ptk {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit) {
    for (unsigned long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from this CTA's shared memory to global memory, in the thread's current
// bulk async-group.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the thread's committed bulk copies have read their shared-memory
// source (the buffer may then be reused or released).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Bounded wait by every calling thread for phase `parity` of an mbarrier that
// counts the bytes of bulk loads; true if the phase completed.  If the wait
// gives up, the error word gets bit 0 and, when copies were issued, a second
// bounded wait gives them a chance to land before the caller skips the work
// that needed them (and, eventually, releases the shared memory).  Threads
// may disagree, so callers combine the results over the CTA (or cluster).
__device__ __forceinline__ bool mbar_wait_io(unsigned long long* bar, unsigned parity, const DevBatch& a,
                                             bool issued = true) {
    if (mbar_wait_bounded(bar, parity, a.wait_limit)) return true;
    atomicOr(a.err, 1);
    if (issued) mbar_wait_bounded(bar, parity, a.wait_limit > WAIT_LIMIT_DEFAULT ? a.wait_limit : WAIT_LIMIT_DEFAULT);
    return false;
}

}  // namespace ptk
