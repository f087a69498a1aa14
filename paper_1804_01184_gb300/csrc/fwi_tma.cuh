// fwi_tma.cuh -- TMA row pipeline for the row-streaming kernels (sm_103a).
//
// One elected thread issues 1-D bulk copies (cp.async.bulk, the TMA engine) of whole
// computational rows into shared-memory rings, D rows ahead of the consumers; each stage
// completes on an mbarrier (expect_tx).  Consumers wait with a bounded try_wait loop: on
// expiry they raise ST_ETIMEOUT and the CTA leaves after the next barrier.  Issued stages
// are always consumed, so no copy is in flight when a CTA exits normally.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fwi {

enum : int { ST_ETIMEOUT = 4 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// async-proxy writes after generic-proxy accesses of the same shared memory
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait: false after ~2^22 polls (each poll may suspend the thread for a while)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int k = 0; k < (1 << 22); ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace fwi
