// evc_bulk.cuh -- sm_90+/sm_103a asynchronous bulk copies (global -> shared,
// cp.async.bulk with mbarrier completion) and bounded mbarrier waits, written
// as inline PTX for the streaming kernels.
//
// Every wait is bounded: after kWaitCycles SM clock cycles (about a second)
// the waiting thread records DERR_TIMEOUT in the run's error flag and the
// kernel winds down instead of spinning forever.
#pragma once

#include <cstdint>

namespace evc {

constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make the barrier initialisation visible to the async (bulk-copy) proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Orders this thread's generic-proxy writes to shared memory before later
// async-proxy accesses (a bulk copy that overwrites the same bytes).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false once `cycles`
// SM clock cycles have passed without it.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long cycles)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    return mbar_wait_for(bar, parity, kWaitCycles);
}

// The same wait taken by all 32 lanes of a warp with one outcome: a lane that
// gave up makes the whole warp give up, so the lanes never split at a
// following __syncwarp or shuffle.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity)
{
    return __all_sync(0xffffffffu, mbar_wait(bar, parity));
}

// bytes (multiple of 16) from 16-byte aligned global src to 16-byte aligned
// shared dst; completion counted on bar as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace evc
