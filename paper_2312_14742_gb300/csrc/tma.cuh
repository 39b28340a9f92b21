// Tensor-memory-accelerator (TMA) loads into shared memory, completed on an
// mbarrier, for the staged tiled kernel.
//
// One thread issues a tiled 3D bulk copy of a box of the state into shared
// memory; the copy reports its bytes to an mbarrier of that buffer, and every
// thread waits for the barrier's phase before reading the box. Waits are
// bounded: a wait that runs past its limit returns false; the kernel then
// counts a timeout in its caller's device counter (StepArgs::timeouts, read
// and cleared by the host, which reports LBM_ETIMEOUT), stops issuing copies
// and storing, so that a missing completion can never hang the GPU.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace lbm {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the given phase parity; gives up after about 2^31 clock cycles
// (about one second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < (1ll << 31))
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Tiled 3D copy of the box at element coordinates (c0, c1, c2) into dst
// (128-byte aligned shared memory); completion is counted on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace lbm
