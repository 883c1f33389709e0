// tma.cuh -- Tensor Memory Accelerator (TMA) 2-D tile loads into shared
// memory with mbarrier completion, as inline PTX for sm_103a.
//
// A strip's domain window is fetched by one cp.async.bulk.tensor issued by
// one lane; the copy signals an mbarrier with its byte count and the warp
// waits on the barrier's phase.  Every wait is bounded: after kSpinLimit
// polls it reports failure instead of spinning forever.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fic {

// 128-byte opaque tensor map (CUtensorMap), 64-byte aligned in global memory.
struct alignas(64) TmaMap {
    uint64_t w[16];
};
static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "tensor map size");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy writes (a TMA into a buffer that was just read).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2-D tiled load of box (x, y) of the tensor map into shared memory.  x must
// be a multiple of 16 elements of 1 byte (16-byte rule of the innermost
// coordinate); elements outside the tensor read as zero.
__device__ __forceinline__ void tma_load_2d(void *dst, const TmaMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of the barrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_test_parity(bar, parity)) return true;
        if (it > 8) __nanosleep(32);
    }
    return false;
}

}  // namespace fic
