// fr_tma.cuh -- Tensor Memory Accelerator (TMA) tile loads and mbarrier
// waits for the streaming kernels.
//
// A 2-D tensor map describes a row-major fp32 grid; one elected thread issues
// cp.async.bulk.tensor loads of boxes into shared memory, each completing on an
// mbarrier with the box's byte count.  Boxes may start outside the grid (the
// halo of an edge tile); those elements read NaN, which no comparison finds
// strictly lower, exactly as the +inf border of the scalar kernels.  Every
// wait is bounded by the GPU's global timer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace fr {

// Host: a 2-D tiled tensor map over a float32 grid [ny][nx] with boxes of
// box_x x box_y elements and NaN out-of-bounds fill.  Requires nx % 4 == 0
// and a 16-byte aligned base (the row stride must be a multiple of 16 bytes).
bool encode_tile_map_f32(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int box_x,
                         int box_y);

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the async proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a block barrier) before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}" : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long tma_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the barrier for at most limit_ns; false if the
// limit ran out first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tma_global_ns();
    while (!mbar_try_wait(bar, parity))
        if (tma_global_ns() - t0 > limit_ns) return false;
    return true;
}

}  // namespace fr
