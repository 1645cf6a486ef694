// tma.cuh -- Tensor Memory Accelerator loads and mbarrier waits (sm_90+ PTX,
// used here on sm_103a).
//
// A 2-D tensor map describes an operand (or workspace) as rows of S words;
// one cp.async.bulk.tensor instruction copies a box of (columns x rows)
// words into shared memory, row-major and dense, and signals an mbarrier
// with the number of bytes written.  Rows outside the map's row count are
// filled with zeros (and cost no memory traffic).  Every wait on an mbarrier
// is bounded: on expiry the waiter records POLY_ETIMEOUT in the library's
// device status word and the kernel skips the work that needed the data.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "internal.h"

namespace pm {

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the asynchronous proxy (TMA).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls the mbarrier phase `parity` at most `limit` times (each try_wait may
// itself suspend the thread for a short, hardware-chosen time).  Returns
// false (after recording POLY_ETIMEOUT in *status) if the phase never
// completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, u32 parity, int *status, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicExch(status, -6 /* POLY_ETIMEOUT */);
    return false;
}

// Box (x = first column, y = first row) of a 2-D map into shared memory.
// x * 4 bytes must be a multiple of 16 (x a multiple of 4 words).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace pm
