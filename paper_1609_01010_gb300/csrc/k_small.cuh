// k_small.cuh -- one CTA per product for transform lengths L <= 8192 (a
// launch for one product of L >= 1024 -- a server request or the
// allocation-free entry point -- runs on a cluster instead: k_small_cl.cuh).
//
// The product is laid out as T = L/512 rows of 512 words in shared memory
// (operands a and b side by side).  Steps, all in one launch:
//   1. column stage: TFT over the top log2 T levels with pruning of zero input
//      rows and of rows past k = ceil(n/512) (Section 3's truncation, applied
//      per row of 512 words);
//   2. row stage: one warp per needed row runs the remaining 9 levels of both
//      operands (Stockham passes of radix 16/16/2 in registers), the
//      pointwise product u^_i = g^_i h^_i with the scale folded in, and the
//      unscaled inverse of the 9 levels;
//   3. column stage of the ITFT (step list, in place), then the k*512 >= n
//      outputs are reduced to [0, p) and stored.
// L < 512 is computed as L = 512: the product does not depend on L.
#pragma once
#include "bodies.cuh"
#include "k_small_cl.cuh"

namespace pm {

template <class A, int LOGT>
__global__ void __launch_bounds__(32 << LOGT) k_small(const SmallDesc *__restrict__ descs, SmallDesc one,
                                                      ModParams m, TwTables tw) {
    const SmallDesc d = descs ? descs[blockIdx.x] : one;
    small_body<A, LOGT>(d, m, tw);
}

// A single product with T >= 2 rows runs on a cluster (k_small_cl.cuh);
// descriptor arrays and T = 1 use one CTA per product.
template <class A, int LOGT>
static cudaError_t launch_small_t(const SmallDesc *d_desc, const SmallDesc &one, int count, ModParams m, TwTables tw,
                                  cudaStream_t st) {
    if constexpr (LOGT >= 1) {
        if (!d_desc && count == 1) return launch_small_cl_t<A, LOGT>(one, m, tw, st);
    }
    constexpr int T = 1 << LOGT;
    const size_t smem = (size_t)2 * T * (1 << SMALL_LOG_S) * sizeof(u32);
    cudaError_t e = ensure_smem(k_small<A, LOGT>, smem);
    if (e != cudaSuccess) return e;
    k_small<A, LOGT><<<count, 32 * T, smem, st>>>(d_desc, one, m, tw);
    return cudaGetLastError();
}

template <class A>
static cudaError_t dispatch_small(int logT, const SmallDesc *d_desc, const SmallDesc &one, int count, ModParams m,
                                  TwTables tw, cudaStream_t st) {
    switch (logT) {
        case 0: return launch_small_t<A, 0>(d_desc, one, count, m, tw, st);
        case 1: return launch_small_t<A, 1>(d_desc, one, count, m, tw, st);
        case 2: return launch_small_t<A, 2>(d_desc, one, count, m, tw, st);
        case 3: return launch_small_t<A, 3>(d_desc, one, count, m, tw, st);
        case 4: return launch_small_t<A, 4>(d_desc, one, count, m, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pm
