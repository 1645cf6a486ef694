// k_small_strict.cu -- one-CTA product kernels instantiated for the
// word-bound (2^30 < p < 2^31) arithmetic regime.
#include "k_small.cuh"

namespace pm {

cudaError_t launch_small_strict(int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count, ModParams m,
                              TwTables tw, cudaStream_t st) {
    SmallDesc one{};
    if (h_one) one = *h_one;
    return dispatch_small<Arith<false>>(logT, d_desc, one, count, m, tw, st);
}

}  // namespace pm
