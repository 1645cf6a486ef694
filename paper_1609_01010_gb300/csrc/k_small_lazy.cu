// k_small_lazy.cu -- one-CTA product kernels instantiated for the
// lazy (p < 2^30) arithmetic regime.
#include "k_small.cuh"

namespace pm {

cudaError_t launch_small_lazy(int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count, ModParams m,
                              TwTables tw, cudaStream_t st) {
    SmallDesc one{};
    if (h_one) one = *h_one;
    return dispatch_small<Arith<true>>(logT, d_desc, one, count, m, tw, st);
}

}  // namespace pm
