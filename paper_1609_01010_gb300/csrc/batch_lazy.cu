// batch_lazy.cu -- persistent batched kernel instantiated for the
// lazy (p < 2^30) arithmetic regime.
#include "batch_kernel.cuh"

namespace pm {

cudaError_t launch_batch_lazy(int uniform_C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return launch_batch_t<Arith<true>>(uniform_C, P, smem, grid, st);
}

}  // namespace pm
