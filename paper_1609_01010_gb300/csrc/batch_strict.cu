// batch_strict.cu -- persistent batched kernel instantiated for the
// word-bound (2^30 < p < 2^31) arithmetic regime.
#include "batch_kernel.cuh"

namespace pm {

cudaError_t launch_batch_strict(int uniform_C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return launch_batch_t<Arith<false>>(uniform_C, P, smem, grid, st);
}

}  // namespace pm
