// batch_strict.cu -- persistent batched kernel instantiated for the
// word-bound (2^30 < p < 2^31) arithmetic regime.
#include "batch_kernel.cuh"

namespace pm {

cudaError_t launch_batch_strict(int C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    if (C == 128) return launch_batch_t<Arith<false>, 128>(P, smem, grid, st);
    if (C == 32) return launch_batch_t<Arith<false>, 32>(P, smem, grid, st);
    return launch_batch_t<Arith<false>, 8>(P, smem, grid, st);
}

}  // namespace pm
