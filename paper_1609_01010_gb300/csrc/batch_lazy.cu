// batch_lazy.cu -- persistent batched kernel instantiated for the
// lazy (p < 2^30) arithmetic regime.
#include "batch_kernel.cuh"

namespace pm {

cudaError_t launch_batch_lazy(int C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    if (C == 128) return launch_batch_t<Arith<true>, 128>(P, smem, grid, st);
    if (C == 32) return launch_batch_t<Arith<true>, 32>(P, smem, grid, st);
    return launch_batch_t<Arith<true>, 8>(P, smem, grid, st);
}

}  // namespace pm
