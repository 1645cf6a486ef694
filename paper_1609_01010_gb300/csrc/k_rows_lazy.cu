// k_rows_lazy.cu -- row-stage kernels, lazy (p < 2^30) regime.
#include "k_large.cuh"

namespace pm {

cudaError_t launch_row_lazy(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    return launch_row<Arith<true>>(d, m, tw, st);
}

}  // namespace pm
