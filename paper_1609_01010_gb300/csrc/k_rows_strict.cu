// k_rows_strict.cu -- row-stage kernels, word-bound (2^30 < p < 2^31) regime.
#include "k_large.cuh"

namespace pm {

cudaError_t launch_row_strict(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    return launch_row<Arith<false>>(d, m, tw, st);
}

}  // namespace pm
