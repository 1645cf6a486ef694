// dispatch.cu -- picks the arithmetic regime of a prime: Harvey's lazy
// butterflies when p < 2^30, word-bound ones otherwise.
#include "batch.h"

namespace pm {

cudaError_t launch_small_lazy(int, const SmallDesc *, const SmallDesc *, int, ModParams, TwTables, cudaStream_t);
cudaError_t launch_small_strict(int, const SmallDesc *, const SmallDesc *, int, ModParams, TwTables, cudaStream_t);
cudaError_t launch_large_lazy(const LargeDesc &, Schedule, ModParams, TwTables, cudaStream_t);
cudaError_t launch_large_strict(const LargeDesc &, Schedule, ModParams, TwTables, cudaStream_t);
cudaError_t launch_batch_lazy(int, const BatchParams &, size_t, int *, cudaStream_t);
cudaError_t launch_batch_strict(int, const BatchParams &, size_t, int *, cudaStream_t);

cudaError_t launch_small(bool lazy, int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count,
                         ModParams m, TwTables tw, cudaStream_t st) {
    return lazy ? launch_small_lazy(logT, d_desc, h_one, count, m, tw, st)
                : launch_small_strict(logT, d_desc, h_one, count, m, tw, st);
}

cudaError_t launch_large(bool lazy, const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st) {
    return lazy ? launch_large_lazy(d, sch, m, tw, st) : launch_large_strict(d, sch, m, tw, st);
}

cudaError_t launch_batch(bool lazy, int C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return lazy ? launch_batch_lazy(C, P, smem, grid, st) : launch_batch_strict(C, P, smem, grid, st);
}

}  // namespace pm
