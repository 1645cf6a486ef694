// dispatch.cu -- picks the arithmetic regime of a prime: Harvey's lazy
// butterflies when p < 2^30, word-bound ones otherwise.
#include <map>
#include <mutex>
#include <utility>

#include "batch.h"

namespace pm {

cudaError_t ensure_smem_ptr(const void *kern, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(kern, dev);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

cudaError_t launch_small_lazy(int, const SmallDesc *, const SmallDesc *, int, ModParams, TwTables, cudaStream_t);
cudaError_t launch_small_strict(int, const SmallDesc *, const SmallDesc *, int, ModParams, TwTables, cudaStream_t);
cudaError_t launch_large_lazy(const LargeDesc &, Schedule, ModParams, TwTables, cudaStream_t, cudaEvent_t *);
cudaError_t launch_large_strict(const LargeDesc &, Schedule, ModParams, TwTables, cudaStream_t, cudaEvent_t *);
cudaError_t launch_batch_lazy(int, const BatchParams &, size_t, int *, cudaStream_t);
cudaError_t launch_batch_strict(int, const BatchParams &, size_t, int *, cudaStream_t);

cudaError_t launch_small(bool lazy, int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count,
                         ModParams m, TwTables tw, cudaStream_t st) {
    return lazy ? launch_small_lazy(logT, d_desc, h_one, count, m, tw, st)
                : launch_small_strict(logT, d_desc, h_one, count, m, tw, st);
}

cudaError_t launch_large(bool lazy, const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                         cudaEvent_t *ev) {
    return lazy ? launch_large_lazy(d, sch, m, tw, st, ev) : launch_large_strict(d, sch, m, tw, st, ev);
}

cudaError_t launch_batch(bool lazy, int C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return lazy ? launch_batch_lazy(C, P, smem, grid, st) : launch_batch_strict(C, P, smem, grid, st);
}

}  // namespace pm
