// dispatch.cu -- picks the arithmetic regime of a prime: Harvey's lazy
// butterflies when p < 2^30, word-bound ones otherwise.
#include <map>
#include <mutex>
#include <tuple>
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
// column-stage launchers, one per (direction, regime, tile width): k_cols.cu
#define PM_DECL_COL(NAME) cudaError_t NAME(const LargeDesc &, ModParams, TwTables, cudaStream_t);
PM_DECL_COL(launch_colf_lazy_c8)
PM_DECL_COL(launch_colf_lazy_c32)
PM_DECL_COL(launch_colf_lazy_c128)
PM_DECL_COL(launch_colf_strict_c8)
PM_DECL_COL(launch_colf_strict_c32)
PM_DECL_COL(launch_colf_strict_c128)
PM_DECL_COL(launch_coli_lazy_c8)
PM_DECL_COL(launch_coli_lazy_c32)
PM_DECL_COL(launch_coli_lazy_c128)
PM_DECL_COL(launch_coli_strict_c8)
PM_DECL_COL(launch_coli_strict_c32)
PM_DECL_COL(launch_coli_strict_c128)
#undef PM_DECL_COL

static cudaError_t launch_col(bool fwd, bool lazy, int C, const LargeDesc &d, ModParams m, TwTables tw,
                              cudaStream_t st) {
    if (fwd) {
        if (lazy) {
            if (C == 8) return launch_colf_lazy_c8(d, m, tw, st);
            if (C == 32) return launch_colf_lazy_c32(d, m, tw, st);
            if (C == 128) return launch_colf_lazy_c128(d, m, tw, st);
        } else {
            if (C == 8) return launch_colf_strict_c8(d, m, tw, st);
            if (C == 32) return launch_colf_strict_c32(d, m, tw, st);
            if (C == 128) return launch_colf_strict_c128(d, m, tw, st);
        }
    } else {
        if (lazy) {
            if (C == 8) return launch_coli_lazy_c8(d, m, tw, st);
            if (C == 32) return launch_coli_lazy_c32(d, m, tw, st);
            if (C == 128) return launch_coli_lazy_c128(d, m, tw, st);
        } else {
            if (C == 8) return launch_coli_strict_c8(d, m, tw, st);
            if (C == 32) return launch_coli_strict_c32(d, m, tw, st);
            if (C == 128) return launch_coli_strict_c128(d, m, tw, st);
        }
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_row_lazy(const LargeDesc &, ModParams, TwTables, cudaStream_t);
cudaError_t launch_row_strict(const LargeDesc &, ModParams, TwTables, cudaStream_t);
cudaError_t launch_batch_lazy(int, const BatchParams &, size_t, int *, cudaStream_t);
cudaError_t launch_batch_strict(int, const BatchParams &, size_t, int *, cudaStream_t);

cudaError_t persistent_grid(const void *kern, int threads, size_t smem, int items, int *grid) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t, int>, int> cache;  // -> CTAs per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto key = std::make_tuple(kern, threads, smem, dev);
    int total = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) total = it->second;
    }
    if (!total) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        total = (per_sm < 1 ? 1 : per_sm) * sms;
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = total;
    }
    *grid = items < total ? items : total;
    if (*grid < 1) *grid = 1;
    return cudaSuccess;
}

cudaError_t launch_small(bool lazy, int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count,
                         ModParams m, TwTables tw, cudaStream_t st) {
    return lazy ? launch_small_lazy(logT, d_desc, h_one, count, m, tw, st)
                : launch_small_strict(logT, d_desc, h_one, count, m, tw, st);
}

// The three kernels of a large product on one stream; ev (optional) gets
// events before the column stage and after each kernel.
cudaError_t launch_large(bool lazy, const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                         cudaEvent_t *ev) {
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], st);
    e = launch_col(true, lazy, sch.C, d, m, tw, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    e = lazy ? launch_row_lazy(d, m, tw, st) : launch_row_strict(d, m, tw, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    e = launch_col(false, lazy, sch.C, d, m, tw, st);
    if (ev) cudaEventRecord(ev[3], st);
    return e;
}

cudaError_t launch_batch(bool lazy, int C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return lazy ? launch_batch_lazy(C, P, smem, grid, st) : launch_batch_strict(C, P, smem, grid, st);
}

}  // namespace pm
