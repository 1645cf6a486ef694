// dispatch.cu -- picks the arithmetic regime of a prime: Harvey's lazy
// butterflies when p < 2^30, word-bound ones otherwise.
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "batch.h"
#include "k_cols_tma.cuh"

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
PM_DECL_COL(launch_colf_lazy_c128)
PM_DECL_COL(launch_colf_strict_c8)
PM_DECL_COL(launch_colf_strict_c128)
PM_DECL_COL(launch_coli_lazy_c8)
PM_DECL_COL(launch_coli_lazy_c128)
PM_DECL_COL(launch_coli_strict_c8)
PM_DECL_COL(launch_coli_strict_c128)
#undef PM_DECL_COL

static cudaError_t launch_col(bool fwd, bool lazy, int C, const LargeDesc &d, ModParams m, TwTables tw,
                              cudaStream_t st) {
    if (fwd) {
        if (lazy) {
            if (C == 8) return launch_colf_lazy_c8(d, m, tw, st);
            if (C == 128) return launch_colf_lazy_c128(d, m, tw, st);
        } else {
            if (C == 8) return launch_colf_strict_c8(d, m, tw, st);
            if (C == 128) return launch_colf_strict_c128(d, m, tw, st);
        }
    } else {
        if (lazy) {
            if (C == 8) return launch_coli_lazy_c8(d, m, tw, st);
            if (C == 128) return launch_coli_lazy_c128(d, m, tw, st);
        } else {
            if (C == 8) return launch_coli_strict_c8(d, m, tw, st);
            if (C == 128) return launch_coli_strict_c128(d, m, tw, st);
        }
    }
    return cudaErrorInvalidValue;
}
// TMA-fed column-stage launchers (32-column tiles): k_cols_tma.cu
#define PM_DECL_TCOL(NAME) cudaError_t NAME(const LargeDesc &, ModParams, TwTables, const ColMaps &, cudaStream_t);
PM_DECL_TCOL(launch_tcolf_lazy)
PM_DECL_TCOL(launch_tcolf_strict)
PM_DECL_TCOL(launch_tcoli_lazy)
PM_DECL_TCOL(launch_tcoli_strict)
#undef PM_DECL_TCOL

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

// ------------------------------------------------------------ tensor maps
// cuTensorMapEncodeTiled from the driver, fetched once through the runtime
// (the library links no driver library of its own).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

// Map of `rows` full rows of S words at `base` (boxes of 32 columns x box
// rows); false where TMA cannot describe it (no encoder, base not 16-byte
// aligned, no full row), and the kernel then loads that operand's tiles
// with its threads.
static bool encode_rows(CUtensorMap *m, const void *base, int64_t S, int64_t rows, int box) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || rows < 1 || (((uintptr_t)base) & 15u) != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)S * 4};
    cuuint32_t boxd[2] = {(cuuint32_t)TC, (cuuint32_t)box};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(base), dims, strides, boxd, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int pow2_at_least(int64_t x) {
    int r = 1;
    while (r < x) r <<= 1;
    return r;
}

// TFT column stage: operand o's tiles load rows [0, T'), T' the smallest
// power of two holding its nonzero rows (every level above T' is a copy of
// zeros the column passes skip), or all T rows for the unpruned comparator.
static void col_maps_fwd(const LargeDesc &d, ColMaps *cm) {
    const int64_t S = d.g.S, T = d.g.T;
    for (int o = 0; o < 2; ++o) {
        const u32 *g = o ? d.b : d.a;
        const int64_t z = o ? d.zb : d.za;
        const int64_t nz = (z + S - 1) / S;
        const int rows = d.prune ? (int)std::min<int64_t>(T, pow2_at_least(nz)) : (int)T;
        const int box = rows < 256 ? rows : 256;
        cm->rows[o] = rows;
        cm->box[o] = box;
        cm->ok[o] = encode_rows(&cm->m[o], g, S, z / S, box) ? 1 : 0;
    }
}

// ITFT column stage: the k workspace rows of the product, in boxes of at
// most 256 rows (rows past k read as zeros and are never used).
static void col_maps_inv(const LargeDesc &d, ColMaps *cm) {
    const int64_t S = d.g.S, T = d.g.T, k = d.g.k;
    const int box = T < 256 ? (int)T : 256;
    cm->rows[0] = (int)((k + box - 1) / box * box);
    cm->box[0] = box;
    cm->ok[0] = encode_rows(&cm->m[0], d.wa, S, k, box) ? 1 : 0;
    cm->ok[1] = 0;
    cm->rows[1] = cm->box[1] = 0;
}

// The three kernels of a large product on one stream; ev (optional) gets
// events before the column stage and after each kernel.  Schedules with
// 32-column tiles (t <= 10) run the TMA-fed column kernels.
cudaError_t launch_large(bool lazy, const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                         cudaEvent_t *ev) {
    cudaError_t e;
    const bool tma = sch.C == TC && d.g.t >= 1 && d.g.t <= 10;
    // The inverse column stage runs on the TMA-fed 32-column tiles also after
    // an 8- or 128-column forward stage when the rows are long enough to give
    // at least 128 tiles (S >= 4096): 36.96 against 37.38 us per product at
    // L = 2^21; with 64 tiles (L = 2^20, S = 2048) it was slower, 25.9 against
    // 23.9 us.
    const bool tma_inv = d.g.t >= 1 && d.g.t <= 10 && (sch.C == TC || d.g.S >= 4096);
    ColMaps cm;
    if (ev) cudaEventRecord(ev[0], st);
    if (tma) {
        memset(&cm, 0, sizeof cm);
        col_maps_fwd(d, &cm);
        e = lazy ? launch_tcolf_lazy(d, m, tw, cm, st) : launch_tcolf_strict(d, m, tw, cm, st);
    } else {
        e = launch_col(true, lazy, sch.C, d, m, tw, st);
    }
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    e = lazy ? launch_row_lazy(d, m, tw, st) : launch_row_strict(d, m, tw, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    if (tma_inv) {
        memset(&cm, 0, sizeof cm);
        col_maps_inv(d, &cm);
        e = lazy ? launch_tcoli_lazy(d, m, tw, cm, st) : launch_tcoli_strict(d, m, tw, cm, st);
    } else {
        e = launch_col(false, lazy, sch.C, d, m, tw, st);
    }
    if (ev) cudaEventRecord(ev[3], st);
    return e;
}

cudaError_t launch_batch(bool lazy, int uniform_C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st) {
    return lazy ? launch_batch_lazy(uniform_C, P, smem, grid, st) : launch_batch_strict(uniform_C, P, smem, grid, st);
}

}  // namespace pm
