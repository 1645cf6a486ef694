// k_large.cuh -- the three-kernel path (single products from L = 1024 up;
// in batches and the server from L = 16384 up).
//
// L = T * S with rows of S = 2^sigma words (sigma = 9..13) and T <= 2048.
//   k_col_fwd   grid (S/C, 2): column stage of TFT(a) and TFT(b) on tiles of
//               C columns, pruned to the input support and to the k needed
//               rows; writes rows [0, k) of each operand to the workspace.
//   k_row_fused grid (k):      one CTA per needed row: remaining sigma levels
//               of both operands, pointwise product with the scale folded in,
//               unscaled inverse of the sigma levels; overwrites wa's row.
//   k_col_itft  grid (S/C):    ITFT column stage (a full inverse when k = T,
//               else the truncated one of coli_tile_ct), then the first n
//               outputs reduced to [0, p).
// Each kernel reads its inputs once from HBM/L2 and writes its outputs once.
// All three are launched with programmatic stream serialization: each stages
// its twiddles before waiting for the previous kernel (griddepcontrol.wait).
#pragma once
#include "bodies.cuh"

namespace pm {

constexpr int COL_THREADS = 128;   // k_col_fwd
constexpr int COLI_THREADS = 256;  // k_col_itft: more warps per tile for its mostly latency-bound passes
// 2 * T * C * 4 bytes of tiles (at most 128 KB, schedule_valid's bound) and
// up to 16 KB of column twiddles.
constexpr size_t COL_SMEM_MAX = 144 * 1024;

// Persistent column kernels: each CTA walks items blockIdx.x, +gridDim.x, ...
// and double-buffers them: the cp.async copies of the next item are in
// flight while the current one computes.  TL = column depth (compile time).
// Copies the column tree's 2^TL table entries (levels < TL) into shared
// memory behind the two tile buffers; the first barrier of the tile loop
// publishes it.
template <int TL>
__device__ __forceinline__ uint2 *stage_col_tw(u32 *smem, u32 words, const uint2 *table) {
    uint2 *s = reinterpret_cast<uint2 *>(smem + 2 * words);
    for (int i = threadIdx.x; i < (1 << TL); i += blockDim.x) s[i] = i ? __ldg(table + i) : make_uint2(0u, 0u);
    return s;
}

template <int C, int TL>
constexpr size_t col_smem_bytes() {
    return (size_t)2 * ((size_t)C << TL) * sizeof(u32) + ((size_t)8 << TL);
}

template <class A, int C, int TL>
__global__ void __launch_bounds__(COL_THREADS, 6) k_col_fwd(const LargeDesc d, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    pdl_launch_dependents();  // the row kernel may start staging its twiddles
    const u32 words = (u32)C << TL;
    tw.fwd = stage_col_tw<TL>(smem, words, tw.fwd);
    // Launched with programmatic stream serialization: the operands (and the
    // workspace, which the stream-ordered pool may hand over from the
    // previous product) are touched only after the previous kernel on the
    // stream has completed.
    pdl_wait();
    const int items = 2 * (int)(d.g.S / C);  // (tile, operand) pairs
    int it = blockIdx.x;
    if (it < items) colf_load<C>(d, it >> 1, it & 1, smem);
    cp_async_commit();
    for (int kb = 0; it < items; it += gridDim.x, kb ^= 1) {
        const int nx = it + gridDim.x;
        if (nx < items) colf_load<C>(d, nx >> 1, nx & 1, smem + (kb ^ 1) * words);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        colf_compute_ct<A, C, TL>(d, it >> 1, it & 1, smem + kb * words, m, tw);
    }
}

// Resident CTAs per SM the row kernel is compiled for.  E = 16: what its
// shared memory (S words of exchange buffer + S twiddles of 8 bytes) allows,
// so registers never limit it further; E = 4 or 8 (S/E threads per row):
// 64 registers a thread, at most 16 CTAs.
constexpr int row_min_blocks(int sigma, int E = 16) {
    return E == 16 ? (sigma >= 13 ? 2 : (sigma == 12 ? 4 : (sigma == 11 ? 8 : 16)))
                   : (65536 / (64 * ((1 << sigma) / E)) < 16 ? 65536 / (64 * ((1 << sigma) / E)) : 16);
}

template <class A, int SIGMA, int E = 16>
__global__ void __launch_bounds__((1 << SIGMA) / E, row_min_blocks(SIGMA, E)) k_row_fused(const LargeDesc d, ModParams m, TwTables tw) {
    pdl_launch_dependents();
    row_body<A, SIGMA, E>(d, blockIdx.x, m, tw);
}

// Words per thread of the row stage: 16 (one 512-word row per warp) when the
// product has rows enough to fill the GPU, fewer -- more threads per row, a
// shorter chain of dependent butterflies in each -- when its k rows x S/16
// threads would leave most SMs with a warp or two (rows of up to 2^11 words).
constexpr int ROW_E4_MAX_THREADS = 152 * 64;    // k S / 16 below this: E = 4
constexpr int ROW_E8_MAX_THREADS = 152 * 256;   // below this: E = 8
inline int row_words_per_thread(int sigma, int64_t k) {
    if (sigma > 11) return 16;
    const int64_t threads16 = k << (sigma - 4);
    return threads16 < ROW_E4_MAX_THREADS ? 4 : (threads16 < ROW_E8_MAX_THREADS ? 8 : 16);
}

template <class A, int C, int TL>
__global__ void __launch_bounds__(COLI_THREADS, 3) k_col_itft(const LargeDesc d, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    __shared__ uint2 top[16];  // the top three levels' twiddles (see ColInvArgs::top)
    if (threadIdx.x < 16) {
        const int e = threadIdx.x & 7;
        top[threadIdx.x] = e == 0 ? make_uint2(0u, 0u) : __ldg((threadIdx.x < 8 ? tw.fwd : tw.inv) + e);
    }
    const u32 words = (u32)C << TL;
    tw.inv = stage_col_tw<TL>(smem, words, tw.inv);
    pdl_wait();  // the product rows come from the row kernel
    const int items = (int)(d.g.S / C);
    int it = blockIdx.x;
    if (it < items) coli_load<C>(d, it, smem);
    cp_async_commit();
    for (int kb = 0; it < items; it += gridDim.x, kb ^= 1) {
        const int nx = it + gridDim.x;
        if (nx < items) coli_load<C>(d, nx, smem + (kb ^ 1) * words);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        coli_compute_ct<A, C, TL>(d, it, smem + kb * words, m, tw, top);
    }
    // Only now may the next kernel on the stream (the next product's column
    // kernel) be scheduled: launched at the start, its CTAs would take SM
    // slots while this kernel still runs and slow mid-size products.
    pdl_launch_dependents();
}

// ------------------------------------------------------------ launchers
// Launch with programmatic stream serialization: the kernel may begin (and
// run up to its pdl_wait) while the previous kernel on the stream finishes.
template <typename... Args>
static cudaError_t launch_pdl(void (*kern)(Args...), int grid, int threads, size_t smem, cudaStream_t st,
                              const LargeDesc &d, ModParams m, TwTables tw) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, d, m, tw);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class A, int C, int TL>
static cudaError_t launch_colf_c(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    const size_t smem = col_smem_bytes<C, TL>();
    cudaError_t e = ensure_smem(k_col_fwd<A, C, TL>, COL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    int grid = 0;
    e = persistent_grid((const void *)k_col_fwd<A, C, TL>, COL_THREADS, smem, 2 * (int)(d.g.S / C), &grid);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_col_fwd<A, C, TL>, grid, COL_THREADS, smem, st, d, m, tw);
}

template <class A, int C, int TL>
static cudaError_t launch_coli_c(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    const size_t smem = col_smem_bytes<C, TL>();
    cudaError_t e = ensure_smem(k_col_itft<A, C, TL>, COL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    int grid = 0;
    e = persistent_grid((const void *)k_col_itft<A, C, TL>, COLI_THREADS, smem, (int)(d.g.S / C), &grid);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_col_itft<A, C, TL>, grid, COLI_THREADS, smem, st, d, m, tw);
}

// t in 1..11 (schedule_valid); C in {8, 32, 128}.
template <class A, int C, bool FWD>
static cudaError_t launch_col_t(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
#define PM_COL_CASE(TLV) \
    case TLV: return FWD ? launch_colf_c<A, C, TLV>(d, m, tw, st) : launch_coli_c<A, C, TLV>(d, m, tw, st);
    switch (d.g.t) {
        PM_COL_CASE(1)
        PM_COL_CASE(2)
        PM_COL_CASE(3)
        PM_COL_CASE(4)
        PM_COL_CASE(5)
        PM_COL_CASE(6)
        PM_COL_CASE(7)
        PM_COL_CASE(8)
        PM_COL_CASE(9)
        PM_COL_CASE(10)
        PM_COL_CASE(11)
        default: return cudaErrorInvalidValue;
    }
#undef PM_COL_CASE
}

template <class A, int SIGMA, int E>
static cudaError_t launch_rows_e(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    constexpr int S = 1 << SIGMA;
    const size_t smem = row_smem_bytes(SIGMA, E);
    cudaError_t e = ensure_smem(k_row_fused<A, SIGMA, E>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_row_fused<A, SIGMA, E>, (int)d.g.k, S / E, smem, st, d, m, tw);
}

template <class A, int SIGMA>
static cudaError_t launch_rows(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    if constexpr (SIGMA <= 11) {
        const int E = row_words_per_thread(SIGMA, d.g.k);
        if (E == 4) return launch_rows_e<A, SIGMA, 4>(d, m, tw, st);
        if (E == 8) return launch_rows_e<A, SIGMA, 8>(d, m, tw, st);
    }
    return launch_rows_e<A, SIGMA, 16>(d, m, tw, st);
}

template <class A>
static cudaError_t launch_row(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    switch (d.g.sigma) {
        case 9: return launch_rows<A, 9>(d, m, tw, st);
        case 10: return launch_rows<A, 10>(d, m, tw, st);
        case 11: return launch_rows<A, 11>(d, m, tw, st);
        case 12: return launch_rows<A, 12>(d, m, tw, st);
        case 13: return launch_rows<A, 13>(d, m, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pm
