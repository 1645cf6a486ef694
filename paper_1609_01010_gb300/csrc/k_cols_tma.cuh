// k_cols_tma.cuh -- column stages of the three-kernel path fed by the Tensor
// Memory Accelerator (the schedules with 32-column tiles).
//
// A tile is 32 columns x T rows of one operand (TFT) or of the product's
// workspace rows (ITFT), row-major in shared memory: 128 bytes per row, so a
// half-warp reading two adjacent columns of 16 column pairs covers one whole
// row and every access pattern of the passes is free of bank conflicts with
// no address swizzle.  One CTA of 512 threads per SM walks the tiles
// persistently through a ring of TCOL stages (two while a tile fits 64 KB):
// thread 0 issues the next tiles' cp.async.bulk.tensor loads as soon as a
// stage is free, so the loads of tile i+1 run under the arithmetic of tile i.
// The tile passes themselves are the compile-time-shaped ones of the other
// column kernels (colf_tile_ct / coli_tile_ct at C = 32).
//
// Operands whose address is not 16-byte aligned (or that hold less than one
// full row) have no tensor map; their tiles are loaded by the threads with
// cp.async instead, one tile at a time.
#pragma once
#include "bodies.cuh"
#include "tma.cuh"

namespace pm {

constexpr int TC = 32;  // tile width (columns)
constexpr int TCOL_THREADS = 512;  // threads per CTA (measured: 1024 spills in the forward passes, no faster inverse)
constexpr long long TMA_WAIT_LIMIT = 1LL << 24;

// Tensor maps of one column stage.  TFT: m[0], m[1] describe operands a and b
// as [full rows][S]; ITFT: m[0] describes the k workspace rows of the
// product.  rows[o]: the rows the loads cover (a multiple of box[o], at most
// T); the map's own row count ends earlier where the data does, and TMA
// fills the rows past it with zeros.
struct ColMaps {
    CUtensorMap m[2];
    int ok[2];    // 1: a valid map (else the threads load the tile)
    int rows[2];  // rows loaded per tile
    int box[2];   // rows per box (<= 256)
};

template <int TL>
__host__ __device__ constexpr int tcol_stages() {
    return ((size_t)TC << TL) * 4 <= 64 * 1024 ? 2 : 1;
}
// 1 KB of alignment slack, the tile stages, the column tree's twiddles
// (2^TL entries), 16 entries of the ITFT's top levels and the mbarriers.
template <int TL>
__host__ __device__ constexpr size_t tcol_smem_bytes() {
    return 1024 + (size_t)tcol_stages<TL>() * ((size_t)TC << TL) * 4 + ((size_t)8 << TL) + 16 * 8 + 64;
}

struct TcolSmem {
    u32 *tiles;
    uint2 *ctw;
    uint2 *top;
    uint64_t *bar;
};

template <int TL>
__device__ __forceinline__ TcolSmem tcol_smem() {
    u32 *raw = dyn_smem();
    const u32 a = smem_u32(raw);
    u32 *base = raw + (((a + 1023u) & ~1023u) - a) / 4;  // TMA destinations 1024-byte aligned
    TcolSmem s;
    s.tiles = base;
    s.ctw = reinterpret_cast<uint2 *>(base + (size_t)tcol_stages<TL>() * ((u32)TC << TL));
    s.top = s.ctw + (1 << TL);
    s.bar = reinterpret_cast<uint64_t *>(s.top + 16);
    return s;
}

// Thread 0: the loads of item `it`'s tile of operand `o` into stage buffer
// `buf`, signalling `bar`.
__device__ __forceinline__ void tcol_issue(const ColMaps &cm, int o, int tile, u32 *buf, uint64_t *bar) {
    const int rows = cm.rows[o], br = cm.box[o];
    PM_DCHECK(br >= 1 && br <= 256 && rows % br == 0, (int *)nullptr);
    mbar_arrive_expect_tx(bar, (u32)rows * TC * 4);
    for (int y = 0; y < rows; y += br) tma_load_2d(buf + y * TC, &cm.m[o], tile * TC, y, bar);
}

// The ragged last row of an operand (z not a multiple of S): TMA filled it
// with zeros (it lies past the map's full rows); its valid columns of this
// tile come from global memory.
__device__ __forceinline__ void tcol_patch_partial(const LargeDesc &d, int o, int tile, u32 *buf, int rows) {
    const u32 *g = o ? d.b : d.a;
    const int64_t z = o ? d.zb : d.za;
    const int64_t S = d.g.S;
    const int64_t zfull = z / S;
    if (zfull >= rows) return;
    const int64_t c0 = (int64_t)tile * TC, valid = z - zfull * S - c0;
    if (valid <= 0) return;
    for (int c = threadIdx.x; c < TC && c < valid; c += blockDim.x) buf[zfull * TC + c] = __ldg(g + zfull * S + c0 + c);
}

template <class A, int TL>
__global__ void __launch_bounds__(TCOL_THREADS, 1)
    k_col_fwd_tma(const LargeDesc d, ModParams m, TwTables tw, const __grid_constant__ ColMaps cm) {
    constexpr int ST = tcol_stages<TL>();
    constexpr u32 words = (u32)TC << TL;
    const TcolSmem sm = tcol_smem<TL>();
    pdl_launch_dependents();  // the row kernel may start staging its twiddles
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(sm.bar + s, 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < (1 << TL); i += blockDim.x) sm.ctw[i] = i ? __ldg(tw.fwd + i) : make_uint2(0u, 0u);
    tw.fwd = sm.ctw;
    __syncthreads();
    // The operands (and the workspace, which the stream-ordered pool may hand
    // over from the previous product) are touched only after the previous
    // kernel on the stream has completed.
    pdl_wait();
    const int items = 2 * (int)(d.g.S / TC);  // (tile, operand) pairs
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            const int it = blockIdx.x + s * gridDim.x;
            if (it < items && cm.ok[it & 1]) tcol_issue(cm, it & 1, it >> 1, sm.tiles + s * words, sm.bar + s);
        }
    }
    u32 phase = 0;  // bit s: parity of the next completion of stage s
    int i = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++i) {
        const int s = i % ST, tile = it >> 1, o = it & 1;
        u32 *buf = sm.tiles + s * words;
        bool ok = true;
        if (cm.ok[o]) {
            ok = mbar_wait_bounded(sm.bar + s, (phase >> s) & 1u, tw.status, TMA_WAIT_LIMIT);
            phase ^= 1u << s;
            if (ok) tcol_patch_partial(d, o, tile, buf, cm.rows[o]);
        } else {
            colf_load<TC>(d, tile, o, buf);
            cp_async_wait_all();
        }
        if (!__syncthreads_and(ok)) {
            // A load that never completed: record it (done by the waiter) and
            // give it one more bounded wait before this CTA may leave, so no
            // copy lands in shared memory after exit.
            if (threadIdx.x == 0) mbar_wait_bounded(sm.bar + s, ((phase >> s) & 1u) ^ 1u, nullptr, TMA_WAIT_LIMIT);
            return;
        }
        colf_compute_ct<A, TC, TL>(d, tile, o, buf, m, tw);
        // The passes' shared-memory accesses of this buffer precede the next
        // load into it (generic proxy before the asynchronous proxy).
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nx = it + ST * gridDim.x;
            if (nx < items && cm.ok[nx & 1]) tcol_issue(cm, nx & 1, nx >> 1, buf, sm.bar + s);
        }
    }
}

template <class A, int TL>
__global__ void __launch_bounds__(TCOL_THREADS, 1)
    k_col_itft_tma(const LargeDesc d, ModParams m, TwTables tw, const __grid_constant__ ColMaps cm) {
    constexpr int ST = tcol_stages<TL>();
    constexpr u32 words = (u32)TC << TL;
    const TcolSmem sm = tcol_smem<TL>();
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(sm.bar + s, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 16) {  // the top three levels' twiddles (see ColInvArgs::top)
        const int e = threadIdx.x & 7;
        sm.top[threadIdx.x] = e == 0 ? make_uint2(0u, 0u) : __ldg((threadIdx.x < 8 ? tw.fwd : tw.inv) + e);
    }
    for (int i = threadIdx.x; i < (1 << TL); i += blockDim.x) sm.ctw[i] = i ? __ldg(tw.inv + i) : make_uint2(0u, 0u);
    tw.inv = sm.ctw;
    __syncthreads();
    pdl_wait();  // the product rows come from the row kernel
    const int items = (int)(d.g.S / TC);
    if (threadIdx.x == 0 && cm.ok[0]) {
        for (int s = 0; s < ST; ++s) {
            const int it = blockIdx.x + s * gridDim.x;
            if (it < items) tcol_issue(cm, 0, it, sm.tiles + s * words, sm.bar + s);
        }
    }
    int i = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++i) {
        const int s = i % ST;
        u32 *buf = sm.tiles + s * words;
        bool ok = true;
        if (cm.ok[0]) {
            ok = mbar_wait_bounded(sm.bar + s, (u32)(i / ST) & 1u, tw.status, TMA_WAIT_LIMIT);
        } else {
            coli_load<TC>(d, it, buf);
            cp_async_wait_all();
        }
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) mbar_wait_bounded(sm.bar + s, ((u32)(i / ST) & 1u) ^ 1u, nullptr, TMA_WAIT_LIMIT);
            return;
        }
        coli_compute_ct<A, TC, TL>(d, it, buf, m, tw, sm.top);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && cm.ok[0]) {
            const int nx = it + ST * gridDim.x;
            if (nx < items) tcol_issue(cm, 0, nx, buf, sm.bar + s);
        }
    }
    // Only now may the next kernel on the stream (the next product's column
    // kernel) be scheduled: see k_col_itft.
    pdl_launch_dependents();
}

// ------------------------------------------------------------ launchers
template <class A, int TL, bool FWD>
static cudaError_t launch_tcol_tl(const LargeDesc &d, ModParams m, TwTables tw, const ColMaps &cm, cudaStream_t st) {
    void (*kern)(const LargeDesc, ModParams, TwTables, const ColMaps);
    if constexpr (FWD) kern = k_col_fwd_tma<A, TL>;
    else kern = k_col_itft_tma<A, TL>;
    const size_t smem = tcol_smem_bytes<TL>();
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int grid = 0;
    const int items = (FWD ? 2 : 1) * (int)(d.g.S / TC);
    e = persistent_grid((const void *)kern, TCOL_THREADS, smem, items, &grid);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(TCOL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, d, m, tw, cm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// t in 1..10 (a tile of 32 x 2^t words fits shared memory for t <= 10).
template <class A, bool FWD>
static cudaError_t launch_tcol(const LargeDesc &d, ModParams m, TwTables tw, const ColMaps &cm, cudaStream_t st) {
#define PM_TCOL_CASE(TLV) \
    case TLV: return launch_tcol_tl<A, TLV, FWD>(d, m, tw, cm, st);
    switch (d.g.t) {
        PM_TCOL_CASE(1)
        PM_TCOL_CASE(2)
        PM_TCOL_CASE(3)
        PM_TCOL_CASE(4)
        PM_TCOL_CASE(5)
        PM_TCOL_CASE(6)
        PM_TCOL_CASE(7)
        PM_TCOL_CASE(8)
        PM_TCOL_CASE(9)
        PM_TCOL_CASE(10)
        default: return cudaErrorInvalidValue;
    }
#undef PM_TCOL_CASE
}

}  // namespace pm
