// k_small_cl.cuh -- one product with 1024 <= L <= 8192 on a thread-block
// cluster of Q = min(T, 8) CTAs (T = L/512 rows of 512 words), one launch.
//
// The one-CTA kernel (k_small.cuh) runs the whole product on one SM, which
// makes these sizes latency-bound on that SM's issue slots.  Here the same
// steps are spread over Q SMs, with the two transposes of the row/column
// decomposition going through distributed shared memory:
//   1. CTA q copies columns [q*512/Q, (q+1)*512/Q) of all T rows of both
//      operands into shared memory by cp.async, together with its rows'
//      twiddles, the column tree's twiddles and the ITFT step list, and runs
//      the column stage of the TFT on them (pruned to the input support and
//      the k needed rows);
//   2. cluster barrier; CTA q gathers its T/Q rows (rows < k) from the Q
//      column tiles, and all its threads (512/E per row, E = 4 or 8 words
//      each) run the 9 row levels of both operands, the pointwise product
//      (prescaled for the truncated inverse, see row_scale) and the unscaled
//      inverse row levels;
//   3. cluster barrier; CTA q gathers its columns of the product rows back
//      from the Q row buffers; cluster barrier (no CTA leaves while another
//      may still read its shared memory);
//   4. the ITFT column stage (step list) on the tile, and the store of the
//      first n coefficients in its columns.
#pragma once
#include <cooperative_groups.h>

#include "bodies.cuh"

namespace pm {

constexpr int SMALL_CL_THREADS = 128;

template <int LOGT>
struct SmallCl {
    static constexpr int T = 1 << LOGT;
    static constexpr int Q = T < 8 ? T : 8;        // CTAs in the cluster
    static constexpr int S = 1 << SMALL_LOG_S;     // row length
    static constexpr int CP = S / Q;               // columns per CTA
    static constexpr int RPC = T / Q;              // rows per CTA
    static constexpr int TILE = T * CP;            // words of one operand's column tile
    static constexpr int ROWS = RPC * S;           // words of one operand's row buffer
    static constexpr int E = S * RPC / SMALL_CL_THREADS;  // row words per thread in the row stage
    // two tiles, two row buffers, and each row's forward and inverse twiddles
    // (S - 1 entries of 8 bytes each, stage_tw layout)
    static constexpr size_t SMEM = (size_t)(2 * TILE + 2 * ROWS) * sizeof(u32) + (size_t)RPC * 2 * S * sizeof(uint2);
    static_assert(E == 4 || E == 8, "row stage: 4 or 8 words per thread");
};

// Step records of the ITFT copied to shared memory (longer lists are read
// from global memory).
constexpr int SMALL_CL_MAX_STEPS = 32;

// Issues the copies of one operand's column tile (rows r < T, columns
// c0..c0+CP, LAY_SWZ layout) into shared memory; entries at or past the
// operand's length z are zeros.  16-byte copies where the operand allows.
template <class G>
__device__ __forceinline__ void cl_load_tile(const u32 *g, int64_t z, u32 c0, u32 *tile) {
    const bool al = (((uintptr_t)g) & 15u) == 0;
    constexpr int CH = G::CP / 4;  // 4-word chunks per row
    for (int i = threadIdx.x; i < G::T * CH; i += blockDim.x) {
        const int r = i / CH, c = (i % CH) * 4;
        u32 *dst = tile + swz((u32)(r * G::CP + c));
        const int64_t e = (int64_t)r * G::S + c0 + c;
        if (e >= z) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        } else if (al && e + 4 <= z) {
            cp_async16(dst, g + e);
        } else {
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (e + w < z) cp_async4(dst + w, g + e + w);
                else dst[w] = 0u;
            }
        }
    }
}

template <class A, int LOGT>
__global__ void __launch_bounds__(SMALL_CL_THREADS) k_small_cl(SmallDesc d, ModParams m, TwTables tw) {
    namespace cg = cooperative_groups;
    using G = SmallCl<LOGT>;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    u32 *smem = dyn_smem();
    u32 *tile_a = smem, *tile_b = smem + G::TILE;
    u32 *rows_a = smem + 2 * G::TILE, *rows_b = rows_a + G::ROWS;
    uint2 *rtw = reinterpret_cast<uint2 *>(rows_b + G::ROWS);  // row w: forward at rtw + 2wS, inverse + S
    const u32 p = m.p;
    const u32 c0 = (u32)q * G::CP;
    const int k = d.k;
    const int r0 = q * G::RPC;

    // 0. copies issued up front, all in flight together: both operands'
    // column tiles, this CTA's rows' twiddles (used in step 2) and the ITFT
    // step list (step 4)
    cl_load_tile<G>(d.a, d.za, c0, tile_a);
    cl_load_tile<G>(d.b, d.zb, c0, tile_b);
    for (int w = 0; w < G::RPC; ++w) {
        if (r0 + w >= k) break;
        stage_tw<SMALL_LOG_S>(rtw + 2 * w * G::S, tw.fwd, LOGT, (u32)(r0 + w));
        stage_tw<SMALL_LOG_S>(rtw + (2 * w + 1) * G::S, tw.inv, LOGT, (u32)(r0 + w));
    }
    cp_async_commit();
    __shared__ __align__(16) ItftStep s_steps[SMALL_CL_MAX_STEPS];
    // the column tree's forward and inverse twiddles (levels < t: table
    // entries [0, T)), read by every task of the column passes
    __shared__ uint2 s_ctw[2][G::T];
    if (threadIdx.x < G::T) {  // entry 0 is not a tree node
        s_ctw[0][threadIdx.x] = threadIdx.x ? __ldg(tw.fwd + threadIdx.x) : make_uint2(0u, 0u);
        s_ctw[1][threadIdx.x] = threadIdx.x ? __ldg(tw.inv + threadIdx.x) : make_uint2(0u, 0u);
    }
    const bool steps_in_smem = d.nsteps <= SMALL_CL_MAX_STEPS;
    if (steps_in_smem) {
        constexpr int W4 = (int)(sizeof(ItftStep) / sizeof(uint4));
        for (int i = threadIdx.x; i < d.nsteps * W4; i += blockDim.x)
            reinterpret_cast<uint4 *>(s_steps)[i] = __ldg(reinterpret_cast<const uint4 *>(d.steps) + i);
    }
    cp_async_wait_all();
    __syncthreads();

    // 1. column stage of both operands on this CTA's columns (t <= 4 levels:
    // one pass, from the tiles in shared memory)
    {
        const int S = G::S;
        const int zba = (int)((d.za + S - 1) / S), zbb = (int)((d.zb + S - 1) / S);
        ColFwdArgs X{tile_a, d.a, nullptr, d.za, c0, SMALL_LOG_S, G::T, LOGT, zba, k, d.prune != 0, s_ctw[0], p,
                     tw.status};
        colf_pass_r<A, G::CP, LAY_SWZ, IO_SMEM, IO_SMEM, true>(LOGT, X, 0);
        X.sm = tile_b;
        X.g = d.b;
        X.z = d.zb;
        X.zb = zbb;
        colf_pass_r<A, G::CP, LAY_SWZ, IO_SMEM, IO_SMEM, true>(LOGT, X, 0);
    }
    cl.sync();

    // 2. gather this CTA's rows, row stage, pointwise, inverse rows.  The
    // loop is unrolled so all of a thread's remote loads are in flight at once.
    static_assert(G::ROWS % (4 * SMALL_CL_THREADS) == 0 && G::TILE % (4 * SMALL_CL_THREADS) == 0,
                  "whole gather rounds of 16-byte chunks");
    // 16-byte chunks: swz keeps 4-word aligned runs together in both layouts.
#pragma unroll
    for (int i = 0; i < G::ROWS / 4 / SMALL_CL_THREADS; ++i) {
        const int e = 4 * ((int)threadIdx.x + i * SMALL_CL_THREADS);
        const int rl = e / G::S, c = e % G::S, r = r0 + rl;
        if (r < k) {
            const int owner = c / G::CP, lc = c % G::CP;
            const u32 at = swz((u32)(r * G::CP + lc));
            const u32 *ra = cl.map_shared_rank(tile_a, owner);
            const u32 *rb = cl.map_shared_rank(tile_b, owner);
            *reinterpret_cast<uint4 *>(rows_a + rl * G::S + swz((u32)c)) = *reinterpret_cast<const uint4 *>(ra + at);
            *reinterpret_cast<uint4 *>(rows_b + rl * G::S + swz((u32)c)) = *reinterpret_cast<const uint4 *>(rb + at);
        }
    }
    __syncthreads();
    {
        // every thread of the CTA works on one of its RPC rows: S/E threads
        // per row, E words each (E = 4 with one row per CTA, 8 with two)
        constexpr int E = G::E, NT = G::S / E;
        constexpr int NP = RowPlan<SMALL_LOG_S, 0, E>::NP;
        const int w = threadIdx.x / NT, lt = threadIdx.x % NT;
        const int r = r0 + w;
        const bool on = r < k;
        const uint2 *ftw = rtw + 2 * w * G::S, *itw = ftw + G::S;
        u32 xa[E], xb[E];
        srowc_fwd<A, SMALL_LOG_S, E, 0>(xa, rows_a + w * G::S, lt, on, ftw, p);
        srowc_fwd<A, SMALL_LOG_S, E, 0>(xb, rows_b + w * G::S, lt, on, ftw, p);
        if (on) {
            const uint2 cs = row_scale(tw, SMALL_LOG_S, (u32)r, (u32)k);
#pragma unroll
            for (int i = 0; i < E; ++i) xa[i] = A::pointwise(xa[i], xb[i], cs, m);
        }
        srowc_inv<A, SMALL_LOG_S, E, NP - 1>(xa, rows_a + w * G::S, lt, on, itw, p);
    }
    cl.sync();

    // 3. gather this CTA's columns of the product rows back into tile_a
#pragma unroll
    for (int i = 0; i < G::TILE / 4 / SMALL_CL_THREADS; ++i) {
        const int e = 4 * ((int)threadIdx.x + i * SMALL_CL_THREADS);
        const int r = e / G::CP, lc = e % G::CP;
        if (r < k) {
            const int owner = r / G::RPC, rl = r % G::RPC;
            const u32 *src = cl.map_shared_rank(rows_a, owner);
            *reinterpret_cast<uint4 *>(tile_a + swz((u32)(r * G::CP + lc))) =
                *reinterpret_cast<const uint4 *>(src + rl * G::S + swz(c0 + (u32)lc));
        }
    }
    cl.sync();

    // 4. ITFT column stage and store
    const ColInvArgs Y{tile_a, nullptr, d.c, d.n, c0, SMALL_LOG_S, k, s_ctw[1], p, s_ctw[0], nullptr, tw.status};
    coli_steps<A, G::CP, LAY_SWZ, true>(Y, steps_in_smem ? s_steps : d.steps, d.nsteps);
    for (int e = threadIdx.x; e < k * G::CP; e += blockDim.x) {
        const int r = e / G::CP, lc = e % G::CP;
        const int64_t o = (int64_t)r * G::S + c0 + lc;
        PM_DCHECK(tile_a[swz((u32)(r * G::CP + lc))] < A::bound(p), tw.status);
        if (o < d.n) d.c[o] = A::to_canon(tile_a[swz((u32)(r * G::CP + lc))], p);
    }
}

template <class A, int LOGT>
static cudaError_t launch_small_cl_t(const SmallDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    using G = SmallCl<LOGT>;
    cudaError_t e = ensure_smem(k_small_cl<A, LOGT>, G::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G::Q, 1, 1);
    cfg.blockDim = dim3(SMALL_CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_small_cl<A, LOGT>, d, m, tw);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace pm
