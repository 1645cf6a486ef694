// k_small_cl.cuh -- one product with 1024 <= L <= 8192 on a thread-block
// cluster of Q = min(T, 8) CTAs (T = L/512 rows of 512 words), one launch.
//
// The one-CTA kernel (k_small.cuh) runs the whole product on one SM, which
// makes these sizes latency-bound on that SM's issue slots.  Here the same
// steps are spread over Q SMs, with the two transposes of the row/column
// decomposition going through distributed shared memory:
//   1. CTA q holds columns [q*512/Q, (q+1)*512/Q) of all T rows of both
//      operands and runs the column stage of the TFT on them (pruned to the
//      input support and the k needed rows);
//   2. cluster barrier; CTA q gathers its T/Q rows (rows < k) from the Q
//      column tiles, and one warp per row runs the 9 row levels of both
//      operands, the pointwise product (prescaled for the truncated inverse,
//      see row_scale) and the unscaled inverse row levels;
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
    static constexpr size_t SMEM = (size_t)(2 * TILE + 2 * ROWS) * sizeof(u32);
};

template <class A, int LOGT>
__global__ void __launch_bounds__(SMALL_CL_THREADS) k_small_cl(SmallDesc d, ModParams m, TwTables tw) {
    namespace cg = cooperative_groups;
    using G = SmallCl<LOGT>;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    u32 *smem = dyn_smem();
    u32 *tile_a = smem, *tile_b = smem + G::TILE;
    u32 *rows_a = smem + 2 * G::TILE, *rows_b = rows_a + G::ROWS;
    const u32 p = m.p;
    const u32 c0 = (u32)q * G::CP;
    const int k = d.k;

    // 1. column stage of both operands on this CTA's columns
    {
        const int S = G::S;
        const int zba = (int)((d.za + S - 1) / S), zbb = (int)((d.zb + S - 1) / S);
        ColFwdArgs X{tile_a, d.a, nullptr, d.za, c0, SMALL_LOG_S, G::T, LOGT, zba, k, d.prune != 0, tw.fwd, p,
                     tw.status};
        colf_tile<A, G::CP, LAY_SWZ>(X, false);
        X.sm = tile_b;
        X.g = d.b;
        X.z = d.zb;
        X.zb = zbb;
        colf_tile<A, G::CP, LAY_SWZ>(X, false);
    }
    cl.sync();

    // 2. gather this CTA's rows, row stage, pointwise, inverse rows
    const int r0 = q * G::RPC;
    for (int e = threadIdx.x; e < G::ROWS; e += blockDim.x) {
        const int rl = e / G::S, c = e % G::S, r = r0 + rl;
        if (r >= k) continue;
        const int owner = c / G::CP, lc = c % G::CP;
        const u32 at = swz((u32)(r * G::CP + lc));
        const u32 *ra = cl.map_shared_rank(tile_a, owner);
        const u32 *rb = cl.map_shared_rank(tile_b, owner);
        rows_a[rl * G::S + swz((u32)c)] = ra[at];
        rows_b[rl * G::S + swz((u32)c)] = rb[at];
    }
    __syncthreads();
    {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int r = r0 + w;
        if (w < G::RPC && r < k) {
            constexpr int NP = RowPlan<SMALL_LOG_S, 0>::NP;
            u32 xa[16], xb[16];
            srow_fwd<A, SMALL_LOG_S, 0>(xa, rows_a + w * G::S, lane, LOGT, (u32)r, tw.fwd, p);
            srow_fwd<A, SMALL_LOG_S, 0>(xb, rows_b + w * G::S, lane, LOGT, (u32)r, tw.fwd, p);
            const uint2 cs = row_scale(tw, SMALL_LOG_S, (u32)r, (u32)k);
#pragma unroll
            for (int i = 0; i < 16; ++i) xa[i] = A::pointwise(xa[i], xb[i], cs, m);
            srow_inv<A, SMALL_LOG_S, NP - 1>(xa, rows_a + w * G::S, lane, LOGT, (u32)r, tw.inv, p);
        }
    }
    cl.sync();

    // 3. gather this CTA's columns of the product rows back into tile_a
    for (int e = threadIdx.x; e < G::TILE; e += blockDim.x) {
        const int r = e / G::CP, lc = e % G::CP;
        if (r >= k) continue;
        const int owner = r / G::RPC, rl = r % G::RPC;
        const u32 *src = cl.map_shared_rank(rows_a, owner);
        tile_a[swz((u32)(r * G::CP + lc))] = src[rl * G::S + swz(c0 + (u32)lc)];
    }
    cl.sync();

    // 4. ITFT column stage and store
    const ColInvArgs Y{tile_a, nullptr, d.c, d.n, c0, SMALL_LOG_S, k, tw.inv, p, tw.fwd, nullptr, tw.status};
    coli_steps<A, G::CP, LAY_SWZ>(Y, d.steps, d.nsteps);
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
