// bodies.cuh -- CTA bodies of the product kernels, shared by the one-launch
// kernels (k_small.cu, k_large.cu) and the persistent batched kernel
// (batch.cu).
#pragma once
#include "device.cuh"

namespace pm {

// Workspace reads bypass L1 (ld.global.cg): in the persistent kernel another
// CTA may have produced them earlier in the same launch.
__device__ __forceinline__ u32 ld_cg(const u32 *p) { return __ldcg(p); }

// The dynamic shared-memory window of the calling CTA.  Bodies are compiled
// as separate (non-inlined) device functions so the persistent kernel stays
// small; taking the window here keeps shared-memory addressing explicit.
__device__ __forceinline__ u32 *dyn_smem() {
    extern __shared__ __align__(16) u32 pm_dyn_smem[];
    return pm_dyn_smem;
}

// ---------------------------------------------------------- small product
// One product with L = T * 512 <= 8192 (see k_small.cu).  Any blockDim that
// is a multiple of 32; shared memory: 2 * T * 512 words.
template <class A, int LOGT>
__device__ __noinline__ void small_body(const SmallDesc &d, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    constexpr int T = 1 << LOGT;
    constexpr int S = 1 << SMALL_LOG_S;
    u32 *sa = smem, *sb = smem + T * S;
    const u32 p = m.p;
    const int zba = (int)((d.za + S - 1) / S), zbb = (int)((d.zb + S - 1) / S);
    col_fwd_tile<A, S>(sa, d.a, d.za, S, 0, T, LOGT, zba, d.k, d.prune != 0, tw.fwd, p);
    col_fwd_tile<A, S>(sb, d.b, d.zb, S, 0, T, LOGT, zbb, d.k, d.prune != 0, tw.fwd, p);

    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int w = threadIdx.x >> 5; w < d.k; w += nw) {
        constexpr int NP = RowPlan<SMALL_LOG_S, 0>::NP;
        u32 xa[16], xb[16];
        srow_fwd<A, SMALL_LOG_S, 0>(xa, sa + w * S, lane, LOGT, (u32)w, tw.fwd, p);
        srow_fwd<A, SMALL_LOG_S, 0>(xb, sb + w * S, lane, LOGT, (u32)w, tw.fwd, p);
#pragma unroll
        for (int i = 0; i < 16; ++i) xa[i] = A::pointwise(xa[i], xb[i], d.cscale, m);
        srow_inv<A, SMALL_LOG_S, NP - 1>(xa, sa + w * S, lane, LOGT, (u32)w, tw.inv, p);
    }
    __syncthreads();
    col_itft_steps<A, S>(sa, d.steps, d.nsteps, tw.inv, p);
    for (int64_t e = threadIdx.x; e < d.n; e += blockDim.x) d.c[e] = A::to_canon(sa[swz((u32)e)], p);
    __syncthreads();
}

template <class A>
__device__ void small_dispatch(const SmallDesc &d, ModParams m, TwTables tw) {
    switch (d.logT) {
        case 0: small_body<A, 0>(d, m, tw); break;
        case 1: small_body<A, 1>(d, m, tw); break;
        case 2: small_body<A, 2>(d, m, tw); break;
        case 3: small_body<A, 3>(d, m, tw); break;
        default: small_body<A, 4>(d, m, tw); break;
    }
}

// ---------------------------------------------------------- large product
// Column stage of operand `opnd` on column tile `tile` (C columns); writes
// the k needed rows to the workspace.  Shared memory: T * C words.
template <class A, int C>
__device__ __noinline__ void colf_body(const LargeDesc &d, int tile, int opnd, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    const u32 *g = opnd ? d.b : d.a;
    const int64_t z = opnd ? d.zb : d.za;
    u32 *W = opnd ? d.wb : d.wa;
    const int64_t S = d.g.S, c0 = (int64_t)tile * C;
    const int T = (int)d.g.T, t = d.g.t;
    const int k = d.prune ? (int)d.g.k : T;
    int zb = z > c0 ? (int)((z - c0 + S - 1) / S) : 0;
    if (zb > T) zb = T;
    col_fwd_tile<A, C>(smem, g, z, S, c0, T, t, zb, k, d.prune != 0, tw.fwd, m.p);
    for (int tau = threadIdx.x; tau < k * C; tau += blockDim.x) {
        const int r = tau / C, c = tau % C;
        W[(int64_t)r * S + c0 + c] = smem[swz(r * C + c)];
    }
    __syncthreads();
}

// Row ib: remaining sigma levels of both operands, pointwise product,
// unscaled inverse; result overwrites wa's row.  blockDim must be S/16;
// shared memory: 4 * S words.
template <class A, int SIGMA>
__device__ __noinline__ void row_body(const LargeDesc &d, u32 ib, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    constexpr int S = 1 << SIGMA;
    constexpr int NP = RowPlan<SIGMA, 0>::NP;
    u32 *a0 = smem, *a1 = smem + S, *b0 = smem + 2 * S, *b1 = smem + 3 * S;
    const u32 tid = threadIdx.x;
    const u32 p = m.p;
    u32 *rowa = d.wa + (int64_t)ib * S;
    const u32 *rowb = d.wb + (int64_t)ib * S;
    u32 xa[16], xb[16];
    lrow_fwd<A, SIGMA, 0>(xa, rowa, a0, a1, tid, d.g.t, ib, tw.fwd, p);
    lrow_fwd<A, SIGMA, 0>(xb, rowb, b0, b1, tid, d.g.t, ib, tw.fwd, p);
#pragma unroll
    for (int i = 0; i < 16; ++i) xa[i] = A::pointwise(xa[i], xb[i], d.cscale, m);
    lrow_inv<A, SIGMA, NP - 1>(xa, rowa, a0, a1, tid, d.g.t, ib, tw.inv, p);
    __syncthreads();
}

// ITFT column stage of tile `tile` and the store of the first n outputs.
// Shared memory: T * C words.
template <class A, int C>
__device__ __noinline__ void coli_body(const LargeDesc &d, int tile, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    const int64_t S = d.g.S, c0 = (int64_t)tile * C;
    const int T = (int)d.g.T, k = (int)d.g.k;
    for (int tau = threadIdx.x; tau < T * C; tau += blockDim.x) {
        const int r = tau / C, c = tau % C;
        smem[swz(r * C + c)] = r < k ? ld_cg(d.wa + (int64_t)r * S + c0 + c) : 0u;
    }
    __syncthreads();
    col_itft_steps<A, C>(smem, d.steps, d.nsteps, tw.inv, m.p);
    for (int tau = threadIdx.x; tau < k * C; tau += blockDim.x) {
        const int r = tau / C, c = tau % C;
        const int64_t e = (int64_t)r * S + c0 + c;
        if (e < d.n) d.c[e] = A::to_canon(smem[swz(r * C + c)], m.p);
    }
    __syncthreads();
}

}  // namespace pm
