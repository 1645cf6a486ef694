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

// The pointwise constant of row r (of k computed rows of 2^sigma words):
// 2^32 / (2^sigma * h) mod p, where 2^sigma undoes the unscaled row inverse
// and h is the size of the FULL record of the truncated inverse that covers
// row r (k's binary expansion splits rows [0, k) into aligned blocks of
// decreasing powers of two; r lies in the block of size 2^b with b the top
// bit of r ^ k).  k = T gives the plain 1/L.
__device__ __forceinline__ uint2 row_scale(const TwTables &tw, int sigma, u32 r, u32 k) {
    return __ldg(tw.pscale + sigma + (31 - __clz(r ^ k)));
}

// ---------------------------------------------------------- small product
// One product with L = T * 512 <= 8192 (see k_small.cu).  Any blockDim that
// is a multiple of 32; shared memory: 2 * T * 512 words.
template <class A, int LOGT>
__device__ __forceinline__ void small_body(const SmallDesc &d, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    constexpr int T = 1 << LOGT;
    constexpr int S = 1 << SMALL_LOG_S;
    u32 *sa = smem, *sb = smem + T * S;
    const u32 p = m.p;
    const int zba = (int)((d.za + S - 1) / S), zbb = (int)((d.zb + S - 1) / S);
    ColFwdArgs X{sa, d.a, nullptr, d.za, 0u, SMALL_LOG_S, T, LOGT, zba, d.k, d.prune != 0, tw.fwd, p, tw.status};
    colf_tile<A, S, LAY_SWZ>(X, false);
    X.sm = sb;
    X.g = d.b;
    X.z = d.zb;
    X.zb = zbb;
    colf_tile<A, S, LAY_SWZ>(X, false);

    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int w = threadIdx.x >> 5; w < d.k; w += nw) {
        constexpr int NP = RowPlan<SMALL_LOG_S, 0>::NP;
        u32 xa[16], xb[16];
        srow_fwd<A, SMALL_LOG_S, 0>(xa, sa + w * S, lane, LOGT, (u32)w, tw.fwd, p);
        srow_fwd<A, SMALL_LOG_S, 0>(xb, sb + w * S, lane, LOGT, (u32)w, tw.fwd, p);
        const uint2 cs = row_scale(tw, SMALL_LOG_S, (u32)w, (u32)d.k);
#pragma unroll
        for (int i = 0; i < 16; ++i) xa[i] = A::pointwise(xa[i], xb[i], cs, m);
        srow_inv<A, SMALL_LOG_S, NP - 1>(xa, sa + w * S, lane, LOGT, (u32)w, tw.inv, p);
    }
    __syncthreads();
    const ColInvArgs Y{sa, nullptr, d.c, d.n, 0u, SMALL_LOG_S, d.k, tw.inv, p, tw.fwd, nullptr, tw.status};
    coli_steps<A, S, LAY_SWZ>(Y, d.steps, d.nsteps);
    for (int64_t e = threadIdx.x; e < d.n; e += blockDim.x) {
        PM_DCHECK(sa[swz((u32)e)] < A::bound(p) && e < ((int64_t)T << SMALL_LOG_S), tw.status);
        d.c[e] = A::to_canon(sa[swz((u32)e)], p);
    }
    __syncthreads();
}

// Out-of-line copies for the persistent batched kernel (keeps it small;
// the one-launch kernels inline the bodies).
template <class A, int LOGT>
__device__ __noinline__ void small_body_ool(const SmallDesc d, ModParams m, TwTables tw) {
    small_body<A, LOGT>(d, m, tw);
}

template <class A>
__device__ void small_dispatch(const SmallDesc &d, ModParams m, TwTables tw) {
    switch (d.logT) {
        case 0: small_body_ool<A, 0>(d, m, tw); break;
        case 1: small_body_ool<A, 1>(d, m, tw); break;
        case 2: small_body_ool<A, 2>(d, m, tw); break;
        case 3: small_body_ool<A, 3>(d, m, tw); break;
        default: small_body_ool<A, 4>(d, m, tw); break;
    }
}

// ---------------------------------------------------------- large product
// Column stage of operand `opnd` on column tile `tile` (C columns); writes
// the k needed rows to the workspace.  Shared memory: T * C words.
// Issues the cp.async copies of column tile `tile` of operand `opnd` (rows
// r < T, columns c0..c0+C) into buf (LAY_TILE); entries at or past the
// operand's length are written as zeros.  16-byte copies when the operand is
// 16-byte aligned, 4-byte copies otherwise (packed batch operands).
template <int C>
__device__ __forceinline__ void colf_load(const LargeDesc &d, int tile, int opnd, u32 *buf) {
    const u32 *g = opnd ? d.b : d.a;
    const int64_t z = opnd ? d.zb : d.za;
    const u32 c0 = (u32)tile * C;
    const int logS = d.g.sigma;
    const bool al = (((uintptr_t)g) & 15u) == 0;
    constexpr int logCH = ilog2c(C) - 2;  // 4-word chunks per row
    const int nch = (int)d.g.T << logCH;
    for (int i = threadIdx.x; i < nch; i += blockDim.x) {
        const u32 r = (u32)i >> logCH, c = ((u32)i & ((1u << logCH) - 1u)) << 2;
        u32 *dst = buf + col_elem_addr<C, LAY_TILE>(r, c);
        const int64_t e = ((int64_t)r << logS) + c0 + c;
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

// Column stage of a tile already in buf; the last pass writes rows < k of
// the workspace.  Ends with a barrier.
template <class A, int C>
__device__ __forceinline__ void colf_compute(const LargeDesc &d, int tile, int opnd, u32 *buf, ModParams m,
                                          TwTables tw) {
    const int64_t z = opnd ? d.zb : d.za;
    const int64_t S = d.g.S, c0 = (int64_t)tile * C;
    const int T = (int)d.g.T, t = d.g.t;
    int zb = z > c0 ? (int)((z - c0 + S - 1) / S) : 0;
    if (zb > T) zb = T;
    const ColFwdArgs X{buf, nullptr, opnd ? d.wb : d.wa, z, (u32)c0, d.g.sigma, T, t, zb,
                       d.prune ? (int)d.g.k : T, d.prune != 0, tw.fwd, m.p, tw.status};
    if (t == 0) {
        for (int c = threadIdx.x; c < C; c += blockDim.x) X.W[c0 + c] = buf[col_elem_addr<C, LAY_TILE>(0, c)];
        __syncthreads();
        return;
    }
    const int np = col_npass(t);
    int s0 = 0;
    for (int i = 0; i < np; ++i) {
        const int R = col_pass_R(t, np, i);
        if (i == np - 1) colf_pass_r<A, C, LAY_TILE, IO_SMEM, IO_GLOBAL>(R, X, s0);
        else colf_pass_r<A, C, LAY_TILE, IO_SMEM, IO_SMEM>(R, X, s0);
        __syncthreads();
        s0 += R;
    }
}

// Compile-time-shaped column stage of a loaded tile (TL = t levels).
template <class A, int C, int TL>
__device__ __forceinline__ void colf_compute_ct(const LargeDesc &d, int tile, int opnd, u32 *buf, ModParams m,
                                             TwTables tw) {
    const int64_t z = opnd ? d.zb : d.za;
    const int64_t S = d.g.S, c0 = (int64_t)tile * C;
    const int T = 1 << TL;
    int zb = z > c0 ? (int)((z - c0 + S - 1) / S) : 0;
    if (zb > T) zb = T;
    const ColFwdArgs X{buf, nullptr, opnd ? d.wb : d.wa, z, (u32)c0, d.g.sigma, T, TL, zb,
                       d.prune ? (int)d.g.k : T, d.prune != 0, tw.fwd, m.p, tw.status};
    colf_tile_ct<A, C, TL>(X);
}

// One column-stage item with a single buffer (the persistent batched kernel).
template <class A, int C>
__device__ __noinline__ void colf_body(const LargeDesc d, int tile, int opnd, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    colf_load<C>(d, tile, opnd, smem);
    cp_async_wait_all();
    __syncthreads();
    colf_compute<A, C>(d, tile, opnd, smem, m, tw);
}

// Row ib: remaining sigma levels of both operands, pointwise product,
// unscaled inverse; result overwrites wa's row.  blockDim must be S/E (E
// words per thread: 16 in 4-level passes, or 8 / 4 in 3- / 2-level passes for
// products with few rows, which then spread each row over more threads).
// Shared memory (row_smem_bytes): one exchange buffer of S words, the row's
// S-1 forward twiddles (8 bytes each) and, for sigma <= 12, the inverse
// twiddles of the sub-levels before the last pass (2^UL entries).  Pass 0
// reads both rows from global memory while the twiddles arrive by cp.async;
// the last pass's inverse twiddles are fetched during the forward passes
// (srow2_fwd_1b, EARLY), so the inverse starts without a staging wait.  For
// sigma = 13 (whose shared inverse levels would take 32 KB) the inverse
// table is staged over the forward one after the pointwise product.
template <class A, int SIGMA, int E = 16>
__device__ __forceinline__ void row_body(const LargeDesc &d, u32 ib, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    constexpr int S = 1 << SIGMA;
    constexpr int NP = RowPlan<SIGMA, 0, E>::NP;
    constexpr int UL = row_last_u0<SIGMA, E>();
    constexpr bool EARLY = SIGMA <= 12;
    u32 *buf = smem;
    uint2 *twb = reinterpret_cast<uint2 *>(smem + S);
    uint2 *twlo = twb + S;  // EARLY: inverse sub-levels < UL
    const u32 tid = threadIdx.x;
    const u32 p = m.p;
    const int t = d.g.t;
    u32 *rowa = d.wa + (int64_t)ib * S;
    stage_tw<SIGMA>(twb, tw.fwd, t, ib);
    if constexpr (EARLY) stage_tw<UL>(twlo, tw.inv, t, ib);
    cp_async_commit();
    pdl_wait();  // the rows come from the column-stage kernel
    u32 xa[E], xb[E];
    srow2_load_g<SIGMA, E>(xa, xb, rowa, d.wb + (int64_t)ib * S, tid);
    cp_async_wait<0>();
    __syncthreads();
    srow2_fwd_1b<A, SIGMA, 0, EARLY, E>(xa, xb, buf, twb, tid, p, tw.inv, t, ib);
    // The pointwise constant, loaded here rather than before the passes: held
    // through them it costs the 4096-word row two registers and a spill.
    const uint2 cs = row_scale(tw, SIGMA, ib, (u32)d.g.k);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        PM_DCHECK(xa[i] < 2 * A::bound(p) && xb[i] < 2 * A::bound(p) && ib < (u32)d.g.k, tw.status);
        xa[i] = A::pointwise(xa[i], xb[i], cs, m);
        PM_DCHECK(xa[i] < A::bound(p), tw.status);
    }
    RowTw rt;
    if constexpr (EARLY) {
        cp_async_wait_all();  // this thread's own last-pass inverse twiddles
        rt = RowTw{twlo, twb, reinterpret_cast<const uint2 *>(buf)};
    } else {
        __syncthreads();  // every thread is done with the forward twiddles and buf
        stage_tw<SIGMA>(twb, tw.inv, t, ib);
        cp_async_wait_all();
        __syncthreads();
        rt = RowTw{twb, twb, twb + (S >> 1)};
    }
    srow2_inv<A, SIGMA, NP - 1, E>(xa, buf, rowa, rt, tid, p);
    __syncthreads();
}

template <class A, int SIGMA>
__device__ __noinline__ void row_body_ool(const LargeDesc d, u32 ib, ModParams m, TwTables tw) {
    row_body<A, SIGMA>(d, ib, m, tw);
}

// Issues the cp.async copies of the k needed workspace rows of tile `tile`.
template <int C>
__device__ __forceinline__ void coli_load(const LargeDesc &d, int tile, u32 *buf) {
    const u32 c0 = (u32)tile * C;
    constexpr int logCH = ilog2c(C) - 2;
    const int nch = (int)d.g.k << logCH;
    const int logS = d.g.sigma;
    for (int i = threadIdx.x; i < nch; i += blockDim.x) {
        const u32 r = (u32)i >> logCH, c = ((u32)i & ((1u << logCH) - 1u)) << 2;
        cp_async16(buf + col_elem_addr<C, LAY_TILE>(r, c), d.wa + ((int64_t)r << logS) + c0 + c);
    }
}

// Stores rows [0, k) of a column tile (reduced to [0, p)) to the product,
// entries below n only.  Ends with a barrier.
template <class A, int C>
__device__ __forceinline__ void coli_store(const LargeDesc &d, u32 c0, const u32 *buf, u32 p) {
    const int k = (int)d.g.k;
    const int64_t S = d.g.S;
    for (int tau = threadIdx.x; tau < k * C; tau += blockDim.x) {
        const u32 r = (u32)tau / C, c = (u32)tau % C;
        const int64_t e = (int64_t)r * S + c0 + c;
        if (e < d.n) d.c[e] = A::to_canon(buf[col_elem_addr<C, LAY_TILE>(r, c)], p);
    }
    __syncthreads();
}

// ITFT column stage of a tile already in buf, and the store of its part of
// the first n outputs (reduced to [0, p)).  Ends with a barrier.
template <class A, int C>
__device__ __forceinline__ void coli_compute(const LargeDesc &d, int tile, u32 *buf, ModParams m, TwTables tw) {
    const u32 c0 = (u32)tile * C;
    const int T = (int)d.g.T, k = (int)d.g.k;
    const ColInvArgs X{buf, d.wa, d.c, d.n, c0, d.g.sigma, k, tw.inv, m.p, tw.fwd, nullptr, tw.status};
    if (d.g.t == 0) {
        for (int c = threadIdx.x; c < C; c += blockDim.x)
            if ((int64_t)(c0 + c) < d.n) d.c[c0 + c] = A::to_canon(buf[col_elem_addr<C, LAY_TILE>(0, c)], m.p);
        __syncthreads();
        return;
    }
    if (k == T) {  // no truncation: one unscaled full inverse, last pass to the output
        coli_full<A, C, LAY_TILE>(X, 0, 0u, 0, d.g.t, false, true);
        return;
    }
    coli_steps<A, C, LAY_TILE>(X, d.steps, d.nsteps);
    coli_store<A, C>(d, c0, buf, m.p);
}

// Column inverse of a loaded tile with compile-time pass shapes: the full
// inverse when k = T, the truncated one otherwise (k a multiple of T/8).
template <class A, int C, int TL>
__device__ __forceinline__ void coli_compute_ct(const LargeDesc &d, int tile, u32 *buf, ModParams m, TwTables tw,
                                             const uint2 *top) {
    const ColInvArgs X{buf,   d.wa,   d.c, d.n, (u32)tile * C, d.g.sigma, (int)d.g.k, tw.inv, m.p, tw.fwd, top,
                       tw.status};
    coli_tile_ct<A, C, TL>(X);
}

template <class A, int C>
__device__ __noinline__ void coli_body(const LargeDesc d, int tile, ModParams m, TwTables tw) {
    u32 *smem = dyn_smem();
    coli_load<C>(d, tile, smem);
    cp_async_wait_all();
    __syncthreads();
    coli_compute<A, C>(d, tile, smem, m, tw);
}

}  // namespace pm
