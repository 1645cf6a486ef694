// device.cuh -- CTA-level building blocks of the TFT polynomial product.
//
// Data model (block-relaxed TFT): a length-L transform is a T x S matrix of
// rows (L = T * S).  The merged Cooley-Tukey tree's top t = log2 T levels
// combine whole rows ("column stage"), the bottom sigma = log2 S levels work
// inside one row ("row stage").  Node (s, i) uses the twiddle
// tw[2^s + i] = psi_{s+1}^{rev_s(i)}, so no separate twist is needed between
// the stages (see internal.h).
//
// Row stage: Stockham ordering.  A pass over R levels starting at sub-level
// u0 reads element q of group G from address G + q*(S>>R) and writes its
// outputs to (G<<R) + q, so reads are unit-stride across threads and writes
// are 2^R contiguous words per thread (16-byte vector stores).  Shared-memory
// addresses go through swz(), which XORs the 16-byte-chunk bits [4:2] with
// bits [7:5]: unit-stride warps stay conflict-free and eight threads storing
// 16 contiguous words each hit eight distinct bank groups.
//
// Column stage: tile of C columns x T rows in shared memory, row r column c
// at swz(r*C + c); a warp's lanes cover consecutive columns, so every access
// is unit-stride.  TFT pruning (Section 3): rows of a node beyond the input
// support are zero, which makes whole tree levels plain copies, and nodes
// whose leaves all lie beyond the k needed rows are skipped.
#pragma once
#include "internal.h"

namespace pm {

__device__ __forceinline__ u32 swz(u32 w) { return w ^ (((w >> 5) & 7u) << 2); }

// ----------------------------------------------------------------- groups
// A group holds 2^R elements x[q] of one node at depth lev0 (node index
// node0); level lev0+d splits it into 2^d sub-nodes of 2^(R-d) elements.
template <class A, int R>
__device__ __forceinline__ void grp_fwd(u32 *x, const uint2 *__restrict__ tw, int lev0, u32 node0, u32 p) {
#pragma unroll
    for (int d = 0; d < R; ++d) {
        const int half = 1 << (R - 1 - d);
#pragma unroll
        for (int e = 0; e < (1 << d); ++e) {
            const uint2 w = __ldg(tw + tw_index(lev0 + d, (node0 << d) + e));
#pragma unroll
            for (int jj = 0; jj < half; ++jj) {
                const int lo = e * 2 * half + jj;
                A::ct(x[lo], x[lo + half], w, p);
            }
        }
    }
}

// Same with per-level copy flags: bit d of copymask set means every upper
// input at level lev0+d is zero, so the butterfly is (a, 0) -> (a, a).
template <class A, int R>
__device__ __forceinline__ void grp_fwd_cp(u32 *x, const uint2 *__restrict__ tw, int lev0, u32 node0, u32 p,
                                           u32 copymask) {
#pragma unroll
    for (int d = 0; d < R; ++d) {
        const int half = 1 << (R - 1 - d);
        if ((copymask >> d) & 1u) {
#pragma unroll
            for (int e = 0; e < (1 << d); ++e)
#pragma unroll
                for (int jj = 0; jj < half; ++jj) {
                    const int lo = e * 2 * half + jj;
                    x[lo + half] = x[lo];
                }
        } else {
#pragma unroll
            for (int e = 0; e < (1 << d); ++e) {
                const uint2 w = __ldg(tw + tw_index(lev0 + d, (node0 << d) + e));
#pragma unroll
                for (int jj = 0; jj < half; ++jj) {
                    const int lo = e * 2 * half + jj;
                    A::ct(x[lo], x[lo + half], w, p);
                }
            }
        }
    }
}

template <class A, int R>
__device__ __forceinline__ void grp_inv(u32 *x, const uint2 *__restrict__ itw, int lev0, u32 node0, u32 p) {
#pragma unroll
    for (int d = R - 1; d >= 0; --d) {
        const int half = 1 << (R - 1 - d);
#pragma unroll
        for (int e = 0; e < (1 << d); ++e) {
            const uint2 w = __ldg(itw + tw_index(lev0 + d, (node0 << d) + e));
#pragma unroll
            for (int jj = 0; jj < half; ++jj) {
                const int lo = e * 2 * half + jj;
                A::gs(x[lo], x[lo + half], w, p);
            }
        }
    }
}

// ------------------------------------------------------ row-stage helpers
template <int SIGMA, int P>
struct RowPlan {
    static constexpr int NP = (SIGMA + 3) / 4;  // passes
    static constexpr int R = (P < NP - 1) ? 4 : (SIGMA - 4 * (NP - 1));
    static constexpr int S = 1 << SIGMA;
    static constexpr int NT = S / 16;  // threads per row
    static constexpr int NG = 16 >> R; // groups per thread
    static constexpr int U0 = 4 * P;   // first sub-level of the pass
};

template <int R, int S>
__device__ __forceinline__ void ld_str_s(const u32 *buf, u32 G, u32 *x) {
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) x[q] = buf[swz(G + q * (S >> R))];
}
template <int R, int S>
__device__ __forceinline__ void st_str_s(u32 *buf, u32 G, const u32 *x) {
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) buf[swz(G + q * (S >> R))] = x[q];
}
template <int R, int S>
__device__ __forceinline__ void ld_str_g(const u32 *g, u32 G, u32 *x) {
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) x[q] = __ldcg(g + G + q * (S >> R));
}
template <int R, int S>
__device__ __forceinline__ void st_str_g(u32 *g, u32 G, const u32 *x) {
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) g[G + q * (S >> R)] = x[q];
}
template <int R>
__device__ __forceinline__ void st_con_s(u32 *buf, u32 G, const u32 *x) {
    const u32 b = G << R;
    if constexpr (R >= 2) {
#pragma unroll
        for (int k = 0; k < (1 << R) / 4; ++k)
            *reinterpret_cast<uint4 *>(buf + swz(b + 4 * k)) = make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
    } else if constexpr (R == 1) {
        *reinterpret_cast<uint2 *>(buf + swz(b)) = make_uint2(x[0], x[1]);
    } else {
        buf[swz(b)] = x[0];
    }
}
template <int R>
__device__ __forceinline__ void ld_con_s(const u32 *buf, u32 G, u32 *x) {
    const u32 b = G << R;
    if constexpr (R >= 2) {
#pragma unroll
        for (int k = 0; k < (1 << R) / 4; ++k) {
            const uint4 v = *reinterpret_cast<const uint4 *>(buf + swz(b + 4 * k));
            x[4 * k] = v.x;
            x[4 * k + 1] = v.y;
            x[4 * k + 2] = v.z;
            x[4 * k + 3] = v.w;
        }
    } else if constexpr (R == 1) {
        const uint2 v = *reinterpret_cast<const uint2 *>(buf + swz(b));
        x[0] = v.x;
        x[1] = v.y;
    } else {
        x[0] = buf[swz(b)];
    }
}

// Butterflies of one pass on the thread's groups.  Row ib sits at depth t;
// its sub-node v at sub-level U0 is tree node (ib << U0) + v at depth t+U0.
template <class A, int SIGMA, int P>
__device__ __forceinline__ void row_fwd_compute(u32 *x, u32 tid, int t, u32 ib, const uint2 *__restrict__ tw, u32 p) {
    using RP = RowPlan<SIGMA, P>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 G = tid + g * RP::NT;
        const u32 v = G & ((1u << RP::U0) - 1u);
        grp_fwd<A, RP::R>(x + (g << RP::R), tw, t + RP::U0, (ib << RP::U0) + v, p);
    }
}
template <class A, int SIGMA, int P>
__device__ __forceinline__ void row_inv_compute(u32 *x, u32 tid, int t, u32 ib, const uint2 *__restrict__ itw, u32 p) {
    using RP = RowPlan<SIGMA, P>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 G = tid + g * RP::NT;
        const u32 v = G & ((1u << RP::U0) - 1u);
        grp_inv<A, RP::R>(x + (g << RP::R), itw, t + RP::U0, (ib << RP::U0) + v, p);
    }
}

// Large rows: CTA-wide, ping-pong buffers b0/b1 (one barrier per pass).
// Forward: pass 0 reads the row from global memory; the last pass leaves
// the leaves in registers (thread tid holds leaves (tid + g*NT) << R .. + 2^R).
template <class A, int SIGMA, int P>
__device__ __forceinline__ void lrow_fwd(u32 *x, const u32 *gsrc, u32 *b0, u32 *b1, u32 tid, int t, u32 ib,
                                         const uint2 *__restrict__ tw, u32 p) {
    using RP = RowPlan<SIGMA, P>;
    if constexpr (P == 0) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_str_g<RP::R, RP::S>(gsrc, tid + g * RP::NT, x + (g << RP::R));
    } else {
        const u32 *src = ((P - 1) & 1) ? b1 : b0;
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_str_s<RP::R, RP::S>(src, tid + g * RP::NT, x + (g << RP::R));
    }
    row_fwd_compute<A, SIGMA, P>(x, tid, t, ib, tw, p);
    if constexpr (P < RP::NP - 1) {
        u32 *dst = (P & 1) ? b1 : b0;
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_con_s<RP::R>(dst, tid + g * RP::NT, x + (g << RP::R));
        __syncthreads();
        lrow_fwd<A, SIGMA, P + 1>(x, gsrc, b0, b1, tid, t, ib, tw, p);
    }
}

// Inverse, starting from the leaves in registers (P = NP-1) and ending with
// the row written to global memory in natural order.
template <class A, int SIGMA, int P>
__device__ __forceinline__ void lrow_inv(u32 *x, u32 *gdst, u32 *b0, u32 *b1, u32 tid, int t, u32 ib,
                                         const uint2 *__restrict__ itw, u32 p) {
    using RP = RowPlan<SIGMA, P>;
    if constexpr (P < RP::NP - 1) {
        const u32 *src = ((P + 1) & 1) ? b1 : b0;
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_con_s<RP::R>(src, tid + g * RP::NT, x + (g << RP::R));
    }
    row_inv_compute<A, SIGMA, P>(x, tid, t, ib, itw, p);
    if constexpr (P == 0) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_str_g<RP::R, RP::S>(gdst, tid + g * RP::NT, x + (g << RP::R));
    } else {
        u32 *dst = (P & 1) ? b1 : b0;
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_str_s<RP::R, RP::S>(dst, tid + g * RP::NT, x + (g << RP::R));
        __syncthreads();
        lrow_inv<A, SIGMA, P - 1>(x, gdst, b0, b1, tid, t, ib, itw, p);
    }
}

// Small rows: one warp per row, in place in one buffer (two warp barriers
// per pass).  The row starts and ends in natural order in `buf`.
template <class A, int SIGMA, int P>
__device__ __forceinline__ void srow_fwd(u32 *x, u32 *buf, u32 tid, int t, u32 ib, const uint2 *__restrict__ tw,
                                         u32 p) {
    using RP = RowPlan<SIGMA, P>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) ld_str_s<RP::R, RP::S>(buf, tid + g * RP::NT, x + (g << RP::R));
    row_fwd_compute<A, SIGMA, P>(x, tid, t, ib, tw, p);
    if constexpr (P < RP::NP - 1) {
        __syncwarp();
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_con_s<RP::R>(buf, tid + g * RP::NT, x + (g << RP::R));
        __syncwarp();
        srow_fwd<A, SIGMA, P + 1>(x, buf, tid, t, ib, tw, p);
    }
}
template <class A, int SIGMA, int P>
__device__ __forceinline__ void srow_inv(u32 *x, u32 *buf, u32 tid, int t, u32 ib, const uint2 *__restrict__ itw,
                                         u32 p) {
    using RP = RowPlan<SIGMA, P>;
    if constexpr (P < RP::NP - 1) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_con_s<RP::R>(buf, tid + g * RP::NT, x + (g << RP::R));
    }
    row_inv_compute<A, SIGMA, P>(x, tid, t, ib, itw, p);
    __syncwarp();
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) st_str_s<RP::R, RP::S>(buf, tid + g * RP::NT, x + (g << RP::R));
    __syncwarp();
    if constexpr (P > 0) srow_inv<A, SIGMA, P - 1>(x, buf, tid, t, ib, itw, p);
}

// ------------------------------------------------------ column-stage helpers
// One pass of R tree levels starting at depth s0 over a tile of C columns.
// Rows of node v: v*M .. v*M+M-1 (M = T >> s0); group (v, j) holds rows
// v*M + j + q*J, J = M >> R.  With `from_global`, rows come straight from
// the operand g (row r, column c0+c is element r*S + c0 + c; zero past z).
template <class A, int R, int C>
__device__ __forceinline__ void col_fwd_pass(u32 *sm, const u32 *__restrict__ g, int64_t z, int64_t S, int64_t c0,
                                             int s0, int T, int zb, int k, bool prune, bool from_global,
                                             const uint2 *__restrict__ tw, u32 p) {
    const int M = T >> s0, J = M >> R;
    const int tasks = (T >> R) * C;
    u32 copymask = 0;
    if (prune) {
#pragma unroll
        for (int d = 0; d < R; ++d)
            if (zb <= ((M >> d) >> 1)) copymask |= 1u << d;
    }
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const int G = tau / C, c = tau % C;
        const int v = G / J, j = G % J;
        if (prune && v * M >= k) continue;
        const int r0 = v * M + j;
        u32 x[1 << R];
        if (from_global) {
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) {
                const int64_t e = (int64_t)(r0 + q * J) * S + c0 + c;
                x[q] = (e < z) ? g[e] : 0u;
            }
        } else {
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) x[q] = sm[swz((r0 + q * J) * C + c)];
        }
        grp_fwd_cp<A, R>(x, tw, s0, (u32)v, p, copymask);
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) sm[swz((r0 + q * J) * C + c)] = x[q];
    }
}

// Forward column stage of one tile: t levels (T = 2^t rows); leaves the
// tile (rows < k valid) in shared memory.  zb = rows with any nonzero input.
template <class A, int C>
__device__ void col_fwd_tile(u32 *sm, const u32 *__restrict__ g, int64_t z, int64_t S, int64_t c0, int T, int t,
                             int zb, int k, bool prune, const uint2 *__restrict__ tw, u32 p) {
    if (t == 0) {
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            const int64_t e = c0 + c;
            sm[swz(c)] = (e < z) ? g[e] : 0u;
        }
        __syncthreads();
        return;
    }
    for (int s0 = 0; s0 < t; s0 += 4) {
        const int R = min(4, t - s0);
        const bool fg = (s0 == 0);
        switch (R) {
            case 4: col_fwd_pass<A, 4, C>(sm, g, z, S, c0, s0, T, zb, k, prune, fg, tw, p); break;
            case 3: col_fwd_pass<A, 3, C>(sm, g, z, S, c0, s0, T, zb, k, prune, fg, tw, p); break;
            case 2: col_fwd_pass<A, 2, C>(sm, g, z, S, c0, s0, T, zb, k, prune, fg, tw, p); break;
            default: col_fwd_pass<A, 1, C>(sm, g, z, S, c0, s0, T, zb, k, prune, fg, tw, p); break;
        }
        __syncthreads();
    }
}

// Inverse pass of R levels [lev0, lev0+R) inside the subtree rooted at
// (s_root, i_root) that covers rows [base, base + M_root).
template <class A, int R, int C>
__device__ __forceinline__ void col_inv_pass(u32 *sm, int lev0, int s_root, u32 i_root, int base, int Msub,
                                             int nnodes, const uint2 *__restrict__ itw, u32 p) {
    const int J = Msub >> R;
    const int tasks = nnodes * J * C;
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const int G = tau / C, c = tau % C;
        const int v = G / J, j = G % J;
        const int r0 = base + v * Msub + j;
        u32 x[1 << R];
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) x[q] = sm[swz((r0 + q * J) * C + c)];
        grp_inv<A, R>(x, itw, lev0, (i_root << (lev0 - s_root)) + (u32)v, p);
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) sm[swz((r0 + q * J) * C + c)] = x[q];
    }
}

// Unscaled inverse of the whole subtree (s, i) on rows [base, base+M):
// returns M times the node's coefficients.  Ends with a barrier.
template <class A, int C>
__device__ void col_full_inv(u32 *sm, int s, u32 i, int base, int M, const uint2 *__restrict__ itw, u32 p) {
    const int lm = 31 - __clz(M);
    const int nch = (lm + 3) / 4;
    for (int ch = nch - 1; ch >= 0; --ch) {
        const int u0 = s + 4 * ch;
        const int R = min(4, lm - 4 * ch);
        const int Msub = M >> (4 * ch), nn = 1 << (4 * ch);
        switch (R) {
            case 4: col_inv_pass<A, 4, C>(sm, u0, s, i, base, Msub, nn, itw, p); break;
            case 3: col_inv_pass<A, 3, C>(sm, u0, s, i, base, Msub, nn, itw, p); break;
            case 2: col_inv_pass<A, 2, C>(sm, u0, s, i, base, Msub, nn, itw, p); break;
            default: col_inv_pass<A, 1, C>(sm, u0, s, i, base, Msub, nn, itw, p); break;
        }
        __syncthreads();
    }
}

// The truncated inverse (ITFT) of a tile from its step list.  On entry rows
// [0, k) hold spectral values (all at one common scale) and rows [k, T) are
// zero; on exit rows [0, k) hold the coefficients at that scale (or, when the
// list is a single top-level ST_FULL, T times it).  Values in [0, B).
template <class A, int C>
__device__ void col_itft_steps(u32 *sm, const ItftStep *__restrict__ steps, int nsteps,
                               const uint2 *__restrict__ itw, u32 p) {
    for (int si = 0; si < nsteps; ++si) {
        const ItftStep st = steps[si];
        if (st.kind == ST_FULL) {
            col_full_inv<A, C>(sm, st.s, st.i, st.base, st.h, itw, p);
            continue;
        }
        const bool upper = (st.kind == ST_PRE_RIGHT || st.kind == ST_PRE_LEFT);
        const int lo = upper ? st.m : 0, hi = upper ? st.h : st.m;
        const int tasks = (hi - lo) * C;
        for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
            const int j = lo + tau / C, c = tau % C;
            u32 *X0 = sm + swz((st.base + j) * C + c);
            u32 *X1 = sm + swz((st.base + j + st.h) * C + c);
            const u32 x0 = A::to_canon(*X0, p), x1 = A::to_canon(*X1, p);
            switch (st.kind) {
                case ST_PRE_RIGHT: {
                    const u32 lo_ = mul_c(x0, st.hinv, p);
                    if (st.zero) {
                        *X0 = lo_;
                        *X1 = lo_;
                    } else {
                        const u32 rc = mul_c(x1, st.r, p);
                        const u32 cj = sub_c(lo_, rc, p);
                        *X0 = cj;
                        *X1 = sub_c(cj, rc, p);
                    }
                    break;
                }
                case ST_POST_RIGHT: {
                    const u32 u = mul_c(x0, st.hinv, p);
                    *X0 = mul_c(u + x1, st.inv2, p);
                    *X1 = mul_c(u - x1 + p, st.i2r, p);
                    break;
                }
                case ST_PRE_LEFT: *X0 = add_c(x0, mul_c(x1, st.r, p), p); break;
                default: *X0 = sub_c(x0, mul_c(x1, st.r, p), p); break;
            }
        }
        __syncthreads();
    }
}

}  // namespace pm
