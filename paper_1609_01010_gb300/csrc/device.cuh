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
#include <type_traits>

#include "internal.h"

namespace pm {

// Debug builds (compiled with PM_DEBUG_CHECKS=1): range and index checks in
// the kernels.  A failed check records POLY_EDEBUG_CHECK (-11) in the
// device status word (polymul_device_status) and the kernel goes on; nothing
// traps.  In ordinary builds the checks compile to nothing.
#if defined(PM_DEBUG_CHECKS) && PM_DEBUG_CHECKS
#define PM_DCHECK(cond, status)                                    \
    do {                                                           \
        if (!(cond) && (status)) atomicCAS((status), 0, -11);      \
    } while (0)
#else
#define PM_DCHECK(cond, status) \
    do {                        \
    } while (0)
#endif

__device__ __forceinline__ u32 swz(u32 w) { return w ^ (((w >> 5) & 7u) << 2); }

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

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
template <class A, int R, bool TS = false>
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
                const uint2 *q = tw + tw_index(lev0 + d, (node0 << d) + e);
                const uint2 w = TS ? *q : __ldg(q);
#pragma unroll
                for (int jj = 0; jj < half; ++jj) {
                    const int lo = e * 2 * half + jj;
                    A::ct(x[lo], x[lo + half], w, p);
                }
            }
        }
    }
}

// Programmatic dependent launch (sm_90+): a kernel launched with
// programmatic stream serialization may start while the previous kernel on
// the stream still runs; pdl_wait() blocks until that kernel has completed
// and its writes are visible.  The previous kernel lets it launch early with
// pdl_launch_dependents().  Both are no-ops for kernels launched without the
// attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A twiddle pair from shared memory (the compile-time-shaped column kernels
// stage the column tree's twiddles there once per CTA).
__device__ __forceinline__ uint2 lds_tw(const uint2 *p) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                 : "=r"(v.x), "=r"(v.y)
                 : "r"((u32)__cvta_generic_to_shared(p)));
    return v;
}

// Two columns at once (x, y), sharing the twiddle loads; tw is the shared
// memory copy of the table (lds_tw).  ROOT: node0 is 0 (a group of the root's
// pass), so each level's first node has twiddle 1 and needs no multiply.
template <class A, int R, bool ROOT = false>
__device__ __forceinline__ void grp_fwd_cp2(u32 *x, u32 *y, const uint2 *tw, int lev0, u32 node0, u32 p,
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
                    y[lo + half] = y[lo];
                }
        } else {
#pragma unroll
            for (int e = 0; e < (1 << d); ++e) {
                if (ROOT && e == 0) {
#pragma unroll
                    for (int jj = 0; jj < half; ++jj) {
                        A::ct_one(x[jj], x[jj + half], p);
                        A::ct_one(y[jj], y[jj + half], p);
                    }
                    continue;
                }
                const uint2 w = lds_tw(tw + tw_index(lev0 + d, (node0 << d) + e));
#pragma unroll
                for (int jj = 0; jj < half; ++jj) {
                    const int lo = e * 2 * half + jj;
                    A::ct(x[lo], x[lo + half], w, p);
                    A::ct(y[lo], y[lo + half], w, p);
                }
            }
        }
    }
}

// Node E at relative depth D of an R-level inverse group, then the nodes
// after it; template recursion keeps every array index a constant.  itw is
// the shared memory copy of the inverse table (lds_tw).
template <class A, int R, int D, int E>
__device__ __forceinline__ void grp_inv2_nodes(u32 *x, u32 *y, const uint2 *itw, int lev0, u32 node0, u32 p) {
    if constexpr (E < (1 << D)) {
        constexpr int half = 1 << (R - 1 - D);
        const uint2 w = lds_tw(itw + tw_index(lev0 + D, (node0 << D) + E));
#pragma unroll
        for (int jj = 0; jj < half; ++jj) {
            A::gs(x[E * 2 * half + jj], x[E * 2 * half + jj + half], w, p);
            A::gs(y[E * 2 * half + jj], y[E * 2 * half + jj + half], w, p);
        }
        grp_inv2_nodes<A, R, D, E + 1>(x, y, itw, lev0, node0, p);
    }
}

template <class A, int R, int D = R - 1>
__device__ __forceinline__ void grp_inv2(u32 *x, u32 *y, const uint2 *itw, int lev0, u32 node0, u32 p) {
    if constexpr (D >= 0) {
        grp_inv2_nodes<A, R, D, 0>(x, y, itw, lev0, node0, p);
        grp_inv2<A, R, D - 1>(x, y, itw, lev0, node0, p);
    }
}

template <class A, int R, bool TS = false>
__device__ __forceinline__ void grp_inv(u32 *x, const uint2 *__restrict__ itw, int lev0, u32 node0, u32 p) {
#pragma unroll
    for (int d = R - 1; d >= 0; --d) {
        const int half = 1 << (R - 1 - d);
#pragma unroll
        for (int e = 0; e < (1 << d); ++e) {
            const uint2 *q = itw + tw_index(lev0 + d, (node0 << d) + e);
            const uint2 w = TS ? *q : __ldg(q);
#pragma unroll
            for (int jj = 0; jj < half; ++jj) {
                const int lo = e * 2 * half + jj;
                A::gs(x[lo], x[lo + half], w, p);
            }
        }
    }
}

// ------------------------------------------------------ row-stage helpers
// Pass P of a row of 2^SIGMA words held E words per thread (E = 16: one
// warp per 512-word row, 4-level passes; E = 4 or 8: 2- or 3-level passes on
// S/E threads of a CTA).
template <int SIGMA, int P, int E = 16>
struct RowPlan {
    static constexpr int LE = ilog2c(E);             // levels of a full pass
    static constexpr int NP = (SIGMA + LE - 1) / LE;  // passes
    static constexpr int R = (P < NP - 1) ? LE : (SIGMA - LE * (NP - 1));
    static constexpr int S = 1 << SIGMA;
    static constexpr int NT = S / E;   // threads per row
    static constexpr int NG = E >> R;  // groups per thread
    static constexpr int U0 = LE * P;  // first sub-level of the pass
};

// G + q*(S>>R) with S>>R a multiple of 256 never carries into bits [7:5],
// so swz(G + q*(S>>R)) = swz(G) + q*(S>>R): one swizzle per group.
template <int R, int S>
__device__ __forceinline__ void ld_str_s(const u32 *buf, u32 G, u32 *x) {
    if constexpr ((S >> R) % 256 == 0) {
        const u32 *b = buf + swz(G);
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) x[q] = b[q * (S >> R)];
    } else {
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) x[q] = buf[swz(G + q * (S >> R))];
    }
}
template <int R, int S>
__device__ __forceinline__ void st_str_s(u32 *buf, u32 G, const u32 *x) {
    if constexpr ((S >> R) % 256 == 0) {
        u32 *b = buf + swz(G);
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) b[q * (S >> R)] = x[q];
    } else {
#pragma unroll
        for (int q = 0; q < (1 << R); ++q) buf[swz(G + q * (S >> R))] = x[q];
    }
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
template <class A, int SIGMA, int P, int E = 16>
__device__ __forceinline__ void row_fwd_compute(u32 *x, u32 tid, int t, u32 ib, const uint2 *__restrict__ tw, u32 p) {
    using RP = RowPlan<SIGMA, P, E>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 G = tid + g * RP::NT;
        const u32 v = G & ((1u << RP::U0) - 1u);
        grp_fwd<A, RP::R>(x + (g << RP::R), tw, t + RP::U0, (ib << RP::U0) + v, p);
    }
}
template <class A, int SIGMA, int P, int E = 16>
__device__ __forceinline__ void row_inv_compute(u32 *x, u32 tid, int t, u32 ib, const uint2 *__restrict__ itw, u32 p) {
    using RP = RowPlan<SIGMA, P, E>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 G = tid + g * RP::NT;
        const u32 v = G & ((1u << RP::U0) - 1u);
        grp_inv<A, RP::R>(x + (g << RP::R), itw, t + RP::U0, (ib << RP::U0) + v, p);
    }
}

// ------------------------------------------------------ staged large rows
// Row stage with everything staged in shared memory by cp.async: both rows
// (natural order, swz layout) and the row's twiddles.  The 2^u twiddles of
// sub-level u sit at entries [2^u, 2^(u+1)) in node order (entry 0 unused),
// so a group's 2^d twiddles of one level are contiguous and are read with
// 16-byte loads (optimal shared-memory wavefronts for the bytes moved).
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    const u32 sa = (u32)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc) {
    const u32 sa = (u32)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
    const u32 sa = (u32)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    cp_async_commit();
    cp_async_wait<0>();
}

// Copies a row of S words (global, natural order) into buf (swz layout).
template <int S>
__device__ __forceinline__ void stage_row(u32 *buf, const u32 *g) {
    for (u32 ch = threadIdx.x; ch < S / 4; ch += blockDim.x) cp_async16(buf + swz(4 * ch), g + 4 * ch);
}

// Copies the twiddles of sub-levels u < LEVELS of row ib's subtree (depth t)
// from the global table into twb (entries [2^u, 2^(u+1)) for sub-level u);
// LEVELS = sigma gives all S-1 of them.
template <int LEVELS>
__device__ __forceinline__ void stage_tw(uint2 *twb, const uint2 *__restrict__ tab, int t, u32 ib) {
    constexpr u32 S = 1u << LEVELS;
    if (threadIdx.x == 0) cp_async8(twb + 1, tab + tw_index(t, ib));  // level 0: one entry
    // levels u >= 1: chunk x (two entries) belongs to level u with x + 1 in [2^(u-1), 2^u)
    for (u32 x = threadIdx.x; x < S / 2 - 1; x += blockDim.x) {
        const int u = 32 - __clz(x + 1);
        const u32 q = x + 1 - (1u << (u - 1));
        cp_async16(twb + (1u << u) + 2 * q, tab + tw_index(t + u, (ib << u) + 2 * q));
    }
}

// The 2^D twiddles of nodes (v << D) .. (v << D) + 2^D - 1 of one level.
template <int D>
__device__ __forceinline__ void ld_tw_level(uint2 *w, const uint2 *lvl, u32 v) {
    if constexpr (D == 0) {
        w[0] = lvl[v];
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(lvl + (v << D));
#pragma unroll
        for (int e = 0; e < (1 << (D - 1)); ++e) {
            const uint4 t = q[e];
            w[2 * e] = make_uint2(t.x, t.y);
            w[2 * e + 1] = make_uint2(t.z, t.w);
        }
    }
}

template <class A, int R, int U0, int D>
__device__ __forceinline__ void grp_fwd_s_lvl(u32 *x, const uint2 *twb, u32 v, u32 p) {
    if constexpr (D < R) {
        constexpr int half = 1 << (R - 1 - D);
        uint2 w[1 << D];
        ld_tw_level<D>(w, twb + (1u << (U0 + D)), v);
#pragma unroll
        for (int e = 0; e < (1 << D); ++e)
#pragma unroll
            for (int jj = 0; jj < half; ++jj) A::ct(x[e * 2 * half + jj], x[e * 2 * half + jj + half], w[e], p);
        grp_fwd_s_lvl<A, R, U0, D + 1>(x, twb, v, p);
    }
}
// Both operands of a row with one twiddle load per node.
template <class A, int R, int U0, int D>
__device__ __forceinline__ void grp_fwd_s2_lvl(u32 *x, u32 *y, const uint2 *twb, u32 v, u32 p) {
    if constexpr (D < R) {
        constexpr int half = 1 << (R - 1 - D);
        uint2 w[1 << D];
        ld_tw_level<D>(w, twb + (1u << (U0 + D)), v);
#pragma unroll
        for (int e = 0; e < (1 << D); ++e)
#pragma unroll
            for (int jj = 0; jj < half; ++jj) {
                A::ct(x[e * 2 * half + jj], x[e * 2 * half + jj + half], w[e], p);
                A::ct(y[e * 2 * half + jj], y[e * 2 * half + jj + half], w[e], p);
            }
        grp_fwd_s2_lvl<A, R, U0, D + 1>(x, y, twb, v, p);
    }
}
template <class A, int R, int U0, int D>
__device__ __forceinline__ void grp_inv_s_lvl(u32 *x, const uint2 *twb, u32 v, u32 p) {
    if constexpr (D >= 0) {
        constexpr int half = 1 << (R - 1 - D);
        uint2 w[1 << D];
        ld_tw_level<D>(w, twb + (1u << (U0 + D)), v);
#pragma unroll
        for (int e = 0; e < (1 << D); ++e)
#pragma unroll
            for (int jj = 0; jj < half; ++jj) A::gs(x[e * 2 * half + jj], x[e * 2 * half + jj + half], w[e], p);
        grp_inv_s_lvl<A, R, U0, D - 1>(x, twb, v, p);
    }
}
// Where the row stage's inverse twiddles live.  Sub-level u's entry 2^u + j
// is lo[2^u + j] for u < UL (the levels every thread reads), mid[2^u + j]
// for UL <= u < sigma - 1, and top[j] for u = sigma - 1, where UL is the
// first sub-level of the last pass.  The last pass's entries are private to
// one thread each (see row_body).
struct RowTw {
    const uint2 *lo, *mid, *top;
};
template <int SIGMA, int E = 16>
__host__ __device__ constexpr int row_last_u0() {
    return RowPlan<SIGMA, 0, E>::LE * (RowPlan<SIGMA, 0, E>::NP - 1);
}
template <int SIGMA, int LEV, int E = 16>
__device__ __forceinline__ const uint2 *rt_level(const RowTw &t) {
    if constexpr (LEV == SIGMA - 1) return t.top;
    else if constexpr (LEV >= row_last_u0<SIGMA, E>()) return t.mid + (1u << LEV);
    else return t.lo + (1u << LEV);
}
template <class A, int SIGMA, int R, int U0, int D, int E = 16>
__device__ __forceinline__ void grp_inv_rt_lvl(u32 *x, const RowTw &rt, u32 v, u32 p) {
    if constexpr (D >= 0) {
        constexpr int half = 1 << (R - 1 - D);
        uint2 w[1 << D];
        ld_tw_level<D>(w, rt_level<SIGMA, U0 + D, E>(rt), v);
#pragma unroll
        for (int e = 0; e < (1 << D); ++e)
#pragma unroll
            for (int jj = 0; jj < half; ++jj) A::gs(x[e * 2 * half + jj], x[e * 2 * half + jj + half], w[e], p);
        grp_inv_rt_lvl<A, SIGMA, R, U0, D - 1, E>(x, rt, v, p);
    }
}

// Copies of one thread's inverse twiddles for the last pass (groups
// v = tid + g*NT): sub-level sigma-1 into top (entry 2^(sigma-1) + j at top[j]),
// the pass's other levels (MID) into twb at their usual entries.
template <int SIGMA, bool MID, int E = 16>
__device__ __forceinline__ void row_last_inv_tw(uint2 *dst, const uint2 *__restrict__ itab, int t, u32 ib, u32 tid) {
    using RP = RowPlan<SIGMA, RowPlan<SIGMA, 0, E>::NP - 1, E>;
    constexpr int U0 = RP::U0, R = RP::R;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 v = tid + g * RP::NT;
        if constexpr (!MID) {
            constexpr int D = R - 1;
            const uint2 *src = itab + tw_index(t + U0 + D, (ib << (U0 + D)) + (v << D));
            if constexpr (D == 0) {
                cp_async8(dst + v, src);
            } else {
#pragma unroll
                for (int e = 0; e < (1 << D); e += 2) cp_async16(dst + (v << D) + e, src + e);
            }
        } else {
#pragma unroll
            for (int D = 0; D < R - 1; ++D) {
                const uint2 *src = itab + tw_index(t + U0 + D, (ib << (U0 + D)) + (v << D));
                uint2 *d2 = dst + (1u << (U0 + D)) + (v << D);
                if (D == 0) {
                    cp_async8(d2, src);
                } else {
#pragma unroll
                    for (int e = 0; e < (1 << D); e += 2) cp_async16(d2 + e, src + e);
                }
            }
        }
    }
}

template <class A, int R, int U0>
__device__ __forceinline__ void grp_fwd_s(u32 *x, const uint2 *twb, u32 v, u32 p) {
    grp_fwd_s_lvl<A, R, U0, 0>(x, twb, v, p);
}
template <class A, int R, int U0>
__device__ __forceinline__ void grp_inv_s(u32 *x, const uint2 *twb, u32 v, u32 p) {
    grp_inv_s_lvl<A, R, U0, R - 1>(x, twb, v, p);
}

// Forward passes of both operands, in place (two barriers per pass); the
// last pass leaves the leaves in registers.
template <class A, int SIGMA, int P>
__device__ __forceinline__ void srow2_fwd(u32 *xa, u32 *xb, u32 *ba, u32 *bb, const uint2 *twb, u32 tid, u32 p) {
    using RP = RowPlan<SIGMA, P>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        ld_str_s<RP::R, RP::S>(ba, tid + g * RP::NT, xa + (g << RP::R));
        ld_str_s<RP::R, RP::S>(bb, tid + g * RP::NT, xb + (g << RP::R));
    }
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 v = (tid + g * RP::NT) & ((1u << RP::U0) - 1u);
        grp_fwd_s2_lvl<A, RP::R, RP::U0, 0>(xa + (g << RP::R), xb + (g << RP::R), twb, v, p);
    }
    if constexpr (P < RP::NP - 1) {
        __syncthreads();
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) {
            st_con_s<RP::R>(ba, tid + g * RP::NT, xa + (g << RP::R));
            st_con_s<RP::R>(bb, tid + g * RP::NT, xb + (g << RP::R));
        }
        __syncthreads();
        srow2_fwd<A, SIGMA, P + 1>(xa, xb, ba, bb, twb, tid, p);
    }
}

// One operand's hand-over from forward pass P to pass P+1 through buf.
template <int SIGMA, int P, int E = 16>
__device__ __forceinline__ void row_xchg(u32 *x, u32 *buf, u32 tid) {
    using RP = RowPlan<SIGMA, P, E>;
    using RN = RowPlan<SIGMA, P + 1, E>;
    __syncthreads();
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) st_con_s<RP::R>(buf, tid + g * RP::NT, x + (g << RP::R));
    __syncthreads();
#pragma unroll
    for (int g = 0; g < RN::NG; ++g) ld_str_s<RN::R, RN::S>(buf, tid + g * RN::NT, x + (g << RN::R));
}

// Forward passes of both operands through ONE exchange buffer: pass 0 starts
// from the strided elements srow2_load_g read from global memory; between
// passes operand a, then operand b, goes through `buf` (four barriers per
// pass boundary instead of two, for half the shared memory).  The last pass
// leaves the leaves in registers.
template <int SIGMA, int E = 16>
__device__ __forceinline__ void srow2_load_g(u32 *xa, u32 *xb, const u32 *ga, const u32 *gb, u32 tid) {
    using RP = RowPlan<SIGMA, 0, E>;
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        ld_str_g<RP::R, RP::S>(ga, tid + g * RP::NT, xa + (g << RP::R));
        ld_str_g<RP::R, RP::S>(gb, tid + g * RP::NT, xb + (g << RP::R));
    }
}

//
// EARLY: the inverse twiddles of the last pass are fetched while the forward
// runs.  Its groups' twiddles are private to their thread, so before the
// last forward pass (once every thread has read `buf`) each thread starts
// the copy of its sub-level sigma-1 inverse twiddles into `buf` (exactly S
// words), and right after the pass (its forward twiddles consumed) the copy
// of its other inverse twiddles of that pass over the forward ones in twb.
template <class A, int SIGMA, int P, bool EARLY, int E = 16>
__device__ __forceinline__ void srow2_fwd_1b(u32 *xa, u32 *xb, u32 *buf, uint2 *twb, u32 tid, u32 p,
                                             const uint2 *__restrict__ itab, int t, u32 ib) {
    using RP = RowPlan<SIGMA, P, E>;
    if constexpr (EARLY && P == RP::NP - 1) {
        __syncthreads();  // every thread has loaded its elements from buf
        row_last_inv_tw<SIGMA, false, E>(reinterpret_cast<uint2 *>(buf), itab, t, ib, tid);
        cp_async_commit();
    }
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 v = (tid + g * RP::NT) & ((1u << RP::U0) - 1u);
        grp_fwd_s2_lvl<A, RP::R, RP::U0, 0>(xa + (g << RP::R), xb + (g << RP::R), twb, v, p);
    }
    if constexpr (P < RP::NP - 1) {
        row_xchg<SIGMA, P, E>(xa, buf, tid);
        row_xchg<SIGMA, P, E>(xb, buf, tid);
        srow2_fwd_1b<A, SIGMA, P + 1, EARLY, E>(xa, xb, buf, twb, tid, p, itab, t, ib);
    } else if constexpr (EARLY) {
        row_last_inv_tw<SIGMA, true, E>(twb, itab, t, ib, tid);
        cp_async_commit();
    }
}

// Inverse passes from the leaves in registers; the last pass (P = 0) writes
// the row to global memory in natural order.
template <class A, int SIGMA, int P, int E = 16>
__device__ __forceinline__ void srow2_inv(u32 *x, u32 *ba, u32 *gdst, const RowTw &rt, u32 tid, u32 p) {
    using RP = RowPlan<SIGMA, P, E>;
    if constexpr (P < RP::NP - 1) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_con_s<RP::R>(ba, tid + g * RP::NT, x + (g << RP::R));
    }
#pragma unroll
    for (int g = 0; g < RP::NG; ++g) {
        const u32 v = (tid + g * RP::NT) & ((1u << RP::U0) - 1u);
        grp_inv_rt_lvl<A, SIGMA, RP::R, RP::U0, RP::R - 1, E>(x + (g << RP::R), rt, v, p);
    }
    if constexpr (P == 0) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_str_g<RP::R, RP::S>(gdst, tid + g * RP::NT, x + (g << RP::R));
    } else {
        __syncthreads();
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_str_s<RP::R, RP::S>(ba, tid + g * RP::NT, x + (g << RP::R));
        __syncthreads();
        srow2_inv<A, SIGMA, P - 1, E>(x, ba, gdst, rt, tid, p);
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

// Rows spread over the threads of a CTA: NT = S/E threads per row, E words
// each, passes of log2 E levels with block barriers between them (every
// thread of the CTA reaches every barrier; `on` is false for the threads of
// a row that is not needed, which skip the work).  Same Stockham layout as
// srow_fwd / srow_inv (the row starts and ends in natural order in `buf`);
// the twiddles come from the row's shared-memory copy (stage_tw layout).
template <class A, int SIGMA, int E, int P>
__device__ __forceinline__ void srowc_fwd(u32 *x, u32 *buf, u32 tid, bool on, const uint2 *twb, u32 p) {
    using RP = RowPlan<SIGMA, P, E>;
    if (on) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) ld_str_s<RP::R, RP::S>(buf, tid + g * RP::NT, x + (g << RP::R));
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) {
            const u32 v = (tid + g * RP::NT) & ((1u << RP::U0) - 1u);
            grp_fwd_s<A, RP::R, RP::U0>(x + (g << RP::R), twb, v, p);
        }
    }
    if constexpr (P < RP::NP - 1) {
        __syncthreads();
        if (on) {
#pragma unroll
            for (int g = 0; g < RP::NG; ++g) st_con_s<RP::R>(buf, tid + g * RP::NT, x + (g << RP::R));
        }
        __syncthreads();
        srowc_fwd<A, SIGMA, E, P + 1>(x, buf, tid, on, twb, p);
    }
}
template <class A, int SIGMA, int E, int P>
__device__ __forceinline__ void srowc_inv(u32 *x, u32 *buf, u32 tid, bool on, const uint2 *itwb, u32 p) {
    using RP = RowPlan<SIGMA, P, E>;
    if (on) {
        if constexpr (P < RP::NP - 1) {
#pragma unroll
            for (int g = 0; g < RP::NG; ++g) ld_con_s<RP::R>(buf, tid + g * RP::NT, x + (g << RP::R));
        }
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) {
            const u32 v = (tid + g * RP::NT) & ((1u << RP::U0) - 1u);
            grp_inv_s<A, RP::R, RP::U0>(x + (g << RP::R), itwb, v, p);
        }
    }
    __syncthreads();
    if (on) {
#pragma unroll
        for (int g = 0; g < RP::NG; ++g) st_str_s<RP::R, RP::S>(buf, tid + g * RP::NT, x + (g << RP::R));
    }
    __syncthreads();
    if constexpr (P > 0) srowc_inv<A, SIGMA, E, P - 1>(x, buf, tid, on, itwb, p);
}

// ------------------------------------------------------ column-stage helpers
// A column tile holds rows r < T of C consecutive columns.  Two layouts:
//  LAY_SWZ  (one-CTA kernel, C = 512): row r, column c at swz(r*C + c), the
//           same mapping the row stage's Stockham passes use;
//  LAY_TILE (three-kernel path, C = 8, 16 or 32): row r, column c at
//           (r ^ h(r))*C + c with h(r) = fold_b(r >> 1), the XOR of the b-bit
//           chunks of r >> 1, b = log2(32 / C).  A warp spans 32/C tasks;
//           in every pass shape those tasks' rows then fall in distinct bank
//           groups (checked exhaustively for T <= 2048).  h is linear over the
//           disjoint bit fields of a row index r0 | (q << logJ), so per
//           element it costs one XOR with a compile-time constant.
// Passes cover at most 4 tree levels (16 registers per task), split evenly.
enum { LAY_SWZ = 0, LAY_TILE = 1 };
enum { IO_SMEM = 0, IO_GLOBAL = 1 };

__device__ __forceinline__ int col_npass(int t) { return (t + 3) / 4; }
__device__ __forceinline__ int col_pass_R(int t, int npass, int idx) { return t / npass + (idx < t % npass ? 1 : 0); }

// XOR of the b-bit chunks of x (b = 1 or 2); a loop, so a literal x folds.
__host__ __device__ __forceinline__ constexpr u32 cfold(u32 x, int b) {
    u32 h = 0;
    for (int i = 0; i < 32; i += b) h ^= (x >> i) & ((1u << b) - 1u);
    return h;
}
template <int C>
struct TileSw {
    static constexpr int b = (C >= 32) ? 0 : (C == 16 ? 1 : 2);
};
template <int C>
__device__ __forceinline__ u32 tile_h(u32 r) {
    constexpr int b = TileSw<C>::b;
    if constexpr (b == 0) {
        return 0u;
    } else if constexpr (b == 1) {
        return __popc(r >> 1) & 1u;
    } else {
        u32 x = r >> 1;
        x ^= x >> 16;
        x ^= x >> 8;
        x ^= x >> 4;
        x ^= x >> 2;
        return x & 3u;
    }
}

// Address of element q (row r0 + (q << logJ), column c) of a task.  The row
// swizzle is applied after the (disjoint-bit) sum, as h(r0) ^ h(q << logJ).
template <int C, int LAY>
struct ColAddr {
    u32 base;  // r0 * C + c
    u32 H0;    // h(r0) * C
    int mode;  // which compile-time swizzle constant applies to q << logJ
    int sh;    // logJ + log2(C)
    __device__ __forceinline__ ColAddr(u32 r0, u32 c, int logJ) {
        sh = logJ + (31 - __clz(C));
        base = r0 * C + c;
        if constexpr (LAY == LAY_TILE) {
            H0 = tile_h<C>(r0) * C;
            mode = logJ == 0 ? 0 : (((logJ - 1) & 1) ? 2 : 1);
        } else {
            H0 = 0;
            mode = 0;
        }
    }
    __device__ __forceinline__ u32 at(int q) const {  // q is a literal after unrolling
        const u32 w = base + ((u32)q << sh);
        if constexpr (LAY == LAY_SWZ) {
            return swz(w);
        } else {
            constexpr int b = TileSw<C>::b;
            if constexpr (b == 0) {
                return w;
            } else {
                // h(q << logJ) for logJ = 0, logJ >= 1 with logJ - 1 even, odd
                const u32 h0 = cfold((u32)q >> 1, b) * C, h1 = cfold((u32)q, b) * C, h2 = cfold((u32)q << 1, b) * C;
                const u32 hq = mode == 0 ? h0 : (mode == 1 ? h1 : h2);
                return w ^ H0 ^ hq;
            }
        }
    }
};

struct ColFwdArgs {
    u32 *sm;            // tile in shared memory
    const u32 *g;       // operand (global)
    u32 *W;             // workspace rows (global), row r column c0+c at r*S + c0 + c
    int64_t z;          // operand length
    u32 c0;             // first column of the tile
    int logS;           // log2 of the row length S
    int T, t;           // rows, tree levels of the column stage
    int zb;             // rows holding any nonzero input
    int k;              // rows needed
    bool prune;
    const uint2 *tw;
    u32 p;
    int *status = nullptr;  // device status word (debug-build checks)
};

// One forward pass of R levels starting at depth s0.
template <class A, int R, int C, int LAY, int SRC, int DST, bool TS = false>
__device__ __forceinline__ void colf_pass(const ColFwdArgs &X, int s0) {
    constexpr int logC = ilog2c(C);
    const int logM = X.t - s0, logJ = logM - R;
    const int M = 1 << logM;
    const int tasks = (X.T >> R) << logC;
    u32 copymask = 0;
    if (X.prune) {
#pragma unroll
        for (int d = 0; d < R; ++d)
            if (X.zb <= ((M >> d) >> 1)) copymask |= 1u << d;
    }
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const u32 G = (u32)tau >> logC, c = (u32)tau & (C - 1);
        const u32 v = G >> logJ, j = G & ((1u << logJ) - 1u);
        if (X.prune && (int)(v << logM) >= X.k) continue;
        const u32 r0 = (v << logM) + j;
        u32 x[1 << R];
        if constexpr (SRC == IO_GLOBAL) {
            const u32 e0 = (r0 << X.logS) + X.c0 + c;
            const int sh = logJ + X.logS;
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) {
                const u32 e = e0 + ((u32)q << sh);
                x[q] = ((int64_t)e < X.z) ? __ldg(X.g + e) : 0u;
            }
        } else {
            const ColAddr<C, LAY> ad(r0, c, logJ);
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) x[q] = X.sm[ad.at(q)];
        }
        grp_fwd_cp<A, R, TS>(x, X.tw, s0, v, X.p, copymask);
        if constexpr (DST == IO_GLOBAL) {
            const u32 e0 = (r0 << X.logS) + X.c0 + c;
            const int sh = logJ + X.logS;
#pragma unroll
            for (int q = 0; q < (1 << R); ++q)
                if ((int)(r0 + ((u32)q << logJ)) < X.k) {
                    PM_DCHECK(x[q] < 2 * A::bound(X.p) && c < C && (int64_t)(X.c0 + c) < ((int64_t)1 << X.logS),
                              X.status);
                    X.W[e0 + ((u32)q << sh)] = x[q];
                }
        } else {
            const ColAddr<C, LAY> ad(r0, c, logJ);
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) X.sm[ad.at(q)] = x[q];
        }
    }
}

template <class A, int C, int LAY, int SRC, int DST, bool TS = false>
__device__ __forceinline__ void colf_pass_r(int R, const ColFwdArgs &X, int s0) {
    // at most 4 levels: one 16-word register array; an if-chain over sizes
    // up to 4 keeps it in registers (a 32-word variant next to others spills it)
    if (R == 4) colf_pass<A, 4, C, LAY, SRC, DST, TS>(X, s0);
    else if (R == 3) colf_pass<A, 3, C, LAY, SRC, DST, TS>(X, s0);
    else if (R == 2) colf_pass<A, 2, C, LAY, SRC, DST, TS>(X, s0);
    else colf_pass<A, 1, C, LAY, SRC, DST, TS>(X, s0);
}

// Forward column stage of one tile.  The first pass reads the operand from
// global memory; with `to_global` the last pass writes rows < k to the
// workspace, otherwise the tile ends in shared memory (followed by a barrier).
template <class A, int C, int LAY>
__device__ void colf_tile(const ColFwdArgs &X, bool to_global) {
    if (X.t == 0) {  // one row: plain copy
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            const u32 e = X.c0 + c;
            const u32 v = ((int64_t)e < X.z) ? __ldg(X.g + e) : 0u;
            if (to_global) X.W[e] = v;
            else X.sm[LAY == LAY_SWZ ? swz(c) : (u32)c] = v;
        }
        __syncthreads();
        return;
    }
    const int np = col_npass(X.t);
    int s0 = 0;
    for (int i = 0; i < np; ++i) {
        const int R = col_pass_R(X.t, np, i);
        const bool first = i == 0, last = i == np - 1;
        if (first && last && to_global) colf_pass_r<A, C, LAY, IO_GLOBAL, IO_GLOBAL>(R, X, s0);
        else if (first) colf_pass_r<A, C, LAY, IO_GLOBAL, IO_SMEM>(R, X, s0);
        else if (last && to_global) colf_pass_r<A, C, LAY, IO_SMEM, IO_GLOBAL>(R, X, s0);
        else colf_pass_r<A, C, LAY, IO_SMEM, IO_SMEM>(R, X, s0);
        __syncthreads();
        s0 += R;
    }
}

struct ColInvArgs {
    u32 *sm;
    const u32 *W;   // workspace rows (global) for a first pass from global memory
    u32 *out;       // product (global) for a last pass to global memory
    int64_t n;      // product length
    u32 c0;
    int logS;
    int k;          // rows that hold spectral values / output coefficients
    const uint2 *itw;
    u32 p;
    const uint2 *tw;  // forward table (r of the truncated inverse's records)
    // coli_tile_ct only: the top three levels' twiddles in shared memory,
    // top[e] = fwd[e] and top[8 + e] = inv[e] for tree nodes e = 1..7
    const uint2 *top;
    int *status = nullptr;  // device status word (debug-build checks)
};

// Inverse pass of R levels [lev0, lev0+R) of the subtree rooted at (s_root,
// i_root) covering rows [base, base + 2^logMroot); nodes at depth lev0 have
// 2^logMsub rows.
template <class A, int R, int C, int LAY, int SRC, int DST, bool TS = false>
__device__ __forceinline__ void coli_pass(const ColInvArgs &X, int lev0, int s_root, u32 i_root, int base,
                                          int logMsub, int logNodes) {
    constexpr int logC = ilog2c(C);
    const int logJ = logMsub - R;
    const int tasks = 1 << (logNodes + logJ + logC);
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const u32 G = (u32)tau >> logC, c = (u32)tau & (C - 1);
        const u32 v = G >> logJ, j = G & ((1u << logJ) - 1u);
        const u32 r0 = (u32)base + (v << logMsub) + j;
        u32 x[1 << R];
        if constexpr (SRC == IO_GLOBAL) {
            const u32 e0 = (r0 << X.logS) + X.c0 + c;
            const int sh = logJ + X.logS;
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) x[q] = __ldcg(X.W + e0 + ((u32)q << sh));
        } else {
            const ColAddr<C, LAY> ad(r0, c, logJ);
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) x[q] = X.sm[ad.at(q)];
        }
        grp_inv<A, R, TS>(x, X.itw, lev0, (i_root << (lev0 - s_root)) + v, X.p);
        if constexpr (DST == IO_GLOBAL) {
            const u32 e0 = (r0 << X.logS) + X.c0 + c;
            const int sh = logJ + X.logS;
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) {
                const u32 e = e0 + ((u32)q << sh);
                PM_DCHECK(x[q] < A::bound(X.p), X.status);
                if ((int64_t)e < X.n) X.out[e] = A::to_canon(x[q], X.p);
            }
        } else {
            const ColAddr<C, LAY> ad(r0, c, logJ);
#pragma unroll
            for (int q = 0; q < (1 << R); ++q) X.sm[ad.at(q)] = x[q];
        }
    }
}

template <class A, int C, int LAY, int SRC, int DST, bool TS = false>
__device__ __forceinline__ void coli_pass_r(int R, const ColInvArgs &X, int lev0, int s_root, u32 i_root, int base,
                                            int logMsub, int logNodes) {
    if (R == 4) coli_pass<A, 4, C, LAY, SRC, DST, TS>(X, lev0, s_root, i_root, base, logMsub, logNodes);
    else if (R == 3) coli_pass<A, 3, C, LAY, SRC, DST, TS>(X, lev0, s_root, i_root, base, logMsub, logNodes);
    else if (R == 2) coli_pass<A, 2, C, LAY, SRC, DST, TS>(X, lev0, s_root, i_root, base, logMsub, logNodes);
    else coli_pass<A, 1, C, LAY, SRC, DST, TS>(X, lev0, s_root, i_root, base, logMsub, logNodes);
}

// Unscaled inverse of the subtree (s, i) on rows [base, base + 2^lm): M times
// its coefficients.  Passes run from the deepest levels up.  from_g: the
// first pass reads the workspace; to_g: the last pass writes the product.
// Ends with a barrier.
template <class A, int C, int LAY, bool TS = false>
__device__ void coli_full(const ColInvArgs &X, int s, u32 i, int base, int lm, bool from_g, bool to_g) {
    if (lm == 0) return;
    const int np = col_npass(lm);
    // chunk ch covers relative depths [d0(ch), d0(ch) + R(ch)); executed from ch = np-1 down to 0
    for (int ch = np - 1; ch >= 0; --ch) {
        int d0 = 0;
        for (int q = 0; q < ch; ++q) d0 += col_pass_R(lm, np, q);
        const int R = col_pass_R(lm, np, ch);
        const bool first = ch == np - 1, last = ch == 0;
        const int lev0 = s + d0, logMsub = lm - d0, logNodes = d0;
        if (first && from_g && last && to_g)
            coli_pass_r<A, C, LAY, IO_GLOBAL, IO_GLOBAL, TS>(R, X, lev0, s, i, base, logMsub, logNodes);
        else if (first && from_g)
            coli_pass_r<A, C, LAY, IO_GLOBAL, IO_SMEM, TS>(R, X, lev0, s, i, base, logMsub, logNodes);
        else if (last && to_g)
            coli_pass_r<A, C, LAY, IO_SMEM, IO_GLOBAL, TS>(R, X, lev0, s, i, base, logMsub, logNodes);
        else
            coli_pass_r<A, C, LAY, IO_SMEM, IO_SMEM, TS>(R, X, lev0, s, i, base, logMsub, logNodes);
        __syncthreads();
    }
}

// ------------------------------------------- compile-time column passes
// The same passes with the column depth TL (and so every pass shape, shift
// and twiddle offset) known at compile time; used by the one-product
// kernels.  An element address is one XOR with a constant and an immediate
// offset: (r0*C + c) ^ h(r0)*C ^ h(q<<logJ)*C + (q << (logJ + log2 C)), the
// XOR and the add commuting when logJ >= b (disjoint bits).
template <int C, int LOGJ, int Q>
struct CtAddr {
    static constexpr int b = TileSw<C>::b;
    static constexpr int mode = LOGJ == 0 ? 0 : (((LOGJ - 1) & 1) ? 2 : 1);
    static constexpr u32 hq =
        b == 0 ? 0u : (mode == 0 ? cfold((u32)Q >> 1, b) : (mode == 1 ? cfold((u32)Q, b) : cfold((u32)Q << 1, b))) * C;
    static constexpr u32 off = (u32)Q << (LOGJ + ilog2c(C));
    // rc = r0*C + c, H0 = h(r0)*C
    static __device__ __forceinline__ u32 at(u32 rc, u32 H0) {
        if constexpr (b == 0) return rc + off;
        else if constexpr (LOGJ >= b) return ((rc ^ H0) ^ hq) + off;
        else return (rc + off) ^ H0 ^ hq;
    }
};

// Two adjacent columns (c even) per task: one 64-bit access per row.
template <int C, int LOGJ, int R, int Q = 0>
__device__ __forceinline__ void ct_load2(u32 *x, u32 *y, const u32 *sm, u32 rc, u32 H0) {
    if constexpr (Q < (1 << R)) {
        const uint2 v = *reinterpret_cast<const uint2 *>(sm + CtAddr<C, LOGJ, Q>::at(rc, H0));
        x[Q] = v.x;
        y[Q] = v.y;
        ct_load2<C, LOGJ, R, Q + 1>(x, y, sm, rc, H0);
    }
}
template <int C, int LOGJ, int R, int Q = 0>
__device__ __forceinline__ void ct_store2(const u32 *x, const u32 *y, u32 *sm, u32 rc, u32 H0) {
    if constexpr (Q < (1 << R)) {
        *reinterpret_cast<uint2 *>(sm + CtAddr<C, LOGJ, Q>::at(rc, H0)) = make_uint2(x[Q], y[Q]);
        ct_store2<C, LOGJ, R, Q + 1>(x, y, sm, rc, H0);
    }
}

// Forward pass of R levels at depth S0 of a TL-level column stage.  A task is
// one group of 2^R rows in two adjacent columns.
template <class A, int R, int C, int TL, int S0, int DST>
__device__ __forceinline__ void colf_pass_ct(const ColFwdArgs &X, u32 copymask) {
    constexpr int logC2 = ilog2c(C) - 1, logM = TL - S0, logJ = logM - R;
    constexpr int tasks = (1 << (TL - R)) << logC2;
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const u32 G = (u32)tau >> logC2, c = ((u32)tau & ((C >> 1) - 1)) << 1;
        const u32 v = G >> logJ, j = G & ((1u << logJ) - 1u);
        if (X.prune && (int)(v << logM) >= X.k) continue;
        const u32 r0 = (v << logM) | j;
        const u32 rc = r0 * C + c, H0 = tile_h<C>(r0) * C;
        u32 x[1 << R], y[1 << R];
        ct_load2<C, logJ, R>(x, y, X.sm, rc, H0);
        grp_fwd_cp2<A, R, S0 == 0>(x, y, X.tw, S0, v, X.p, copymask >> S0);  // S0 = 0: v is 0
        if constexpr (DST == IO_GLOBAL) {
            const u32 e0 = (r0 << X.logS) + X.c0 + c;
            const int sh = logJ + X.logS;
#pragma unroll
            for (int q = 0; q < (1 << R); ++q)
                if ((int)(r0 + ((u32)q << logJ)) < X.k) {
                    PM_DCHECK(x[q] < 2 * A::bound(X.p) && y[q] < 2 * A::bound(X.p) &&
                                  (int64_t)(X.c0 + c + 1) < ((int64_t)1 << X.logS),
                              X.status);
                    *reinterpret_cast<uint2 *>(X.W + e0 + ((u32)q << sh)) = make_uint2(x[q], y[q]);
                }
        } else {
            ct_store2<C, logJ, R>(x, y, X.sm, rc, H0);
        }
    }
}

template <int TL, int I>
struct ColSplit {  // pass I of an even split of TL levels into passes of <= 4
    static constexpr int np = (TL + 3) / 4;
    static constexpr int R = TL / np + (I < TL % np ? 1 : 0);
    static constexpr int S0 = I == 0 ? 0 : ColSplit<TL, I - 1>::S0 + ColSplit<TL, I - 1>::R;
};
template <int TL>
struct ColSplit<TL, -1> {
    static constexpr int R = 0, S0 = 0;
};

template <class A, int C, int TL, int I>
__device__ __forceinline__ void colf_passes_ct(const ColFwdArgs &X, u32 copymask) {
    using P = ColSplit<TL, I>;
    if constexpr (I < P::np) {
        if constexpr (I == P::np - 1) {
            colf_pass_ct<A, P::R, C, TL, P::S0, IO_GLOBAL>(X, copymask);
        } else {
            colf_pass_ct<A, P::R, C, TL, P::S0, IO_SMEM>(X, copymask);
        }
        __syncthreads();
        colf_passes_ct<A, C, TL, I + 1>(X, copymask);
    }
}

// Whole forward column stage of a loaded tile (TL >= 1 levels); the last pass
// writes rows < k of the workspace.  Ends with a barrier.
template <class A, int C, int TL>
__device__ __forceinline__ void colf_tile_ct(const ColFwdArgs &X) {
    u32 copymask = 0;  // bit s: every upper input at depth s is zero
    if (X.prune) {
#pragma unroll
        for (int s = 0; s < TL; ++s)
            if (X.zb <= ((X.T >> s) >> 1)) copymask |= 1u << s;
    }
    colf_passes_ct<A, C, TL, 0>(X, copymask);
}

template <int C, int LAY>
__device__ __forceinline__ u32 col_elem_addr(u32 r, u32 c) {
    if constexpr (LAY == LAY_SWZ) return swz(r * C + c);
    else return (r * C + c) ^ (tile_h<C>(r) * C);
}

// x / 2 mod p for x in [0, B): (x + p) / 2 when x is odd.  Stays in [0, B).
__device__ __forceinline__ u32 half_mod(u32 x, u32 p) { return (x + (x & 1u) * p) >> 1; }

// The truncated inverse (ITFT) of a tile in shared memory from its step list.
// On entry rows [0, k) hold spectral values, each already multiplied by
// 1/h for the size h of the FULL record that inverts it (the row stage
// folds that factor into its pointwise constant), so every FULL leaves true
// coefficients and no record needs an h^-1 multiply.  Rows >= k are never
// read before written.  On exit rows [0, k) hold the coefficients.  Values
// stay in [0, B) throughout.  Elementwise records handle two adjacent
// columns per task.
template <class A, int C, int LAY, bool TS = false>
__device__ void coli_steps(const ColInvArgs &X, const ItftStep *__restrict__ steps, int nsteps) {
    constexpr int logC2 = ilog2c(C) - 1;
    const u32 p = X.p, B = A::bound(p);
    for (int si = 0; si < nsteps; ++si) {
        const ItftStep st = steps[si];
        if (st.kind == ST_FULL) {
            coli_full<A, C, LAY, TS>(X, st.s, st.i, st.base, 31 - __clz(st.h), false, false);
            continue;
        }
        const bool upper = (st.kind == ST_PRE_RIGHT || st.kind == ST_PRE_LEFT);
        const int lo = upper ? st.m : 0, hi = upper ? st.h : st.m;
        const int tasks = (hi - lo) << logC2;
        for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
            const u32 j = (u32)lo + ((u32)tau >> logC2), c = ((u32)tau & ((C >> 1) - 1)) << 1;
            uint2 *P0 = reinterpret_cast<uint2 *>(X.sm + col_elem_addr<C, LAY>((u32)st.base + j, c));
            uint2 *P1 = reinterpret_cast<uint2 *>(X.sm + col_elem_addr<C, LAY>((u32)(st.base + st.h) + j, c));
            const uint2 v0 = *P0;
            if (st.kind == ST_PRE_RIGHT && st.zero) {  // X_{j+h} = X_j
                *P1 = v0;
                continue;
            }
            const uint2 v1 = *P1;
            const u32 x[2] = {v0.x, v0.y}, y[2] = {v1.x, v1.y};
            u32 o0[2], o1[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (st.kind == ST_POST_RIGHT) {  // ((x + y) / 2, (x - y) / (2r))
                    o0[e] = half_mod(A::fwd_to_inv(x[e] + y[e], p), p);
                    u32 t = shoup(x[e] - y[e] + B, st.i2r, p);
                    o1[e] = A::lazy ? t : canon2(t, p);
                } else {
                    u32 t = shoup(y[e], st.r, p);
                    if (!A::lazy) t = canon2(t, p);
                    if (st.kind == ST_PRE_RIGHT) {  // X_j = x - r y; X_{j+h} = X_j - r y
                        const u32 xj = A::fwd_to_inv(x[e] - t + B, p);
                        o0[e] = xj;
                        o1[e] = A::fwd_to_inv(xj - t + B, p);
                    } else if (st.kind == ST_PRE_LEFT) {
                        o0[e] = A::fwd_to_inv(x[e] + t, p);
                    } else {  // ST_POST_LEFT
                        o0[e] = A::fwd_to_inv(x[e] - t + B, p);
                    }
                }
            }
            *P0 = make_uint2(o0[0], o0[1]);
            if (st.kind == ST_PRE_RIGHT || st.kind == ST_POST_RIGHT) *P1 = make_uint2(o1[0], o1[1]);
        }
        __syncthreads();
    }
}

// ------------------------------------ truncated column inverse, one kernel
// With k a multiple of T/8 (relaxed truncation; any k when T <= 8), every
// bookkeeping record of the ITFT recursion sits in the top TOP = min(t, 3)
// levels, and below them the recursion only inverts whole subtrees.  Those
// subtree inverses are the deep levels of a plain full inverse restricted to
// rows < k, so the kernel runs (1) the full inverse's passes over levels
// [TOP, t) on rows < k, then (2) one pass in which each task holds the
// 2^TOP rows j, j + T/2^TOP, ... of two columns in registers and runs the
// top levels of the recursion there -- subtree butterflies, PRE/POST records
// -- before storing the rows < k of the product.  k = T is the full inverse.

// (a, b) -> ((a + b) / 2, (a - b) / (2r)) with ri = r^-1; [0, B) -> [0, B).
template <class A>
__device__ __forceinline__ void post_right(u32 &a, u32 &b, uint2 ri, u32 p) {
    const u32 B = A::bound(p);
    u32 d = shoup(a - b + B, ri, p);
    if (!A::lazy) d = canon2(d, p);
    const u32 s = A::fwd_to_inv(a + b, p);
    a = half_mod(s, p);
    b = half_mod(d, p);
}

// x, y: the M = 2^(levels) blocks of node (S, I) (two columns).  Unscaled
// inverse of the whole node.
template <class A, int M, int S, int I>
__device__ __forceinline__ void top_full_inv(u32 *x, u32 *y, const uint2 *top, u32 p) {
    if constexpr (M >= 2) {
        constexpr int h = M / 2;
        top_full_inv<A, h, S + 1, 2 * I>(x, y, top, p);
        top_full_inv<A, h, S + 1, 2 * I + 1>(x + h, y + h, top, p);
        if constexpr (I == 0) {  // the first node of its level: twiddle 1
#pragma unroll
            for (int j = 0; j < h; ++j) {
                A::gs_one(x[j], x[j + h], p);
                A::gs_one(y[j], y[j + h], p);
            }
        } else {
            const uint2 w = top[8 + (1 << S) + I];
#pragma unroll
            for (int j = 0; j < h; ++j) {
                A::gs(x[j], x[j + h], w, p);
                A::gs(y[j], y[j + h], w, p);
            }
        }
    }
}

// The ITFT recursion on node (S, I) of M blocks with k leading spectral
// blocks (runtime); ZERO: the blocks past k hold zero coefficients.  Values
// in [0, B); the spectral blocks arrive prescaled (see coli_steps).
template <class A, int M, int S, int I, bool ZERO>
__device__ __forceinline__ void itft_top(u32 *x, u32 *y, int k, const uint2 *top, u32 p) {
    if constexpr (M >= 2) {
        if (k <= 0) return;
        if (k == M) {
            top_full_inv<A, M, S, I>(x, y, top, p);
            return;
        }
        constexpr int h = M / 2;
        const u32 B = A::bound(p);
        const uint2 r = top[(1 << S) + I];
        if (k >= h) {
            const int m = k - h;
            top_full_inv<A, h, S + 1, 2 * I>(x, y, top, p);
#pragma unroll
            for (int j = 0; j < h; ++j) {
                if (j < m) continue;
                if (ZERO) {  // X_{j+h} = X_j
                    x[j + h] = x[j];
                    y[j + h] = y[j];
                } else {  // X_j -= r X_{j+h}; X_{j+h} = X_j - r X_{j+h}
                    u32 t = shoup(x[j + h], r, p), u = shoup(y[j + h], r, p);
                    if (!A::lazy) {
                        t = canon2(t, p);
                        u = canon2(u, p);
                    }
                    x[j] = A::fwd_to_inv(x[j] - t + B, p);
                    y[j] = A::fwd_to_inv(y[j] - u + B, p);
                    x[j + h] = A::fwd_to_inv(x[j] - t + B, p);
                    y[j + h] = A::fwd_to_inv(y[j] - u + B, p);
                }
            }
            itft_top<A, h, S + 1, 2 * I + 1, false>(x + h, y + h, m, top, p);
            const uint2 ri = top[8 + (1 << S) + I];
#pragma unroll
            for (int j = 0; j < h; ++j) {
                if (j >= m) continue;
                post_right<A>(x[j], x[j + h], ri, p);
                post_right<A>(y[j], y[j + h], ri, p);
            }
        } else {
            if (!ZERO) {
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    if (j < k) continue;
                    u32 t = shoup(x[j + h], r, p), u = shoup(y[j + h], r, p);
                    if (!A::lazy) {
                        t = canon2(t, p);
                        u = canon2(u, p);
                    }
                    x[j] = A::fwd_to_inv(x[j] + t, p);
                    y[j] = A::fwd_to_inv(y[j] + u, p);
                }
            }
            itft_top<A, h, S + 1, 2 * I, ZERO>(x, y, k, top, p);
            if (!ZERO) {
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    if (j >= k) continue;
                    u32 t = shoup(x[j + h], r, p), u = shoup(y[j + h], r, p);
                    if (!A::lazy) {
                        t = canon2(t, p);
                        u = canon2(u, p);
                    }
                    x[j] = A::fwd_to_inv(x[j] - t + B, p);
                    y[j] = A::fwd_to_inv(y[j] - u + B, p);
                }
            }
        }
    }
}

// Deep inverse pass (levels [S0, S0+R), S0 >= TOP) on rows < k only; a
// group never straddles a block of T/2^TOP rows, so it is all in or all out.
template <class A, int R, int C, int TL, int S0, int SRC>
__device__ __forceinline__ void coli_deep_pass(const ColInvArgs &X) {
    constexpr int logC2 = ilog2c(C) - 1, logM = TL - S0, logJ = logM - R;
    constexpr int tasks = (1 << (TL - R)) << logC2;
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const u32 G = (u32)tau >> logC2, c = ((u32)tau & ((C >> 1) - 1)) << 1;
        const u32 v = G >> logJ, j = G & ((1u << logJ) - 1u);
        const u32 r0 = (v << logM) | j;
        if ((int)r0 >= X.k) continue;
        const u32 rc = r0 * C + c, H0 = tile_h<C>(r0) * C;
        u32 x[1 << R], y[1 << R];
        ct_load2<C, logJ, R>(x, y, X.sm, rc, H0);
        grp_inv2<A, R>(x, y, X.itw, S0, v, X.p);
        ct_store2<C, logJ, R>(x, y, X.sm, rc, H0);
    }
}

template <class A, int C, int TL, int TOP, int I>
__device__ __forceinline__ void coli_deep_passes(const ColInvArgs &X) {
    using P = ColSplit<TL - TOP, I>;
    if constexpr (I >= 0) {
        coli_deep_pass<A, P::R, C, TL, TOP + P::S0, IO_SMEM>(X);
        __syncthreads();
        coli_deep_passes<A, C, TL, TOP, I - 1>(X);
    }
}

template <int C, int LOGJ, int Q, int NQ>
__device__ __forceinline__ void top_load2(u32 *x, u32 *y, const u32 *sm, u32 rc, u32 H0, int q) {
    if constexpr (Q < NQ) {
        if (Q < q) {
            const uint2 v = *reinterpret_cast<const uint2 *>(sm + CtAddr<C, LOGJ, Q>::at(rc, H0));
            x[Q] = v.x;
            y[Q] = v.y;
        } else {
            x[Q] = 0u;
            y[Q] = 0u;
        }
        top_load2<C, LOGJ, Q + 1, NQ>(x, y, sm, rc, H0, q);
    }
}

// Whole truncated (or, for k = T, full) column inverse of a loaded tile;
// stores rows < k (entries < n) of the product.  Ends with a barrier.
template <class A, int C, int TL>
__device__ __forceinline__ void coli_tile_ct(const ColInvArgs &X) {
    constexpr int TOP = TL < 3 ? TL : 3, NQ = 1 << TOP, LOGB = TL - TOP;
    if constexpr (LOGB > 0) coli_deep_passes<A, C, TL, TOP, ColSplit<LOGB, 0>::np - 1>(X);
    const int q = X.k >> LOGB;  // spectral blocks (k is a multiple of 2^LOGB)
    constexpr int logC2 = ilog2c(C) - 1;
    constexpr int tasks = (1 << LOGB) << logC2;
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const u32 j = (u32)tau >> logC2, c = ((u32)tau & ((C >> 1) - 1)) << 1;
        const u32 rc = j * C + c, H0 = tile_h<C>(j) * C;
        u32 x[NQ], y[NQ];
        top_load2<C, LOGB, 0, NQ>(x, y, X.sm, rc, H0, q);
        itft_top<A, NQ, 0, 0, true>(x, y, q, X.top, X.p);
        const u32 e0 = (j << X.logS) + X.c0 + c;
#pragma unroll
        for (int b = 0; b < NQ; ++b) {
            if (b >= q) break;
            const u32 e = e0 + ((u32)b << (LOGB + X.logS));
            PM_DCHECK(x[b] < A::bound(X.p) && y[b] < A::bound(X.p) && c + 1 < C, X.status);
            if ((int64_t)e < X.n) X.out[e] = A::to_canon(x[b], X.p);
            if ((int64_t)e + 1 < X.n) X.out[e + 1] = A::to_canon(y[b], X.p);
        }
    }
    __syncthreads();
}

}  // namespace pm
