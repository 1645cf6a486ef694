// k_generic.cu -- twiddle-table construction and the per-level kernels used
// by the standalone transforms (tft_exec / itft_exec) for any length L.
//
// The per-level kernels apply one depth of the merged Cooley-Tukey tree to an
// array of L words in global memory, one butterfly per thread; the standalone
// ITFT runs its step list with them (see itft_exec in host.cu).
#include "internal.h"

namespace pm {

// tw[2^s + i] = psi^(E), E = rev_s(i) * 2^(lmax-1-s), psi a primitive
// 2^lmax-th root; inverse entries use psi^(2^lmax - E).  psi^E is assembled
// from two host-computed power tables (low 12 bits / high bits of E).
__global__ void k_build_tw(uint2 *fwd, uint2 *inv, int lmax, u32 p, const u32 *__restrict__ pw_lo,
                           const u32 *__restrict__ pw_hi) {
    const u32 total = 1u << lmax;
    for (u32 x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
        if (x == 0) {
            const u32 one_q = (u32)((((u64)1) << 32) / p);
            fwd[0] = make_uint2(1u, one_q);
            inv[0] = make_uint2(1u, one_q);
            continue;
        }
        const int s = 31 - __clz(x);
        const u32 i = x - (1u << s);
        const u32 e = s ? (__brev(i) >> (32 - s)) : 0u;
        const u32 E = e << (lmax - 1 - s);
        const u32 Ei = E ? total - E : 0u;
        const u32 w = (u32)((u64)pw_lo[E & 4095u] * pw_hi[E >> 12] % p);
        const u32 wi = (u32)((u64)pw_lo[Ei & 4095u] * pw_hi[Ei >> 12] % p);
        fwd[x] = make_uint2(w, (u32)(((u64)w << 32) / p));
        inv[x] = make_uint2(wi, (u32)(((u64)wi << 32) / p));
    }
}

cudaError_t launch_build_tw(uint2 *fwd, uint2 *inv, int lmax, u32 p, const u32 *pw_lo, const u32 *pw_hi,
                            cudaStream_t st) {
    const u32 total = 1u << lmax;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_build_tw<<<blocks, 256, 0, st>>>(fwd, inv, lmax, p, pw_lo, pw_hi);
    return cudaGetLastError();
}

static int grid_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

__global__ void k_copy_pad(const u32 *__restrict__ in, int64_t z, u32 *x, int64_t L) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = e < z ? in[e] : 0u;
}

cudaError_t launch_copy_pad(const uint32_t *in, int64_t z, uint32_t *x, int64_t L, cudaStream_t st) {
    k_copy_pad<<<grid_for(L), 256, 0, st>>>(in, z, x, L);
    return cudaGetLastError();
}

// Depth s of TFT(L, z, n): node i covers [i M, i M + M), M = L >> s, and has
// nonzero entries only in its first min(z, M) rows; nodes with i M >= n are
// not needed.
template <class A>
__global__ void k_fwd_level(u32 *x, int64_t L, int s, int64_t n, int64_t z, ModParams m, const uint2 *__restrict__ tw) {
    const int64_t M = L >> s, h = M >> 1;
    const int64_t sup = z < M ? z : M;
    for (int64_t tau = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tau < L / 2;
         tau += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = tau / h, j = tau % h;
        if (i * M >= n || j >= sup) continue;
        u32 *lo = x + i * M + j, *hi = lo + h;
        if (j + h < sup) {
            u32 a = *lo, b = *hi;
            A::ct(a, b, __ldg(tw + tw_index(s, (u32)i)), m.p);
            *lo = a;
            *hi = b;
        } else {
            *hi = *lo;
        }
    }
}

// Depth s of the unscaled inverse inside the subtree rooted at (s_root,
// i_root) covering [base, base + M).
template <class A>
__global__ void k_inv_level(u32 *x, int s, int64_t base, int64_t M, int s_root, u32 i_root, ModParams m,
                            const uint2 *__restrict__ itw) {
    const int64_t Ms = M >> (s - s_root), h = Ms >> 1;
    const int64_t total = M >> 1;
    for (int64_t tau = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tau < total;
         tau += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = tau / h, j = tau % h;
        u32 *lo = x + base + v * Ms + j, *hi = lo + h;
        u32 a = *lo, b = *hi;
        A::gs(a, b, __ldg(itw + tw_index(s, (i_root << (s - s_root)) + (u32)v)), m.p);
        *lo = a;
        *hi = b;
    }
}

template <class A>
__global__ void k_step(ItftStep st, u32 *x, ModParams m) {
    const u32 p = m.p;
    const bool upper = (st.kind == ST_PRE_RIGHT || st.kind == ST_PRE_LEFT);
    const int64_t lo = upper ? st.m : 0, hi = upper ? st.h : st.m;
    for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi;
         j += (int64_t)gridDim.x * blockDim.x) {
        u32 *X0 = x + st.base + j, *X1 = X0 + st.h;
        const u32 x0 = A::to_canon(*X0, p), x1 = A::to_canon(*X1, p);
        switch (st.kind) {
            case ST_PRE_RIGHT: {
                const u32 l = mul_c(x0, st.hinv, p);
                if (st.zero) {
                    *X0 = l;
                    *X1 = l;
                } else {
                    const u32 rc = mul_c(x1, st.r, p);
                    const u32 cj = sub_c(l, rc, p);
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
}

template <class A>
__global__ void k_finish(const u32 *__restrict__ x, u32 *out, int64_t n, uint2 scale, int apply, ModParams m) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        u32 v = x[e];
        v = apply ? mul_c(v, scale, m.p) : canon2(umin32(v, v - A::bound(m.p)), m.p);
        out[e] = v;
    }
}

cudaError_t launch_fwd_level(bool lazy, uint32_t *x, int64_t L, int s, int64_t n, int64_t z, ModParams m,
                             TwTables tw, cudaStream_t st) {
    if (lazy)
        k_fwd_level<Arith<true>><<<grid_for(L / 2), 256, 0, st>>>(x, L, s, n, z, m, tw.fwd);
    else
        k_fwd_level<Arith<false>><<<grid_for(L / 2), 256, 0, st>>>(x, L, s, n, z, m, tw.fwd);
    return cudaGetLastError();
}

cudaError_t launch_inv_level(bool lazy, uint32_t *x, int s, int64_t base, int64_t M, int s_root, uint32_t i_root,
                             ModParams m, TwTables tw, cudaStream_t st) {
    if (lazy)
        k_inv_level<Arith<true>><<<grid_for(M / 2), 256, 0, st>>>(x, s, base, M, s_root, i_root, m, tw.inv);
    else
        k_inv_level<Arith<false>><<<grid_for(M / 2), 256, 0, st>>>(x, s, base, M, s_root, i_root, m, tw.inv);
    return cudaGetLastError();
}

cudaError_t launch_step(bool lazy, const ItftStep &stp, uint32_t *x, ModParams m, cudaStream_t st) {
    const int64_t work = stp.h;
    if (lazy)
        k_step<Arith<true>><<<grid_for(work), 256, 0, st>>>(stp, x, m);
    else
        k_step<Arith<false>><<<grid_for(work), 256, 0, st>>>(stp, x, m);
    return cudaGetLastError();
}

cudaError_t launch_finish(bool lazy, const uint32_t *x, uint32_t *out, int64_t n, uint2 scale, int apply_scale,
                          ModParams m, cudaStream_t st) {
    if (lazy)
        k_finish<Arith<true>><<<grid_for(n), 256, 0, st>>>(x, out, n, scale, apply_scale, m);
    else
        k_finish<Arith<false>><<<grid_for(n), 256, 0, st>>>(x, out, n, scale, apply_scale, m);
    return cudaGetLastError();
}

}  // namespace pm
