// conv.cu -- cyclic and negacyclic convolutions of length N (C-ABI).
//
// Cyclic: c = a * b mod (x^N - 1), the circular convolution of Definition 4
// (Eq. 5), computed as Eq. 11 does: when N is a power of two the product
// kernels run with L = N and all N outputs (n = L, no truncation), which is
// the full transform, pointwise product and inverse of the convolution
// theorem (Eq. 8-10).  Negacyclic: c = a * b mod (x^N + 1), the other factor
// of Eq. 13.  When N is a power of two >= 512 and 2N divides p - 1 it is a
// twisted cyclic convolution of the same length N: with psi a primitive
// 2N-th root of unity (psi^N = -1), x = psi y turns x^N + 1 into
// -(y^N - 1), so c_i psi^i is the cyclic convolution of a_i psi^i and
// b_i psi^i; the twist and the untwist are one element-wise kernel each.
// Every other case (N not a power of two, N < 512, or 2N not dividing
// p - 1) computes the linear product u (TFT path) into a workspace and folds
// it: c_i = u_i + u_{i+N} (cyclic) or u_i - u_{i+N} (negacyclic);
// deg u <= 2N - 2, so one fold suffices.
#include <stdint.h>

#include <algorithm>

#include "host.h"
#include "polymul.h"

namespace pm {

__global__ void k_fold(const u32 *__restrict__ u, int64_t nu, u32 *__restrict__ c, int64_t N, u32 p, int neg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const u32 v = i < nu ? u[i] : 0u;
        const u32 w = i + N < nu ? u[i + N] : 0u;
        c[i] = neg ? sub_c(v, w, p) : add_c(v, w, p);
    }
}

static int conv_fold(uint32_t p, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int64_t N, bool neg,
                     cudaStream_t st) {
    const int64_t nu = za + zb - 1;
    const int l = ceil_log2(nu);
    if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    u32 *u = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&u, (size_t)nu * sizeof(u32), st);
    if (e != cudaSuccess) {
        cuda_fail(e, "convolution workspace");
        return POLY_ENOMEM;
    }
    int rc = run_product(p, 0, a, za, b, zb, u, l, true, st, nullptr);
    if (rc == POLY_OK) {
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>((N + threads - 1) / threads, 4096);
        k_fold<<<(int)blocks, threads, 0, st>>>(u, nu, c, N, p, neg ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "fold launch");
    }
    cudaError_t ef = cudaFreeAsync(u, st);
    if (rc == POLY_OK && ef != cudaSuccess) rc = cuda_fail(ef, "convolution workspace free");
    return rc;
}

// psi^(+-i) for the twist of a length-N = 2^l negacyclic convolution, psi =
// psi_{l+1} the primitive 2^(l+1)-th root: entry 2^l + rev_l(j) of the
// merged tree's table holds psi^j (inverse table: psi^-j), so with i split
// as i = i_hi + i_lo (i_lo < 1024) two Shoup multiplies by resident entries
// give x psi^(+-i).  Canonical in, canonical out.
__device__ __forceinline__ u32 twist_one(u32 x, int64_t i, const uint2 *__restrict__ tab, int l, u32 p) {
    const u32 ii = (u32)i;
    const u32 lo = ii & 1023u, hi = ii & ~1023u;
    const uint2 wl = __ldg(tab + (1u << l) + (l ? (__brev(lo) >> (32 - l)) : 0u));
    const uint2 wh = __ldg(tab + (1u << l) + (l ? (__brev(hi) >> (32 - l)) : 0u));
    return mul_c(mul_c(x, wl, p), wh, p);
}

// a'_i = a_i psi^i (i < za), b'_i = b_i psi^i (i < zb).
__global__ void k_twist2(const u32 *__restrict__ a, int64_t za, const u32 *__restrict__ b, int64_t zb,
                         u32 *__restrict__ ta, u32 *__restrict__ tb, const uint2 *__restrict__ tab, int l, u32 p) {
    const int64_t z = za > zb ? za : zb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < z; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < za) ta[i] = twist_one(a[i], i, tab, l, p);
        if (i < zb) tb[i] = twist_one(b[i], i, tab, l, p);
    }
}

// c_i <- c_i psi^-i in place (tab: the inverse table).
__global__ void k_untwist(u32 *__restrict__ c, int64_t N, const uint2 *__restrict__ tab, int l, u32 p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = twist_one(c[i], i, tab, l, p);
}

static int negacyclic_twisted(uint32_t p, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l,
                              cudaStream_t st) {
    const int64_t N = (int64_t)1 << l;
    PrimeCtx *ctx = nullptr;
    int rc = get_prime(p, 0, l + 1, &ctx, st);  // the table must reach depth l (psi = psi_{l+1})
    if (rc) return rc;
    const int64_t za4 = (za + 3) & ~(int64_t)3;
    u32 *w = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&w, (size_t)(za4 + zb) * sizeof(u32), st);
    if (e != cudaSuccess) {
        cuda_fail(e, "negacyclic workspace");
        return POLY_ENOMEM;
    }
    const int threads = 256;
    const int64_t zmax = std::max(za, zb);
    k_twist2<<<(int)std::min<int64_t>((zmax + threads - 1) / threads, 4096), threads, 0, st>>>(
        a, za, b, zb, w, w + za4, ctx->tw.fwd, l, p);
    e = cudaGetLastError();
    rc = e == cudaSuccess ? run_product(p, 0, w, za, w + za4, zb, c, l, true, st, nullptr, N) : cuda_fail(e, "twist");
    if (rc == POLY_OK) {
        k_untwist<<<(int)std::min<int64_t>((N + threads - 1) / threads, 4096), threads, 0, st>>>(c, N, ctx->tw.inv,
                                                                                               l, p);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "untwist");
    }
    cudaError_t ef = cudaFreeAsync(w, st);
    if (rc == POLY_OK && ef != cudaSuccess) rc = cuda_fail(ef, "negacyclic workspace free");
    return rc;
}

static int conv_check(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, const uint32_t *c,
                      int64_t N, cudaStream_t st) {
    if (!a || !b || !c) return POLY_ENULL;
    if (N < 1 || za < 1 || zb < 1 || za > N || zb > N) return POLY_EINVAL;
    if (validation_on()) {
        u32 root = 0;
        int rc = validate_prime(p, &root);
        if (rc) return rc;
        return validate_coeffs(p, a, za, b, zb, st);
    }
    return POLY_OK;
}

}  // namespace pm

using namespace pm;

extern "C" {

int polymul_cyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, uint32_t *c,
                         int64_t N, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = conv_check(p, a, za, b, zb, c, N, st);
    if (rc) return rc;
    const int l = ceil_log2(N);
    if (((int64_t)1 << l) == N && l >= SMALL_LOG_S) {
        if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
        return run_product(p, 0, a, za, b, zb, c, l, true, st, nullptr, N);
    }
    return conv_fold(p, a, za, b, zb, c, N, false, st);
}

int polymul_negacyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, uint32_t *c,
                             int64_t N, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = conv_check(p, a, za, b, zb, c, N, st);
    if (rc) return rc;
    const int l = ceil_log2(N);
    if (((int64_t)1 << l) == N && l >= SMALL_LOG_S && l + 1 <= POLY_MAX_LOG_L) {
        u32 root = 0;
        rc = validate_prime(p, &root);
        if (rc) return rc;
        if (l + 1 <= __builtin_ctz(p - 1)) return negacyclic_twisted(p, a, za, b, zb, c, l, st);
    }
    return conv_fold(p, a, za, b, zb, c, N, true, st);
}

}  // extern "C"
