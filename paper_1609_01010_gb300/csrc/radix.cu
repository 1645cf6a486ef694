// radix.cu -- products with a transform length L = m 2^k that is not a power
// of two (the general-radix TFT that Section 1 cites from [25, 27] as the
// cure for the power-of-two stair-case), truncated at the radix-m level the
// way Section 5's relaxed algorithms truncate: at block granularity.
//
// With w a principal L-th root of unity and zeta = w^N (N = 2^k) a primitive
// m-th root, x^L - 1 = prod_{j<m} (x^N - zeta^j).  A product u of degree < n
// <= m2 N (m2 = ceil(n / N) <= m) is fixed by its residues modulo the first
// m2 factors, so only those are computed:
//   1. k_radix_fold:   for both operands and j < m2, the residue
//        g_j[i] = sum_q g[i + qN] zeta^(jq)           (g mod (x^N - zeta^j))
//      twisted by beta_j^i, beta_j = w^j (beta_j^N = zeta^j), which turns
//      the product modulo x^N - zeta^j into a cyclic convolution of length N;
//   2. m2 cyclic convolutions of length N (Definition 4, Eq. 11) by the
//      power-of-two kernels, on forked streams so that they overlap;
//   3. k_radix_unfold: untwist by beta_j^-i and solve the m2 x m2 Vandermonde
//      system V[j][q] = zeta^(jq) position by position (the inverse m-point
//      DFT when m2 = m) for the blocks u[qN .. qN + N).
// Twist factors w^(ij) come from two small tables per j (low and high bits of
// i), two Shoup multiplications each; the Vandermonde inverse is solved on
// the host (m2 <= 15).
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "host.h"
#include "polymul.h"

namespace pm {

namespace radix {
constexpr int MAXM = 15;      // largest radix
constexpr int MIN_LOG_N = 9;  // N >= 512: the cyclic convolutions use the full-transform kernels
constexpr int MAX_LOG_N = 23;
constexpr int LO_BITS = 10;   // twist tables: low 10 bits of i, then the rest
}  // namespace radix

struct RadixParams {
    u32 p;
    int m, m2, k;
    int64_t N, z[2], n;
    const uint2 *lo, *hi;  // twist tables of this direction: lo[j][il], hi[j][ih]
    int lo_len, hi_len;
    uint2 zpow[radix::MAXM];                 // zeta^e, e < m
    uint2 vinv[radix::MAXM][radix::MAXM];    // V^-1 (unfold)
};

// beta_j^(+-i) x: two Shoup multiplications by the table entries of i.
__device__ __forceinline__ u32 radix_twist(u32 x, const RadixParams &P, int j, u32 i) {
    const u32 il = i & ((1u << radix::LO_BITS) - 1u), ih = i >> radix::LO_BITS;
    const u32 t = mul_c(x, __ldg(P.lo + (size_t)j * P.lo_len + il), P.p);
    return mul_c(t, __ldg(P.hi + (size_t)j * P.hi_len + ih), P.p);
}

// One thread per (operand, i): out[(o M2 + j) N + i] = beta_j^i g_j[i].
// M2 (the number of factors computed) is a compile-time constant so that
// the per-thread arrays stay in registers.
template <int M2>
__global__ void __launch_bounds__(256) k_radix_fold(const u32 *__restrict__ a, const u32 *__restrict__ b,
                                                    u32 *__restrict__ out, const RadixParams P) {
    const int64_t N = P.N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int o = idx >= N;
        const u32 i = (u32)(idx - (o ? N : 0));
        const u32 *g = o ? b : a;
        const int64_t z = P.z[o];
        u32 x[M2];
#pragma unroll
        for (int q = 0; q < M2; ++q) {
            const int64_t e = (int64_t)i + (int64_t)q * N;
            x[q] = e < z ? __ldg(g + e) : 0u;
        }
#pragma unroll
        for (int j = 0; j < M2; ++j) {
            u32 s = 0;
            int e = 0;  // j q mod m
#pragma unroll
            for (int q = 0; q < M2; ++q) {
                s = add_c(s, mul_c(x[q], P.zpow[e], P.p), P.p);
                e += j;
                if (e >= P.m) e -= P.m;
            }
            out[((int64_t)o * M2 + j) * N + i] = radix_twist(s, P, j, i);
        }
    }
}

// One thread per i: v_j = beta_j^-i u_j[i]; block q of u at [qN, qN + N) is
// sum_j V^-1[q][j] v_j, stored below n.
template <int M2>
__global__ void __launch_bounds__(256) k_radix_unfold(const u32 *__restrict__ ut, u32 *__restrict__ c,
                                                      const RadixParams P) {
    const int64_t N = P.N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        u32 v[M2];
#pragma unroll
        for (int j = 0; j < M2; ++j) v[j] = radix_twist(__ldg(ut + (int64_t)j * N + i), P, j, (u32)i);
#pragma unroll
        for (int q = 0; q < M2; ++q) {
            const int64_t e = i + (int64_t)q * N;
            if (e >= P.n) break;
            u32 s = 0;
#pragma unroll
            for (int j = 0; j < M2; ++j) s = add_c(s, mul_c(v[j], P.vinv[q][j], P.p), P.p);
            c[e] = s;
        }
    }
}

static int elementwise_blocks(int64_t items) {
    const int64_t b = (items + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

template <int M2>
static cudaError_t launch_radix_t(bool fold, const u32 *a, const u32 *b, u32 *out, const RadixParams &P,
                                  cudaStream_t st) {
    if (fold) k_radix_fold<M2><<<elementwise_blocks(2 * P.N), 256, 0, st>>>(a, b, out, P);
    else k_radix_unfold<M2><<<elementwise_blocks(P.N), 256, 0, st>>>(a, out, P);
    return cudaGetLastError();
}

// fold: a, b -> out; unfold: a (the products) -> out (c).
static cudaError_t launch_radix(bool fold, const u32 *a, const u32 *b, u32 *out, const RadixParams &P,
                                cudaStream_t st) {
    switch (P.m2) {
#define PM_RADIX_CASE(M) \
    case M: return launch_radix_t<M>(fold, a, b, out, P, st);
        PM_RADIX_CASE(1)
        PM_RADIX_CASE(2)
        PM_RADIX_CASE(3)
        PM_RADIX_CASE(4)
        PM_RADIX_CASE(5)
        PM_RADIX_CASE(6)
        PM_RADIX_CASE(7)
        PM_RADIX_CASE(8)
        PM_RADIX_CASE(9)
        PM_RADIX_CASE(10)
        PM_RADIX_CASE(11)
        PM_RADIX_CASE(12)
        PM_RADIX_CASE(13)
        PM_RADIX_CASE(14)
        PM_RADIX_CASE(15)
#undef PM_RADIX_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ host side
// Twist tables per (device, p, m, k): w^(+-j i) split as lo[j][il] =
// w^(+-j il), hi[j][ih] = w^(+-j LO ih) with i = ih LO + il.  Resident until
// process exit, like the twiddle tables.
struct RadixTables {
    uint2 *fwd_lo = nullptr, *fwd_hi = nullptr, *inv_lo = nullptr, *inv_hi = nullptr;
    int lo_len = 0, hi_len = 0;
    u32 w = 0;
};

static std::mutex g_radix_mu;
static std::map<std::tuple<int, u32, int, int>, RadixTables> g_radix;

static int radix_tables(u32 p, u32 root, int m, int k, cudaStream_t st, RadixTables **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_radix_mu);
    auto key = std::make_tuple(dev, p, m, k);
    auto it = g_radix.find(key);
    if (it != g_radix.end()) {
        *out = &it->second;
        return POLY_OK;
    }
    RadixTables T;
    const int64_t N = (int64_t)1 << k;
    T.lo_len = (int)std::min<int64_t>(N, (int64_t)1 << radix::LO_BITS);
    T.hi_len = (int)(N / T.lo_len);
    const u64 L = (u64)m * (u64)N;
    T.w = h_powmod(root, (u64)(p - 1) / L, p);
    const u32 winv = h_invmod(T.w, p);
    std::vector<uint2> h((size_t)2 * m * (T.lo_len + T.hi_len));
    uint2 *flo = h.data(), *fhi = flo + (size_t)m * T.lo_len;
    uint2 *ilo = fhi + (size_t)m * T.hi_len, *ihi = ilo + (size_t)m * T.lo_len;
    for (int j = 0; j < m; ++j) {
        for (int dir = 0; dir < 2; ++dir) {
            const u32 wj = h_powmod(dir ? winv : T.w, (u64)j, p);
            uint2 *lo = (dir ? ilo : flo) + (size_t)j * T.lo_len, *hi = (dir ? ihi : fhi) + (size_t)j * T.hi_len;
            u64 x = 1;
            for (int il = 0; il < T.lo_len; ++il, x = x * wj % p) lo[il] = shoup_pair((u32)x, p);
            const u32 step = h_powmod(wj, (u64)T.lo_len, p);
            x = 1;
            for (int ih = 0; ih < T.hi_len; ++ih, x = x * step % p) hi[ih] = shoup_pair((u32)x, p);
        }
    }
    uint2 *d = nullptr;
    e = cudaMalloc((void **)&d, h.size() * sizeof(uint2));
    if (e != cudaSuccess) {
        cuda_fail(e, "radix twist tables");
        return POLY_ENOMEM;
    }
    e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(uint2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "radix twist tables upload");
    }
    T.fwd_lo = d;
    T.fwd_hi = d + (fhi - flo);
    T.inv_lo = d + (ilo - flo);
    T.inv_hi = d + (ihi - flo);
    *out = &g_radix.emplace(key, T).first->second;
    return POLY_OK;
}

// Inverse of V[j][q] = z^(jq) (j, q < r) mod p by Gauss-Jordan elimination.
static bool vandermonde_inverse(u32 z, int r, u32 p, u32 out[radix::MAXM][radix::MAXM]) {
    u64 A[radix::MAXM][2 * radix::MAXM];
    for (int j = 0; j < r; ++j) {
        const u32 zj = h_powmod(z, (u64)j, p);
        u64 x = 1;
        for (int q = 0; q < r; ++q, x = x * zj % p) A[j][q] = x;
        for (int q = 0; q < r; ++q) A[j][r + q] = (u64)(j == q);
    }
    for (int col = 0; col < r; ++col) {
        int piv = col;
        while (piv < r && A[piv][col] == 0) ++piv;
        if (piv == r) return false;  // not reached: the nodes zeta^j are distinct
        for (int q = 0; q < 2 * r; ++q) std::swap(A[col][q], A[piv][q]);
        const u64 inv = h_invmod((u32)A[col][col], p);
        for (int q = 0; q < 2 * r; ++q) A[col][q] = A[col][q] * inv % p;
        for (int i = 0; i < r; ++i) {
            if (i == col || A[i][col] == 0) continue;
            const u64 f = A[i][col];
            for (int q = 0; q < 2 * r; ++q) A[i][q] = (A[i][q] + (u64)(p - f) * A[col][q]) % p;
        }
    }
    for (int i = 0; i < r; ++i)
        for (int q = 0; q < r; ++q) out[i][q] = (u32)A[i][r + q];
    return true;
}

static int radix_product(u32 p, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int m, cudaStream_t st) {
    u32 root = 0;
    int rc = validate_prime(p, &root);
    if (rc) return rc;
    const int64_t n = za + zb - 1;
    int k = radix::MIN_LOG_N;
    while ((int64_t)m << k < n) ++k;
    if (k > radix::MAX_LOG_N || k > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    const int64_t N = (int64_t)1 << k;
    if ((p - 1) % (u32)m != 0) return POLY_EINVAL;
    if ((u64)(p - 1) % ((u64)m * (u64)N) != 0) return POLY_ETOO_LONG;
    const int m2 = (int)((n + N - 1) / N);
    RadixTables *T = nullptr;
    rc = radix_tables(p, root, m, k, st, &T);
    if (rc) return rc;
    AuxStreams *rs = nullptr;
    rc = aux_streams(&rs);
    if (rc) return rc;

    RadixParams P{};
    P.p = p;
    P.m = m;
    P.m2 = m2;
    P.k = k;
    P.N = N;
    P.z[0] = za;
    P.z[1] = zb;
    P.n = n;
    P.lo_len = T->lo_len;
    P.hi_len = T->hi_len;
    const u32 zeta = h_powmod(T->w, (u64)N, p);
    for (int e = 0; e < m; ++e) P.zpow[e] = shoup_pair(h_powmod(zeta, (u64)e, p), p);
    u32 vi[radix::MAXM][radix::MAXM];
    if (!vandermonde_inverse(zeta, m2, p, vi)) return POLY_EINVAL_PRIME;
    for (int q = 0; q < m2; ++q)
        for (int j = 0; j < m2; ++j) P.vinv[q][j] = shoup_pair(vi[q][j], p);

    u32 *ws = nullptr;  // twisted residues of a and b (2 m2 N words), their products (m2 N)
    cudaError_t e = cudaMallocAsync((void **)&ws, (size_t)3 * m2 * N * sizeof(u32), st);
    if (e != cudaSuccess) {
        cuda_fail(e, "radix workspace");
        return POLY_ENOMEM;
    }
    u32 *res = ws, *prod = ws + (size_t)2 * m2 * N;
    P.lo = T->fwd_lo;
    P.hi = T->fwd_hi;
    e = launch_radix(true, a, b, res, P, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "radix fold launch");
    if (rc == POLY_OK && (e = cudaEventRecord(rs->fork, st)) != cudaSuccess) rc = cuda_fail(e, "fork event");
    bool used[AUX_STREAMS] = {};
    for (int j = 0; j < m2 && rc == POLY_OK; ++j) {
        const int s = j % (AUX_STREAMS + 1);  // stream 0 = the caller's, then the auxiliary ones
        cudaStream_t sj = s == 0 ? st : rs->s[s - 1];
        if (s > 0 && !used[s - 1]) {
            if ((e = cudaStreamWaitEvent(sj, rs->fork, 0)) != cudaSuccess) {
                rc = cuda_fail(e, "fork wait");
                break;
            }
            used[s - 1] = true;
        }
        rc = run_product(p, 0, res + (size_t)j * N, N, res + (size_t)(m2 + j) * N, N, prod + (size_t)j * N, k, true,
                         sj, nullptr, N);
    }
    for (int s = 0; s < AUX_STREAMS && rc == POLY_OK; ++s) {
        if (!used[s]) continue;
        if ((e = cudaEventRecord(rs->join[s], rs->s[s])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, rs->join[s], 0)) != cudaSuccess)
            rc = cuda_fail(e, "join event");
    }
    if (rc == POLY_OK) {
        P.lo = T->inv_lo;
        P.hi = T->inv_hi;
        e = launch_radix(false, prod, nullptr, c, P, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "radix unfold launch");
    }
    e = cudaFreeAsync(ws, st);
    if (rc == POLY_OK && e != cudaSuccess) rc = cuda_fail(e, "radix workspace free");
    return rc;
}

}  // namespace pm

using namespace pm;

extern "C" int polymul_mod_radix_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                                       uint32_t *c, int m, void *stream) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0 || m < 1 || m > radix::MAXM || (m & 1) == 0) return POLY_EINVAL;
    if (m == 1) return polymul_mod_async(p, a, da, b, db, c, stream);
    if (validation_on()) {
        u32 root = 0;
        int rc = validate_prime(p, &root);
        if (!rc) rc = validate_coeffs(p, a, da + 1, b, db + 1, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return radix_product(p, a, da + 1, b, db + 1, c, m, (cudaStream_t)stream);
}
