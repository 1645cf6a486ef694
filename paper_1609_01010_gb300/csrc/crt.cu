// crt.cu -- exact integer product of polynomials with 32-bit coefficients
// through three modular products and the Chinese remainder theorem (the
// "three primes algorithm" that Section 1 names as the way integer
// multiplication rests on modular polynomial multiplication).
//
//   1. k_crt_reduce:  a_i mod q_j and b_i mod q_j for the three primes
//      q_0 = 469762049 (7 2^26 + 1), q_1 = 2013265921 (15 2^27 + 1),
//      q_2 = 754974721 (45 2^24 + 1) into three residue planes.
//   2. three TFT products (Section 3, Eq. 14), one per prime, by the same
//      kernels as polymul_mod_async, on three streams (forked from and
//      joined back into the caller's stream) so that they overlap.
//   3. k_crt_combine: Garner's mixed-radix reconstruction
//        x0 = u0,  x1 = (u1 - x0) q0^-1 mod q1,
//        x2 = (u2 - x0 - q0 x1) (q0 q1)^-1 mod q2,
//        c  = x0 + q0 x1 + q0 q1 x2  (0 <= c < q0 q1 q2 < 2^90),
//      written as three little-endian 32-bit words per coefficient.
// Every coefficient of the integer product is below min(za, zb) (2^32 - 1)^2
// <= 2^23 2^64 < q0 q1 q2 for n <= 2^24 (the largest L all three primes
// support), so the reconstruction is the exact integer.
#include <stdint.h>

#include <algorithm>

#include "host.h"
#include "polymul.h"

namespace pm {

namespace crt {
constexpr u32 Q0 = 469762049u;
constexpr u32 Q1 = 2013265921u;
constexpr u32 Q2 = 754974721u;
constexpr int MAX_LOG_N = 24;  // 2-adic order of q2 - 1
constexpr int UNROLL = 4;       // independent loads in flight per thread
}  // namespace crt

struct CrtConsts {
    uint2 q0inv_q1;    // Shoup pair of q0^-1 mod q1
    uint2 q0_q2;       // Shoup pair of q0 mod q2
    uint2 q01inv_q2;   // Shoup pair of (q0 q1)^-1 mod q2
    u64 q01;           // q0 q1
};

// Residues of the concatenated operands x = a ++ b (nx = za + zb words) into
// three planes r + j*plane.  Grid-stride with UNROLL coalesced loads issued
// before any store, so each thread keeps several HBM reads in flight.
__global__ void __launch_bounds__(256) k_crt_reduce(const u32 *__restrict__ a, int64_t za, const u32 *__restrict__ b,
                                                    int64_t nx, u32 *__restrict__ r, int64_t plane) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < nx; base += stride * crt::UNROLL) {
        u32 x[crt::UNROLL];
#pragma unroll
        for (int u = 0; u < crt::UNROLL; ++u) {
            const int64_t i = base + u * stride;
            x[u] = i < nx ? (i < za ? __ldg(a + i) : __ldg(b + (i - za))) : 0u;
        }
#pragma unroll
        for (int u = 0; u < crt::UNROLL; ++u) {
            const int64_t i = base + u * stride;
            if (i < nx) {
                r[i] = x[u] % crt::Q0;
                r[plane + i] = x[u] % crt::Q1;
                r[2 * plane + i] = x[u] % crt::Q2;
            }
        }
    }
}

// c_k from its residues u0 (mod q0), u1 (mod q1), u2 (mod q2), all canonical.
__device__ __forceinline__ void garner(u32 u0, u32 u1, u32 u2, const CrtConsts &k, u32 *w) {
    const u32 x0 = u0;                                        // < q0 < q1, q2
    const u32 x1 = mul_c(u1 + crt::Q1 - x0, k.q0inv_q1, crt::Q1);  // u1 - x0 + q1 < 2 q1 < 2^32
    const u32 s = add_c(x0, mul_c(x1, k.q0_q2, crt::Q2), crt::Q2);  // (x0 + q0 x1) mod q2
    const u32 x2 = mul_c(sub_c(u2, s, crt::Q2), k.q01inv_q2, crt::Q2);
    const u64 y = (u64)x0 + (u64)crt::Q0 * x1;                // < q0 q1 < 2^60
    const u64 lo = k.q01 * (u64)x2;
    const u64 hi = __umul64hi(k.q01, (u64)x2);                // q0 q1 x2 < 2^90
    const u64 sum = lo + y;
    w[0] = (u32)sum;
    w[1] = (u32)(sum >> 32);
    w[2] = (u32)(hi + (sum < lo ? 1u : 0u));
}

__global__ void __launch_bounds__(256) k_crt_combine(const u32 *__restrict__ u, int64_t plane, int64_t n,
                                                     u32 *__restrict__ c, CrtConsts k) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += stride * crt::UNROLL) {
        u32 v[crt::UNROLL][3];
#pragma unroll
        for (int q = 0; q < crt::UNROLL; ++q) {
            const int64_t i = base + q * stride;
#pragma unroll
            for (int j = 0; j < 3; ++j) v[q][j] = i < n ? __ldg(u + j * plane + i) : 0u;
        }
#pragma unroll
        for (int q = 0; q < crt::UNROLL; ++q) {
            const int64_t i = base + q * stride;
            if (i < n) {
                u32 w[3];
                garner(v[q][0], v[q][1], v[q][2], k, w);
                c[3 * i] = w[0];
                c[3 * i + 1] = w[1];
                c[3 * i + 2] = w[2];
            }
        }
    }
}

static CrtConsts crt_consts() {
    CrtConsts k;
    k.q0inv_q1 = shoup_pair(h_invmod(crt::Q0 % crt::Q1, crt::Q1), crt::Q1);
    k.q0_q2 = shoup_pair(crt::Q0 % crt::Q2, crt::Q2);
    const u32 q01_mod_q2 = (u32)(((u64)crt::Q0 * crt::Q1) % crt::Q2);
    k.q01inv_q2 = shoup_pair(h_invmod(q01_mod_q2, crt::Q2), crt::Q2);
    k.q01 = (u64)crt::Q0 * crt::Q1;
    return k;
}

// Grid of the two element-wise kernels: enough CTAs for every SM several
// times over, never more than the work needs.
static int elementwise_grid(int64_t items) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            sms = 148;
    }
    const int64_t need = (items + 256 * crt::UNROLL - 1) / (256 * crt::UNROLL);
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

static int crt3(const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, cudaStream_t st) {
    AuxStreams *cs = nullptr;  // the products mod q1 and q2 run on cs->s[0], cs->s[1]
    int rs = aux_streams(&cs);
    if (rs) return rs;
    const int64_t n = za + zb - 1;
    const int l = ceil_log2(n);
    const int64_t nx = za + zb;
    const int64_t plane = std::max(nx, n);
    // residue planes of the operands (3 x nx) and of the three products (3 x n)
    u32 *ws = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&ws, (size_t)(3 * plane + 3 * n) * sizeof(u32), st);
    if (e != cudaSuccess) {
        cuda_fail(e, "three-primes workspace");
        return POLY_ENOMEM;
    }
    u32 *res = ws, *prod = ws + 3 * plane;
    int rc = POLY_OK;
    k_crt_reduce<<<elementwise_grid(nx), 256, 0, st>>>(a, za, b, nx, res, plane);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "residue launch");
    const u32 primes[3] = {crt::Q0, crt::Q1, crt::Q2};
    if (rc == POLY_OK && (e = cudaEventRecord(cs->fork, st)) != cudaSuccess) rc = cuda_fail(e, "fork event");
    for (int j = 0; j < 3 && rc == POLY_OK; ++j) {
        cudaStream_t sj = j == 0 ? st : cs->s[j - 1];
        if (j > 0 && (e = cudaStreamWaitEvent(sj, cs->fork, 0)) != cudaSuccess) {
            rc = cuda_fail(e, "fork wait");
            break;
        }
        const u32 *rj = res + j * plane;
        rc = run_product(primes[j], 0, rj, za, rj + za, zb, prod + j * n, l, true, sj, nullptr);
        if (rc == POLY_OK && j > 0) {
            if ((e = cudaEventRecord(cs->join[j - 1], sj)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, cs->join[j - 1], 0)) != cudaSuccess)
                rc = cuda_fail(e, "join event");
        }
    }
    if (rc == POLY_OK) {
        k_crt_combine<<<elementwise_grid(n), 256, 0, st>>>(prod, n, n, c, crt_consts());
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "CRT launch");
    }
    e = cudaFreeAsync(ws, st);
    if (rc == POLY_OK && e != cudaSuccess) rc = cuda_fail(e, "three-primes workspace free");
    return rc;
}

}  // namespace pm

using namespace pm;

extern "C" int polymul_crt3_async(const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                                  void *stream) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    if (ceil_log2(n) > crt::MAX_LOG_N) return POLY_ETOO_LONG;
    return crt3(a, za, b, zb, c, (cudaStream_t)stream);
}
