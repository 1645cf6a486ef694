// conv.cu -- cyclic and negacyclic convolutions of length N (C-ABI).
//
// Cyclic: c = a * b mod (x^N - 1), the circular convolution of Definition 4
// (Eq. 5), computed as Eq. 11 does: when N is a power of two the product
// kernels run with L = N and all N outputs (n = L, no truncation), which is
// the full transform, pointwise product and inverse of the convolution
// theorem (Eq. 8-10).  Negacyclic: c = a * b mod (x^N + 1), the other factor
// of Eq. 13.  Every other case (N not a power of two, N < 512, and every
// negacyclic N) computes the linear product u (TFT path) into a workspace
// and folds it: c_i = u_i + u_{i+N} (cyclic) or u_i - u_{i+N} (negacyclic);
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

static int conv_check(const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, const uint32_t *c, int64_t N) {
    if (!a || !b || !c) return POLY_ENULL;
    if (N < 1 || za < 1 || zb < 1 || za > N || zb > N) return POLY_EINVAL;
    return POLY_OK;
}

}  // namespace pm

using namespace pm;

extern "C" {

int polymul_cyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, uint32_t *c,
                         int64_t N, void *stream) {
    int rc = conv_check(a, za, b, zb, c, N);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int l = ceil_log2(N);
    if (((int64_t)1 << l) == N && l >= SMALL_LOG_S) {
        if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
        return run_product(p, 0, a, za, b, zb, c, l, true, st, nullptr, N);
    }
    return conv_fold(p, a, za, b, zb, c, N, false, st);
}

int polymul_negacyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, uint32_t *c,
                             int64_t N, void *stream) {
    int rc = conv_check(a, za, b, zb, c, N);
    if (rc) return rc;
    return conv_fold(p, a, za, b, zb, c, N, true, (cudaStream_t)stream);
}

}  // extern "C"
