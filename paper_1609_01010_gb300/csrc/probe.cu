// probe.cu -- measured integer-pipe peaks of this GPU (a diagnostic entry
// point: the roofline denominator of the transform kernels).
//
// Each probe kernel runs a long register-only loop of one operation on 16
// independent accumulators per thread, at the occupancy the hardware allows,
// with no memory traffic inside the loop; the result is written once so the
// loop cannot be removed.  Kinds:
//   0  the forward (Cooley-Tukey) butterfly of the lazy regime, Arith<true>::ct
//      (the instruction mix the transform kernels execute: 3 multiplies and
//      the add/subtract/min of Harvey's butterfly);
//   1  the inverse (Gentleman-Sande) butterfly of the lazy regime, Arith<true>::gs;
//   2  32-bit multiply, low word (mul.lo.u32);
//   3  32-bit multiply, high word (mul.hi.u32);
//   4  32-bit add (add.u32);
//   5  32-bit unsigned minimum (min.u32).
// polymul_probe_int reports operations per second, one operation being one
// butterfly (kinds 0, 1) or one instruction of the named kind (kinds 2..5).
#include <cuda_runtime.h>
#include <stdint.h>

#include "host.h"
#include "modarith.cuh"
#include "polymul.h"

namespace pm {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_ACC = 16;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_int(u32 *out, u32 seed, int iters, u32 p, uint2 w) {
    u32 x[PROBE_ACC];
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < PROBE_ACC; ++i) x[i] = (seed ^ (t * 0x9E3779B9u + i * 0x85EBCA6Bu)) % p;
    const u32 c = seed | 1u;
    for (int it = 0; it < iters; ++it) {
        if constexpr (KIND == 0) {
#pragma unroll
            for (int i = 0; i < PROBE_ACC / 2; ++i) Arith<true>::ct(x[i], x[i + PROBE_ACC / 2], w, p);
        } else if constexpr (KIND == 1) {
#pragma unroll
            for (int i = 0; i < PROBE_ACC / 2; ++i) Arith<true>::gs(x[i], x[i + PROBE_ACC / 2], w, p);
        } else if constexpr (KIND == 2) {
#pragma unroll
            for (int i = 0; i < PROBE_ACC; ++i) asm volatile("mul.lo.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(c));
        } else if constexpr (KIND == 3) {
#pragma unroll
            for (int i = 0; i < PROBE_ACC; ++i) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(c));
        } else if constexpr (KIND == 4) {
#pragma unroll
            for (int i = 0; i < PROBE_ACC; ++i) asm volatile("add.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(c));
        } else {
#pragma unroll
            for (int i = 0; i < PROBE_ACC; ++i) asm volatile("min.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(c + i));
        }
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < PROBE_ACC; ++i) acc ^= x[i];
    out[t] = acc;
}

template <int KIND>
static cudaError_t run_probe(int iters, double *ops_per_s, double *ms_out) {
    const u32 p = 469762049u;
    const uint2 w = shoup_pair(h_powmod(3, (p - 1) >> 12, p), p);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_int<KIND>, PROBE_THREADS, 0);
    if (e != cudaSuccess) return e;
    const int grid = sms * (per_sm < 1 ? 1 : per_sm);
    u32 *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, (size_t)grid * PROBE_THREADS * sizeof(u32));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0;
    if (e == cudaSuccess) {
        k_probe_int<KIND><<<grid, PROBE_THREADS, 0, st>>>(out, 12345u, iters / 8 + 1, p, w);  // warm-up
        cudaEventRecord(e0, st);
        k_probe_int<KIND><<<grid, PROBE_THREADS, 0, st>>>(out, 54321u, iters, p, w);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess) {
        const double per_iter = (KIND <= 1) ? PROBE_ACC / 2 : PROBE_ACC;
        *ops_per_s = (double)grid * PROBE_THREADS * iters * per_iter / (ms * 1e-3);
        *ms_out = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return e;
}

}  // namespace pm

using namespace pm;

extern "C" int polymul_probe_int(int kind, int iters, double *ops_per_s, double *ms) {
    if (!ops_per_s || !ms) return POLY_ENULL;
    if (iters < 1 || iters > (1 << 24)) return POLY_EINVAL;
    cudaError_t e;
    switch (kind) {
        case 0: e = run_probe<0>(iters, ops_per_s, ms); break;
        case 1: e = run_probe<1>(iters, ops_per_s, ms); break;
        case 2: e = run_probe<2>(iters, ops_per_s, ms); break;
        case 3: e = run_probe<3>(iters, ops_per_s, ms); break;
        case 4: e = run_probe<4>(iters, ops_per_s, ms); break;
        case 5: e = run_probe<5>(iters, ops_per_s, ms); break;
        default: return POLY_EINVAL;
    }
    return e == cudaSuccess ? POLY_OK : cuda_fail(e, "integer probe");
}
