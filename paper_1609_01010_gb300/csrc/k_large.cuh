// k_large.cu -- the three-kernel path for transform lengths L >= 16384.
//
// L = T * S with rows of S = 2^sigma words (sigma = 9..13) and T <= 2048.
//   k_col_fwd   grid (S/C, 2): column stage of TFT(a) and TFT(b) on tiles of
//               C columns, pruned to the input support and to the k needed
//               rows; writes rows [0, k) of each operand to the workspace.
//   k_row_fused grid (k):      one CTA per needed row: remaining sigma levels
//               of both operands, pointwise product with the scale folded in,
//               unscaled inverse of the sigma levels; overwrites wa's row.
//   k_col_itft  grid (S/C):    ITFT column stage from the step list, then
//               the first n outputs reduced to [0, p).
// Each kernel reads its inputs once from HBM/L2 and writes its outputs once.
#pragma once
#include "bodies.cuh"

namespace pm {

constexpr int COL_THREADS = 256;
constexpr size_t COL_SMEM_MAX = 160 * 1024;  // T * C * 4 bytes (schedule_valid's bound)

template <class A, int C>
__global__ void __launch_bounds__(COL_THREADS) k_col_fwd(const LargeDesc d, ModParams m, TwTables tw) {
    colf_body<A, C>(d, blockIdx.x, blockIdx.y, m, tw);
}

template <class A, int SIGMA>
__global__ void __launch_bounds__((1 << SIGMA) / 16) k_row_fused(const LargeDesc d, ModParams m, TwTables tw) {
    row_body<A, SIGMA>(d, blockIdx.x, m, tw);
}

template <class A, int C>
__global__ void __launch_bounds__(COL_THREADS) k_col_itft(const LargeDesc d, ModParams m, TwTables tw) {
    coli_body<A, C>(d, blockIdx.x, m, tw);
}

// ------------------------------------------------------------ launchers

template <class A, int C>
static cudaError_t launch_cols(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    const size_t smem = (size_t)d.g.T * C * sizeof(u32);
    cudaError_t e = ensure_smem(k_col_fwd<A, C>, COL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    e = ensure_smem(k_col_itft<A, C>, COL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    const int tiles = (int)(d.g.S / C);
    k_col_fwd<A, C><<<dim3(tiles, 2), COL_THREADS, smem, st>>>(d, m, tw);
    return cudaGetLastError();
}

template <class A, int C>
static cudaError_t launch_cols_inv(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    const size_t smem = (size_t)d.g.T * C * sizeof(u32);
    const int tiles = (int)(d.g.S / C);
    k_col_itft<A, C><<<tiles, COL_THREADS, smem, st>>>(d, m, tw);
    return cudaGetLastError();
}

template <class A, int SIGMA>
static cudaError_t launch_rows(const LargeDesc &d, ModParams m, TwTables tw, cudaStream_t st) {
    constexpr int S = 1 << SIGMA;
    const size_t smem = (size_t)4 * S * sizeof(u32);
    cudaError_t e = ensure_smem(k_row_fused<A, SIGMA>, smem);
    if (e != cudaSuccess) return e;
    k_row_fused<A, SIGMA><<<(int)d.g.k, S / 16, smem, st>>>(d, m, tw);
    return cudaGetLastError();
}

template <class A>
static cudaError_t launch_large_t(const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                                  cudaEvent_t *ev) {
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], st);
    switch (sch.C) {
        case 8: e = launch_cols<A, 8>(d, m, tw, st); break;
        case 16: e = launch_cols<A, 16>(d, m, tw, st); break;
        case 32: e = launch_cols<A, 32>(d, m, tw, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    switch (d.g.sigma) {
        case 9: e = launch_rows<A, 9>(d, m, tw, st); break;
        case 10: e = launch_rows<A, 10>(d, m, tw, st); break;
        case 11: e = launch_rows<A, 11>(d, m, tw, st); break;
        case 12: e = launch_rows<A, 12>(d, m, tw, st); break;
        case 13: e = launch_rows<A, 13>(d, m, tw, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    switch (sch.C) {
        case 8: e = launch_cols_inv<A, 8>(d, m, tw, st); break;
        case 16: e = launch_cols_inv<A, 16>(d, m, tw, st); break;
        default: e = launch_cols_inv<A, 32>(d, m, tw, st); break;
    }
    if (ev) cudaEventRecord(ev[3], st);
    return e;
}

}  // namespace pm
