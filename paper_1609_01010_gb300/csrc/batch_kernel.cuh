// batch_kernel.cuh -- the persistent batched kernel (see batch.cu for the
// work-list protocol).
#pragma once
#include <map>
#include <mutex>

#include "batch.h"
#include "bodies.cuh"
#include "polymul.h"

namespace pm {

__device__ __forceinline__ bool wait_count(const int *ctr, int target, int *status, long long limit) {
    long long it = 0;
    while (*(volatile const int *)ctr < target) {
        if (++it > limit) {
            atomicExch(status, POLY_ETIMEOUT);
            return false;
        }
        __nanosleep(128);
    }
    __threadfence();
    return true;
}

// Column items of a product run at its own tile width (8 .. 2048 words).
// CW != 0: every product of the launch has width CW (no dispatch); CW = 0:
// the width is read per product.
template <class A, int CW>
__device__ __forceinline__ void colf_body_w(int C, const LargeDesc &d, int tile, int opnd, ModParams m, TwTables tw) {
    if constexpr (CW != 0) {
        colf_body<A, CW>(d, tile, opnd, m, tw);
    } else {
        if (C == 2048) colf_body<A, 2048>(d, tile, opnd, m, tw);
        else if (C == 1024) colf_body<A, 1024>(d, tile, opnd, m, tw);
        else if (C == 512) colf_body<A, 512>(d, tile, opnd, m, tw);
        else if (C == 256) colf_body<A, 256>(d, tile, opnd, m, tw);
        else if (C == 128) colf_body<A, 128>(d, tile, opnd, m, tw);
        else if (C == 32) colf_body<A, 32>(d, tile, opnd, m, tw);
        else colf_body<A, 8>(d, tile, opnd, m, tw);
    }
}
template <class A, int CW>
__device__ __forceinline__ void coli_body_w(int C, const LargeDesc &d, int tile, ModParams m, TwTables tw) {
    if constexpr (CW != 0) {
        coli_body<A, CW>(d, tile, m, tw);
    } else {
        if (C == 2048) coli_body<A, 2048>(d, tile, m, tw);
        else if (C == 1024) coli_body<A, 1024>(d, tile, m, tw);
        else if (C == 512) coli_body<A, 512>(d, tile, m, tw);
        else if (C == 256) coli_body<A, 256>(d, tile, m, tw);
        else if (C == 128) coli_body<A, 128>(d, tile, m, tw);
        else if (C == 32) coli_body<A, 32>(d, tile, m, tw);
        else coli_body<A, 8>(d, tile, m, tw);
    }
}

template <class A, int CW>
// Three resident CTAs per SM (at most 85 registers a thread; the largest
// item's shared memory, 64 KB for a 16-row one-CTA product, allows three):
// the items' barrier and load waits are latency-bound, and the extra CTA per
// SM made the 4096-product batch 21 % faster than two CTAs, although the
// one-CTA product bodies then spill a few hundred bytes to local memory.
__global__ void __launch_bounds__(BATCH_THREADS, 3) k_batch(BatchParams P) {
    __shared__ int s_item, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= P.nitems) break;
        const WorkItem w = P.items[it];
        const BatchDesc bd = P.descs[w.prod];
        if (threadIdx.x == 0) {
            bool ok = true;
            if (w.kind == IT_ROW)
                ok = wait_count(P.counters + 2 * w.prod, 2 * (int)(bd.g.S / bd.C), P.status, P.spin_limit);
            else if (w.kind == IT_COLI)
                ok = wait_count(P.counters + 2 * w.prod + 1, (int)bd.g.k, P.status, P.spin_limit);
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            const u32 *pa = (const u32 *)((uintptr_t)P.a + bd.a_off);
            const u32 *pb = (const u32 *)((uintptr_t)P.b + bd.b_off);
            u32 *pc = (u32 *)((uintptr_t)P.c + bd.c_off);
            if (w.kind == IT_SMALL) {
                SmallDesc d;
                d.a = pa;
                d.b = pb;
                d.c = pc;
                d.za = bd.za;
                d.zb = bd.zb;
                d.n = bd.n;
                d.logT = bd.logT;
                d.k = bd.k;
                d.steps = bd.steps;
                d.nsteps = bd.nsteps;
                d.prune = 1;
                small_dispatch<A>(d, P.m, P.tw);
            } else {
                LargeDesc d;
                d.a = pa;
                d.b = pb;
                d.c = pc;
                d.wa = (u32 *)((uintptr_t)P.ws + bd.ws_off);
                d.wb = d.wa + bd.g.k * bd.g.S;
                d.za = bd.za;
                d.zb = bd.zb;
                d.n = bd.n;
                d.g = bd.g;
                d.steps = bd.steps;
                d.nsteps = bd.nsteps;
                d.prune = 1;
                if (w.kind == IT_COLF) colf_body_w<A, CW>(bd.C, d, w.idx, w.opnd, P.m, P.tw);
                else if (w.kind == IT_ROW) row_body_ool<A, BATCH_SIGMA>(d, (u32)w.idx, P.m, P.tw);
                else coli_body_w<A, CW>(bd.C, d, w.idx, P.m, P.tw);
            }
        }
        __threadfence();  // each thread's outputs visible device-wide before the signal
        __syncthreads();
        if (threadIdx.x == 0 && (w.kind == IT_COLF || w.kind == IT_ROW))
            atomicAdd(P.counters + 2 * w.prod + (w.kind == IT_ROW ? 1 : 0), 1);
    }
}

template <class A, int CW>
static cudaError_t launch_batch_cw(const BatchParams &P, size_t smem, int *grid_out, cudaStream_t st) {
    static std::mutex mu;
    static std::map<int, int> occ;  // device -> blocks per SM
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find(dev);
        if (it == occ.end()) {
            e = cudaFuncSetAttribute(k_batch<A, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)BATCH_SMEM_MAX);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<A, CW>, BATCH_THREADS,
                                                              BATCH_SMEM_MAX);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) per_sm = 1;
            occ[dev] = per_sm;
        } else {
            per_sm = it->second;
        }
    }
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = per_sm * sms;
    if (grid > P.nitems) grid = P.nitems;
    if (grid < 1) grid = 1;
    *grid_out = grid;
    k_batch<A, CW><<<grid, BATCH_THREADS, smem, st>>>(P);
    return cudaGetLastError();
}

// uniform_C: the one column-tile width of every large product of the launch
// (any width when there is no large product), or 0 when the widths differ;
// widths 8, 32 and 128 have a kernel of their own, the others dispatch.
template <class A>
static cudaError_t launch_batch_t(int uniform_C, const BatchParams &P, size_t smem, int *grid_out, cudaStream_t st) {
    switch (uniform_C) {
        case 8: return launch_batch_cw<A, 8>(P, smem, grid_out, st);
        case 32: return launch_batch_cw<A, 32>(P, smem, grid_out, st);
        case 128: return launch_batch_cw<A, 128>(P, smem, grid_out, st);
        default: return launch_batch_cw<A, 0>(P, smem, grid_out, st);
    }
}

}  // namespace pm
