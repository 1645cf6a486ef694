// batch.cu -- many independent products of uneven sizes in ONE persistent
// kernel launch, replayed from a CUDA graph.
//
// The batch is a device work list.  A product with L <= 8192 is one item
// (the whole one-CTA product); a larger product is 2*S/C column-stage items,
// k row items and S/C ITFT column items (the three kernels of k_large.cu).
// CTAs of the persistent kernel take items in list order from an atomic
// counter.  A row item waits until all column items of its product are done,
// an ITFT column item until all its rows are done; the list puts every item
// after the items it waits for, so an item only ever waits for items already
// taken by running CTAs and the launch cannot deadlock, whatever the number
// of resident CTAs.  Waits are bounded: on expiry the kernel records
// POLY_ETIMEOUT, skips the item and still signals it.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch.h"
#include "bodies.cuh"
#include "polymul.h"

namespace pm {

// ------------------------------------------------------------ host side
// Size the work list of `count` products.  `ptr_a/b/c[i]` are byte offsets
// (from the exec-time base pointers) of product i's operands and output.
int build_worklist(PrimeCtx *ctx, int64_t count, const int64_t *za, const int64_t *zb, const uint64_t *a_off,
                   const uint64_t *b_off, const uint64_t *c_off, std::vector<BatchDesc> &descs,
                   std::vector<WorkItem> &items, uint64_t *ws_bytes, size_t *smem_bytes) {
    descs.assign(count, BatchDesc{});
    items.clear();
    uint64_t ws = 0;
    size_t smem = 0;
    std::vector<std::pair<int64_t, int64_t>> small, large;  // (n, index)
    for (int64_t i = 0; i < count; ++i) {
        BatchDesc &d = descs[i];
        d.a_off = a_off[i];
        d.b_off = b_off[i];
        d.c_off = c_off[i];
        d.za = za[i];
        d.zb = zb[i];
        d.n = za[i] + zb[i] - 1;
        const int l = ceil_log2(d.n);
        if (l <= SMALL_MAX_LOG_L) {
            SmallDesc sd;
            int rc = prepare_small(ctx, nullptr, d.za, nullptr, d.zb, nullptr, l, true, &sd);
            if (rc) return rc;
            d.large = 0;
            d.logT = sd.logT;
            d.k = sd.k;
            d.steps = sd.steps;
            d.nsteps = sd.nsteps;
            const size_t sm = (size_t)2 * ((size_t)1 << sd.logT) * (1 << SMALL_LOG_S) * 4;
            smem = std::max(smem, sm);
            small.push_back({d.n, i});
        } else {
            if (l - BATCH_SIGMA > LARGE_MAX_LOG_T) return POLY_ETOO_LONG;
            const int C = batch_width_for(l);
            Schedule sch{BATCH_SIGMA, C};
            LargeDesc ld;
            int rc = prepare_large(ctx, nullptr, d.za, nullptr, d.zb, nullptr, l, true, sch, &ld);
            if (rc) return rc;
            d.large = 1;
            d.C = C;
            d.g = ld.g;
            d.steps = ld.steps;
            d.nsteps = ld.nsteps;
            d.ws_off = ws;
            ws += (uint64_t)2 * ld.g.k * ld.g.S * 4;
            smem = std::max(smem, (size_t)ld.g.T * C * 4);
            smem = std::max(smem, row_smem_bytes(BATCH_SIGMA));
            large.push_back({d.n, i});
        }
    }
    std::sort(small.begin(), small.end(), [](auto &x, auto &y) { return x.first > y.first; });
    std::sort(large.begin(), large.end(), [](auto &x, auto &y) { return x.first > y.first; });
    for (auto &pr : large) {
        const BatchDesc &d = descs[pr.second];
        const int tiles = (int)(d.g.S / d.C);
        for (int opnd = 0; opnd < 2; ++opnd)
            for (int t = 0; t < tiles; ++t) items.push_back(WorkItem{IT_COLF, (int32_t)pr.second, t, opnd});
    }
    for (auto &pr : small) items.push_back(WorkItem{IT_SMALL, (int32_t)pr.second, 0, 0});
    for (auto &pr : large) {
        const BatchDesc &d = descs[pr.second];
        for (int64_t r = 0; r < d.g.k; ++r) items.push_back(WorkItem{IT_ROW, (int32_t)pr.second, (int32_t)r, 0});
    }
    for (auto &pr : large) {
        const BatchDesc &d = descs[pr.second];
        const int tiles = (int)(d.g.S / d.C);
        for (int t = 0; t < tiles; ++t) items.push_back(WorkItem{IT_COLI, (int32_t)pr.second, t, 0});
    }
    *ws_bytes = ws;
    *smem_bytes = smem;
    return POLY_OK;
}

int uniform_width(const std::vector<BatchDesc> &descs) {
    int c = 0;
    for (const BatchDesc &d : descs) {
        if (!d.large) continue;
        if (c && d.C != c) return 0;
        c = d.C;
    }
    return c ? c : 128;
}

// Built-in rule: the widest column tile (of 8, 32, 128, 256, 512, 1024 or
// 2048 columns)
// whose T * C words fit the batched kernel's 64 KB of shared memory.  A
// column item's fixed cost (fetching it, its dependency check, its fence and
// barriers) is then spread over as many words as the shared memory allows:
// a product of L = 2^14 (4 rows of 4096) has 2 + 4 + 1 items instead of
// 64 + 4 + 32 with 128-column tiles.
int batch_width_default(int l) {
    for (int C : {2048, 1024, 512, 256, 128, 32, 8})
        if (batch_width_valid(l, C)) return C;
    return 8;
}

bool batch_width_valid(int l, int C) {
    const int t = l - BATCH_SIGMA;
    if (C != 8 && C != 32 && C != 128 && C != 256 && C != 512 && C != 1024 && C != 2048) return false;
    if (t < 1 || t > LARGE_MAX_LOG_T) return false;
    return ((size_t)C << t) * 4 <= BATCH_SMEM_MAX;
}

static std::mutex g_bw_mu;
static std::map<int, int> g_bw;  // tuned widths, by log2 L

int batch_width_for(int l) {
    {
        std::lock_guard<std::mutex> lk(g_bw_mu);
        auto it = g_bw.find(l);
        if (it != g_bw.end() && batch_width_valid(l, it->second)) return it->second;
    }
    return batch_width_default(l);
}

void set_batch_width(int l, int C) {
    std::lock_guard<std::mutex> lk(g_bw_mu);
    g_bw[l] = C;
}

std::map<int, int> all_batch_widths() {
    std::lock_guard<std::mutex> lk(g_bw_mu);
    return g_bw;
}

}  // namespace pm

using namespace pm;

struct polymul_batch {
    uint32_t p;
    int64_t count;
    PrimeCtx *ctx;
    size_t smem;
    std::vector<BatchDesc> h_descs;
    std::vector<WorkItem> h_items;
    BatchDesc *descs = nullptr;
    WorkItem *items = nullptr;
    int *ctrl = nullptr;  // counters[2*count], head, status
    u32 *ws = nullptr;
    uint64_t ws_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t last = nullptr;
    std::map<std::tuple<uintptr_t, uintptr_t, uintptr_t, uintptr_t>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
    int grid = 0;
    long long spin_limit = BATCH_SPIN_LIMIT;
    int withheld = 0;  // items dropped by polymul_batch_test_withhold
    int64_t a_words = 0, b_words = 0;  // extent of the packed operands (validation)
    int uniform_C = 0;                 // see uniform_width
};

static void batch_free(polymul_batch *b) {
    if (!b) return;
    for (auto &kv : b->graphs) {
        if (kv.second.second) cudaGraphExecDestroy(kv.second.second);
        if (kv.second.first) cudaGraphDestroy(kv.second.first);
    }
    if (b->descs) cudaFree(b->descs);
    if (b->items) cudaFree(b->items);
    if (b->ctrl) cudaFree(b->ctrl);
    if (b->ws) cudaFree(b->ws);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->last) cudaEventDestroy(b->last);
    delete b;
}

extern "C" {

int polymul_batch_create(uint32_t p, int64_t count, const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                         polymul_batch **out) {
    if (!out || !a_off || !b_off || !c_off) return POLY_ENULL;
    *out = nullptr;
    if (count < 1 || count > (1 << 24)) return POLY_EINVAL;
    std::vector<int64_t> za(count), zb(count);
    std::vector<uint64_t> ao(count), bo(count), co(count);
    int max_l = 0;
    for (int64_t i = 0; i < count; ++i) {
        za[i] = a_off[i + 1] - a_off[i];
        zb[i] = b_off[i + 1] - b_off[i];
        if (za[i] < 1 || zb[i] < 1 || a_off[i] < 0 || b_off[i] < 0 || c_off[i] < 0) return POLY_EINVAL;
        if (c_off[i + 1] - c_off[i] < za[i] + zb[i] - 1) return POLY_EINVAL;
        ao[i] = (uint64_t)a_off[i] * 4;
        bo[i] = (uint64_t)b_off[i] * 4;
        co[i] = (uint64_t)c_off[i] * 4;
        max_l = std::max(max_l, ceil_log2(za[i] + zb[i] - 1));
    }
    if (max_l > BATCH_SIGMA + LARGE_MAX_LOG_T) return POLY_ETOO_LONG;
    PrimeCtx *ctx = nullptr;
    int rc = get_prime(p, 0, std::max(max_l, SMALL_LOG_S), &ctx, nullptr);
    if (rc) return rc;
    polymul_batch *b = new polymul_batch();
    b->p = p;
    b->count = count;
    for (int64_t i = 0; i < count; ++i) {
        b->a_words = std::max(b->a_words, a_off[i + 1]);
        b->b_words = std::max(b->b_words, b_off[i + 1]);
    }
    b->ctx = ctx;
    rc = build_worklist(ctx, count, za.data(), zb.data(), ao.data(), bo.data(), co.data(), b->h_descs,
                        b->h_items, &b->ws_bytes, &b->smem);
    if (rc) {
        batch_free(b);
        return rc;
    }
    b->uniform_C = uniform_width(b->h_descs);
    if (b->smem > BATCH_SMEM_MAX) {
        batch_free(b);
        return POLY_ETOO_LONG;
    }
    bool ok = cudaMalloc(&b->descs, b->h_descs.size() * sizeof(BatchDesc)) == cudaSuccess &&
              cudaMalloc(&b->items, b->h_items.size() * sizeof(WorkItem)) == cudaSuccess &&
              cudaMalloc(&b->ctrl, (2 * count + 2) * sizeof(int)) == cudaSuccess &&
              (b->ws_bytes == 0 || cudaMalloc(&b->ws, b->ws_bytes) == cudaSuccess);
    if (!ok) {
        batch_free(b);
        return POLY_ENOMEM;
    }
    ok = cudaMemcpy(b->descs, b->h_descs.data(), b->h_descs.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(b->items, b->h_items.data(), b->h_items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemset(b->ctrl, 0, (2 * count + 2) * sizeof(int)) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        batch_free(b);
        return POLY_ECUDA;
    }
    *out = b;
    return POLY_OK;
}

static BatchParams batch_params(polymul_batch *b, const uint32_t *a, const uint32_t *bb, uint32_t *c) {
    BatchParams P;
    P.a = a;
    P.b = bb;
    P.c = c;
    P.ws = b->ws;
    P.descs = b->descs;
    P.items = b->items;
    P.nitems = (int)b->h_items.size() - b->withheld;
    P.counters = b->ctrl;
    P.head = b->ctrl + 2 * b->count;
    P.status = b->ctrl + 2 * b->count + 1;
    P.m = b->ctx->m;
    P.tw = b->ctx->tw;
    P.spin_limit = b->spin_limit;
    return P;
}

static int batch_enqueue(polymul_batch *b, const uint32_t *a, const uint32_t *bb, uint32_t *c, cudaStream_t st) {
    BatchParams P = batch_params(b, a, bb, c);
    if (cudaMemsetAsync(b->ctrl, 0, (2 * b->count + 2) * sizeof(int), st) != cudaSuccess) return POLY_ECUDA;
    return launch_batch(b->ctx->lazy, b->uniform_C, P, b->smem, &b->grid, st) == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

int polymul_batch_exec_nograph(polymul_batch *b, const uint32_t *a, const uint32_t *bb, uint32_t *c, void *stream) {
    if (!b || !a || !bb || !c) return POLY_ENULL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = validate_coeffs(b->p, a, b->a_words, bb, b->b_words, st);
    if (rc) return rc;
    rc = batch_enqueue(b, a, bb, c, st);
    if (rc) return rc;
    return cudaEventRecord(b->last, st) == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

int polymul_batch_exec(polymul_batch *b, const uint32_t *a, const uint32_t *bb, uint32_t *c, void *stream) {
    if (!b || !a || !bb || !c) return POLY_ENULL;
    cudaStream_t st = (cudaStream_t)stream;
    {
        int rc = validate_coeffs(b->p, a, b->a_words, bb, b->b_words, st);
        if (rc) return rc;
    }
    auto key = std::make_tuple((uintptr_t)a, (uintptr_t)bb, (uintptr_t)c, (uintptr_t)0);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        // Capture on the plan's private stream; the instantiated graph is then
        // launched on the caller's stream.
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return POLY_ECUDA;
        int rc = batch_enqueue(b, a, bb, c, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return POLY_ECUDA;
        if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return POLY_ECUDA;
        }
        it = b->graphs.emplace(key, std::make_pair(g, ge)).first;
    }
    if (cudaGraphLaunch(it->second.second, st) != cudaSuccess) return POLY_ECUDA;
    return cudaEventRecord(b->last, st) == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

int polymul_batch_status(polymul_batch *b) {
    if (!b) return POLY_ENULL;
    if (cudaEventSynchronize(b->last) != cudaSuccess) return POLY_ECUDA;
    int s = 0;
    if (cudaMemcpy(&s, b->ctrl + 2 * b->count + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return POLY_ECUDA;
    return s;
}

void polymul_batch_destroy(polymul_batch *b) {
    if (b && b->last) cudaEventSynchronize(b->last);
    batch_free(b);
}

int polymul_batch_test_withhold(polymul_batch *b, int kind, long long spin_limit) {
    if (!b) return POLY_ENULL;
    if (kind < 0) {  // restore
        b->spin_limit = BATCH_SPIN_LIMIT;
        b->withheld = 0;
        return cudaMemcpy(b->items, b->h_items.data(), b->h_items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice) == cudaSuccess
                   ? POLY_OK
                   : POLY_ECUDA;
    }
    // Drop the first item of `kind` from the device work list (the last item
    // moves into its place, so the list shrinks by one).
    std::vector<WorkItem> v = b->h_items;
    size_t i = 0;
    while (i < v.size() && v[i].kind != kind) ++i;
    if (i == v.size()) return POLY_EINVAL;
    v.erase(v.begin() + i);
    v.push_back(WorkItem{-1, 0, 0, 0});  // padding entry past nitems, never taken
    b->spin_limit = spin_limit;
    if (cudaMemcpy(b->items, v.data(), v.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return POLY_ECUDA;
    b->withheld = 1;
    return POLY_OK;
}

int polymul_mod_batched(uint32_t p, int64_t count, const uint32_t *a, const int64_t *a_off, const uint32_t *b,
                        const int64_t *b_off, uint32_t *c, const int64_t *c_off, void *stream) {
    polymul_batch *bt = nullptr;
    int rc = polymul_batch_create(p, count, a_off, b_off, c_off, &bt);
    if (rc) return rc;
    rc = polymul_batch_exec(bt, a, b, c, stream);
    if (!rc) rc = polymul_batch_status(bt);
    polymul_batch_destroy(bt);
    return rc;
}

int polymul_mod_batched_plain(uint32_t p, int64_t count, const uint32_t *a, const int64_t *a_off, const uint32_t *b,
                              const int64_t *b_off, uint32_t *c, const int64_t *c_off, void *stream) {
    if (!a || !b || !c || !a_off || !b_off || !c_off) return POLY_ENULL;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t za = a_off[i + 1] - a_off[i], zb = b_off[i + 1] - b_off[i];
        if (za < 1 || zb < 1) return POLY_EINVAL;
        int rc = polymul_mod_async(p, a + a_off[i], za - 1, b + b_off[i], zb - 1, c + c_off[i], stream);
        if (rc) return rc;
    }
    return POLY_OK;
}

}  // extern "C"
