// autotune.cu -- empirical schedule search (the counterpart of the paper's
// dynamic-programming search that times candidate breakdowns, Section 4).
//
// For each transform length L = 2^l of the three-kernel path, every valid
// (sigma, C) pair -- sigma sets where the tree is split between the column
// and row stages (row length 2^sigma, radix-16 Stockham passes inside a row),
// C the column-tile width -- is timed on a full-length product (n = L - 1)
// with CUDA events around back-to-back products; the fastest is kept and
// used by later plans.  A second phase tunes the batched kernel: for each
// length whose products a batch splits into column, row and ITFT items
// (rows of 2^12 words, fixed by the kernel's CTA shape), a batch of such
// products is timed at every valid column-tile width and the fastest width
// is kept for that length.  The table is written as JSON:
//   {"device": "...", "p": P, "schedules": [{"l": 20, "sigma": 11, "C": 8, "us": 12.3,
//                                            "batch_C": 32, "batch_us": 40.1}, ...]}
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "batch.h"
#include "host.h"
#include "polymul.h"

using namespace pm;

static float time_schedule(PrimeCtx *ctx, int l, Schedule sch, const u32 *a, const u32 *b, u32 *c, u32 *ws,
                           cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    const int64_t L = (int64_t)1 << l, z = L / 2;
    LargeDesc d;
    if (prepare_large(ctx, a, z, b, z, c, l, true, sch, &d)) return -1.f;
    d.wa = ws;
    d.wb = ws + d.g.k * d.g.S;
    // back-to-back products, as a stream of calls runs them (the row and
    // column-ITFT kernels overlap the previous kernel's tail)
    constexpr int reps = 16;
    for (int it = 0; it < 4; ++it)
        if (launch_large(ctx->lazy, d, sch, ctx->m, ctx->tw, st) != cudaSuccess) return -1.f;
    std::vector<float> t;
    for (int rnd = 0; rnd < 5; ++rnd) {
        cudaEventRecord(e0, st);
        for (int it = 0; it < reps; ++it)
            if (launch_large(ctx->lazy, d, sch, ctx->m, ctx->tw, st) != cudaSuccess) return -1.f;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms / reps);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2] * 1000.f;
}

// One batch of `count` products of length 2^l (za = zb = 3 2^(l-3), so n
// needs L = 2^l) at the current width table: median per-product time of
// graph-less launches, microseconds; < 0 on failure.
static float time_batch(u32 p, int l, int64_t count, const u32 *a, const u32 *b, u32 *c, cudaStream_t st,
                        cudaEvent_t e0, cudaEvent_t e1) {
    const int64_t z = (int64_t)3 << (l - 3), n = 2 * z - 1;
    std::vector<int64_t> ao(count + 1), bo(count + 1), co(count + 1);
    for (int64_t i = 0; i <= count; ++i) {
        ao[i] = bo[i] = i * z;
        co[i] = i * n;
    }
    polymul_batch *bt = nullptr;
    if (polymul_batch_create(p, count, ao.data(), bo.data(), co.data(), &bt)) return -1.f;
    float best = -1.f;
    std::vector<float> t;
    for (int rnd = 0; rnd < 6; ++rnd) {
        cudaEventRecord(e0, st);
        const int rc = polymul_batch_exec_nograph(bt, a, b, c, st);
        cudaEventRecord(e1, st);
        if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
            t.clear();
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rnd) t.push_back(ms);  // the first run is a warm-up
    }
    if (polymul_batch_status(bt) == POLY_OK && !t.empty()) {
        std::sort(t.begin(), t.end());
        best = t[t.size() / 2] * 1000.f / (float)count;
    }
    polymul_batch_destroy(bt);
    return best;
}

extern "C" {

int polymul_autotune(uint32_t p, int lo_log, int hi_log, const char *json_path) {
    if (lo_log < SINGLE_SMALL_MAX_LOG_L + 1) lo_log = SINGLE_SMALL_MAX_LOG_L + 1;
    if (hi_log > POLY_MAX_LOG_L || hi_log < lo_log) return POLY_EINVAL;
    PrimeCtx *ctx = nullptr;
    int rc = get_prime(p, 0, hi_log, &ctx, nullptr);
    if (rc) return rc;
    cudaStream_t st;
    cudaEvent_t e0, e1;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return POLY_ECUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int64_t Lmax = (int64_t)1 << hi_log;
    u32 *buf = nullptr;
    // a, b (L/2 each), c (L), workspace (2L)
    if (cudaMalloc(&buf, (size_t)(Lmax / 2 * 2 + Lmax + 2 * Lmax) * 4) != cudaSuccess) {
        cudaStreamDestroy(st);
        return POLY_ENOMEM;
    }
    u32 *a = buf, *b = buf + Lmax / 2, *c = b + Lmax / 2, *ws = c + Lmax;
    cudaMemsetAsync(a, 0x01, (size_t)Lmax * 4, st);
    struct Row {
        int l;
        Schedule s;
        float us;
    };
    std::vector<Row> rows;
    for (int l = lo_log; l <= hi_log; ++l) {
        Schedule best{0, 0};
        float best_us = 1e30f;
        for (int sigma = 9; sigma <= 13; ++sigma)
            for (int C : {8, 32, 128}) {
                Schedule s{sigma, C};
                if (!schedule_valid(l, s)) continue;
                const float us = time_schedule(ctx, l, s, a, b, c, ws, st, e0, e1);
                if (us > 0 && us < best_us) {
                    best_us = us;
                    best = s;
                }
            }
        if (best.sigma) {
            set_schedule(l, best);
            rows.push_back(Row{l, best, best_us});
        }
    }
    cudaFree(buf);
    // phase 2: the batched kernel's column-tile width per length
    struct BRow {
        int l, C;
        float us;
    };
    std::vector<BRow> brows;
    const int blo = std::max(lo_log, SMALL_MAX_LOG_L + 1), bhi = std::min(hi_log, BATCH_SIGMA + LARGE_MAX_LOG_T);
    for (int l = blo; l <= bhi; ++l) {
        const int64_t count = std::max<int64_t>(4, std::min<int64_t>(64, (int64_t)1 << std::max(0, 23 - l)));
        const int64_t z = (int64_t)3 << (l - 3), n = 2 * z - 1;
        u32 *bb = nullptr;
        if (cudaMalloc(&bb, (size_t)count * (2 * z + n) * 4) != cudaSuccess) break;
        cudaMemsetAsync(bb, 0x01, (size_t)count * 2 * z * 4, st);
        const int prev = batch_width_for(l);
        BRow best{l, 0, 1e30f};
        for (int C : {8, 32, 128, 256, 512, 1024, 2048}) {
            if (!batch_width_valid(l, C)) continue;
            set_batch_width(l, C);
            const float us = time_batch(p, l, count, bb, bb + count * z, bb + 2 * count * z, st, e0, e1);
            if (us > 0 && us < best.us) best = BRow{l, C, us};
        }
        cudaFree(bb);
        set_batch_width(l, best.C ? best.C : prev);
        if (best.C) brows.push_back(best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (json_path) {
        FILE *f = fopen(json_path, "w");
        if (!f) return POLY_EINVAL;
        cudaDeviceProp prop;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaGetDeviceProperties(&prop, dev);
        fprintf(f, "{\"device\": \"%s\", \"p\": %u, \"schedules\": [\n", prop.name, p);
        for (size_t i = 0; i < rows.size(); ++i) {
            fprintf(f, "  {\"l\": %d, \"sigma\": %d, \"C\": %d, \"us\": %.3f", rows[i].l, rows[i].s.sigma,
                    rows[i].s.C, rows[i].us);
            for (auto &br : brows)
                if (br.l == rows[i].l) fprintf(f, ", \"batch_C\": %d, \"batch_us\": %.3f", br.C, br.us);
            fprintf(f, "}%s\n", i + 1 < rows.size() ? "," : "");
        }
        fprintf(f, "]}\n");
        fclose(f);
    }
    return POLY_OK;
}

int polymul_load_schedules(const char *json_path) {
    if (!json_path) return POLY_ENULL;
    FILE *f = fopen(json_path, "r");
    if (!f) return POLY_EINVAL;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    fclose(f);
    size_t pos = 0;
    int loaded = 0;
    while ((pos = text.find("{\"l\":", pos)) != std::string::npos) {
        int l = 0, sigma = 0, C = 0;
        if (sscanf(text.c_str() + pos, "{\"l\": %d, \"sigma\": %d, \"C\": %d", &l, &sigma, &C) == 3) {
            Schedule s{sigma, C};
            if (schedule_valid(l, s)) {
                set_schedule(l, s);
                ++loaded;
            }
            // optional batched-kernel width of the same length, within this entry
            const size_t end = text.find('}', pos);
            const size_t bpos = text.find("\"batch_C\":", pos);
            int bc = 0;
            if (bpos != std::string::npos && bpos < end && sscanf(text.c_str() + bpos, "\"batch_C\": %d", &bc) == 1 &&
                batch_width_valid(l, bc))
                set_batch_width(l, bc);
        }
        pos += 5;
    }
    return loaded > 0 ? POLY_OK : POLY_EINVAL;
}

int polymul_get_schedule(int l, int *sigma, int *C) {
    if (!sigma || !C) return POLY_ENULL;
    if (l <= SINGLE_SMALL_MAX_LOG_L || l > POLY_MAX_LOG_L) return POLY_EINVAL;
    const Schedule s = schedule_for(l);
    *sigma = s.sigma;
    *C = s.C;
    return POLY_OK;
}

int polymul_get_batch_width(int l, int *C) {
    if (!C) return POLY_ENULL;
    if (l <= SMALL_MAX_LOG_L || l > BATCH_SIGMA + LARGE_MAX_LOG_T) return POLY_EINVAL;
    *C = batch_width_for(l);
    return POLY_OK;
}

}  // extern "C"
