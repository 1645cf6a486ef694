// batch.h -- work-list structures of the persistent batched kernel (shared by
// the batch plan and the server).
#pragma once
#include <map>
#include <vector>

#include "host.h"

namespace pm {

enum ItemKind : int32_t { IT_SMALL = 0, IT_COLF = 1, IT_ROW = 2, IT_COLI = 3 };

struct WorkItem {
    int32_t kind, prod, idx, opnd;
};

// One product of a batch.  Operand and output addresses are byte offsets
// from the launch's base pointers (absolute addresses when the bases are 0).
struct BatchDesc {
    uint64_t a_off, b_off, c_off;
    uint64_t ws_off;  // byte offset into the workspace (large products)
    int64_t za, zb, n;
    Geometry g;
    const ItftStep *steps;
    int32_t nsteps;
    int32_t large;
    int32_t logT, k;  // small products
    int32_t C;        // large products: column-tile width (8, 32, 128, 256, 512, 1024 or 2048 words)
};

struct BatchParams {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t *ws;
    const BatchDesc *descs;
    const WorkItem *items;
    int nitems;
    int *counters;  // 2 per product: column items done, row items done
    int *head;      // next work item
    int *status;    // POLY_OK or POLY_ETIMEOUT
    ModParams m;
    TwTables tw;
    long long spin_limit;
};

constexpr int BATCH_THREADS = 256;
constexpr int BATCH_SIGMA = 12;  // rows of 4096 words: one row per CTA of 256 threads
constexpr size_t BATCH_SMEM_MAX = 64 * 1024;
// ~1.6 s of polling at 128 ns per poll before a wait is declared failed.
constexpr long long BATCH_SPIN_LIMIT = 1ll << 24;

// uniform_C: the common column-tile width of the launch's large products, or
// 0 when they differ (the kernel then dispatches per product).
cudaError_t launch_batch(bool lazy, int uniform_C, const BatchParams &P, size_t smem, int *grid, cudaStream_t st);
// The common column-tile width of the large products in descs (128 when
// there is none), or 0 when they differ.
int uniform_width(const std::vector<BatchDesc> &descs);
// Work list of `count` products; each large product's column tiles have the
// width batch_width_for(l) of its transform length 2^l.
int build_worklist(PrimeCtx *ctx, int64_t count, const int64_t *za, const int64_t *zb, const uint64_t *a_off,
                   const uint64_t *b_off, const uint64_t *c_off, std::vector<BatchDesc> &descs,
                   std::vector<WorkItem> &items, uint64_t *ws_bytes, size_t *smem_bytes);
// Column-tile width of a product of length 2^l inside a batch: the tuned
// table (polymul_autotune, polymul_load_schedules) or the built-in rule.
int batch_width_for(int l);
int batch_width_default(int l);
bool batch_width_valid(int l, int C);
void set_batch_width(int l, int C);
std::map<int, int> all_batch_widths();

}  // namespace pm
