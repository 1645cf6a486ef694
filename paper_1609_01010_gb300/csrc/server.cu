// server.cu -- continuous-batching server for products of mixed sizes/primes.
//
// submit() queues a request and returns a ticket.  A scheduler thread admits
// queued requests in arrival order while the bytes they hold (operands,
// output and workspace) fit the memory budget, and hands admitted requests
// of one prime, as a group, to a free stream.  Requests that arrive while
// launches are running are admitted into the next group on another stream
// as soon as budget and a stream are free, so their work overlaps on the
// GPU.  Each group ends with an event; the scheduler thread polls the
// events of the groups in flight (it spins while there is work or recent
// activity and sleeps on a condition variable only after 2 ms idle), so a
// completion is seen within about a microsecond; latency = that moment -
// submit.
//
// POLY_SERVE_BATCH (the serving form): one stream in four (at least one)
// is a high-priority lane that takes only small requests (L <= 2^SRV_BATCH_MAX_L), the others
// take every request, large ones first, so the CTAs of small products are
// scheduled ahead of the pending CTAs of large ones instead of queueing
// behind them; a group's small requests run as one launch of the persistent
// batched kernel when there are at least SRV_BATCH_MIN of them (a lone one
// runs plain), the rest as plain products behind it.  POLY_SERVE_PLAIN (the comparator)
// runs every request as its own plain product (1 or 3 kernels) on streams of
// equal priority, groups in arrival order.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"
#include "polymul.h"

namespace pm {

static double now_us() {
    using namespace std::chrono;
    return duration_cast<duration<double, std::micro>>(steady_clock::now().time_since_epoch()).count();
}

// Pinned staging per stream for one launch's work list (allocated at
// creation: pinned allocations are not made while launches are in flight).
constexpr size_t SRV_STAGE_BYTES = (size_t)32 << 20;
// In POLY_SERVE_BATCH, requests with L above 2^SRV_BATCH_MAX_L fill the GPU
// on their own: they run as plain products (the three-kernel path with its
// tuned schedule) behind the group's batched launch.
constexpr int SRV_BATCH_MAX_L = 17;
// ... and a group batches its small requests when it has at least this
// many: a burst of requests that queued while the lanes were busy then costs
// the scheduler thread one work-list upload and one launch instead of one
// to three launches per request (a lone request runs plain).
constexpr size_t SRV_BATCH_MIN = 2;

struct SrvReq {
    uint64_t ticket;
    u32 p;
    const u32 *a, *b;
    u32 *c;
    int64_t za, zb, n;
    uint64_t bytes;
    double t_submit;
};

struct SrvLaunch;

struct SrvStream {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;  // recorded after each group launched on st
    bool busy = false;
    bool small_only = false;  // POLY_SERVE_BATCH: a high-priority lane for small requests
    char *pinned = nullptr;
    size_t pinned_bytes = 0;
};

struct SrvLaunch {
    void *srv;  // the owning polymul_server
    int stream;
    std::vector<uint64_t> tickets;
    std::vector<double> t_submit;
    uint64_t bytes = 0;
    void *dbuf = nullptr;
    int *status_dev = nullptr;
    int *status_host = nullptr;
};

}  // namespace pm

using namespace pm;

struct polymul_server {
    size_t budget = 0;
    int mode = POLY_SERVE_BATCH;
    int dev = 0;
    std::vector<SrvStream> streams;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvReq> pending;
    std::map<uint64_t, int> state;  // 0 queued, 1 running, 2 done
    std::map<uint64_t, int> result;
    std::map<uint64_t, double> latency;  // microseconds, done tickets
    std::vector<SrvLaunch *> inflight;
    std::vector<double> lat_us;
    uint64_t in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    std::map<u32, PrimeCtx *> ctx;
    // Wake-ups of a sleeping scheduler (new request, stop).  The scheduler
    // never holds `mu` across a CUDA call.
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    uint64_t wake_seq = 0;
};

namespace pm {

static void srv_wake(polymul_server *s) {
    {
        std::lock_guard<std::mutex> lk(s->wake_mu);
        ++s->wake_seq;
    }
    s->wake_cv.notify_all();
}

// Work-list bytes a request adds to a launch's staging area (upper bound).
static size_t request_stage_bytes(int64_t n) {
    const int l = ceil_log2(n);
    size_t items = 1;
    if (l > SMALL_MAX_LOG_L) {
        const int64_t S = (int64_t)1 << BATCH_SIGMA;
        items = (size_t)(3 * (S / 16) + ((n + S - 1) / S));
    }
    return sizeof(BatchDesc) + items * sizeof(WorkItem) + 2 * sizeof(int);
}

// Bytes a request holds while admitted: operands, output and the larger of
// its batched and plain workspaces.
static uint64_t request_bytes(int64_t za, int64_t zb) {
    const int64_t n = za + zb - 1;
    uint64_t bytes = (uint64_t)(za + zb + n) * 4;
    const int l = ceil_log2(n);
    if (l > SMALL_MAX_LOG_L)
        bytes += (uint64_t)std::max(large_workspace_words(n, l, Schedule{BATCH_SIGMA, 16}, true),
                                    large_workspace_words(n, l, schedule_for(l), true)) *
                 4;
    return bytes;
}

// Launches one admitted group (one prime) on stream si: the requests that
// go through the batched kernel as one launch, the rest as plain products
// behind it, then one completion callback for the group.  Runs on the
// scheduler thread without the server lock.
static int srv_launch(polymul_server *s, int si, std::vector<SrvReq> &reqs) {
    PrimeCtx *ctx = s->ctx[reqs[0].p];
    SrvStream &ss = s->streams[si];
    std::vector<SrvReq> batched, plain;
    size_t small = 0;
    for (auto &r : reqs) small += ceil_log2(r.n) <= SRV_BATCH_MAX_L;
    const bool batch_small = s->mode == POLY_SERVE_BATCH && small >= SRV_BATCH_MIN;
    for (auto &r : reqs) {
        if (batch_small && ceil_log2(r.n) <= SRV_BATCH_MAX_L) batched.push_back(r);
        else plain.push_back(r);
    }
    SrvLaunch *L = new SrvLaunch();
    L->srv = (void *)s;
    L->stream = si;
    if (!batched.empty()) {
        const int64_t cnt = (int64_t)batched.size();
        std::vector<int64_t> za(cnt), zb(cnt);
        std::vector<uint64_t> ao(cnt), bo(cnt), co(cnt);
        int max_l = 0;
        for (int64_t i = 0; i < cnt; ++i) {
            za[i] = batched[i].za;
            zb[i] = batched[i].zb;
            ao[i] = (uint64_t)(uintptr_t)batched[i].a;
            bo[i] = (uint64_t)(uintptr_t)batched[i].b;
            co[i] = (uint64_t)(uintptr_t)batched[i].c;
            max_l = std::max(max_l, ceil_log2(batched[i].n));
        }
        std::vector<BatchDesc> descs;
        std::vector<WorkItem> items;
        uint64_t ws_bytes = 0;
        size_t smem = 0;
        int rc = build_worklist(ctx, cnt, za.data(), zb.data(), ao.data(), bo.data(), co.data(), descs, items,
                                &ws_bytes, &smem);
        if (rc) {
            delete L;
            return rc;
        }
        const size_t d_bytes = descs.size() * sizeof(BatchDesc);
        const size_t i_bytes = items.size() * sizeof(WorkItem);
        const size_t c_bytes = (2 * cnt + 2) * sizeof(int);
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const size_t stage = up(d_bytes) + up(i_bytes) + up(c_bytes);
        const size_t total = stage + up(ws_bytes);
        if (ss.pinned_bytes < stage + 256) {  // admission keeps launches within the staging area
            delete L;
            return POLY_ENOMEM;
        }
        char *h = ss.pinned;
        memcpy(h, descs.data(), d_bytes);
        memcpy(h + up(d_bytes), items.data(), i_bytes);
        memset(h + up(d_bytes) + up(i_bytes), 0, c_bytes);
        char *dbuf = nullptr;
        if (cudaMallocAsync((void **)&dbuf, total, ss.st) != cudaSuccess) {
            delete L;
            return POLY_ENOMEM;
        }
        L->dbuf = dbuf;
        BatchParams P;
        P.a = nullptr;
        P.b = nullptr;
        P.c = nullptr;
        P.ws = (u32 *)(dbuf + stage);
        P.descs = (const BatchDesc *)dbuf;
        P.items = (const WorkItem *)(dbuf + up(d_bytes));
        P.nitems = (int)items.size();
        P.counters = (int *)(dbuf + up(d_bytes) + up(i_bytes));
        P.head = P.counters + 2 * cnt;
        P.status = P.counters + 2 * cnt + 1;
        P.m = ctx->m;
        P.tw = ctx->tw;
        P.spin_limit = BATCH_SPIN_LIMIT;
        int grid = 0;
        // status word back to pinned host memory, behind the kernel on the stream
        L->status_host = (int *)(h + stage);
        if (cudaMemcpyAsync(dbuf, h, stage, cudaMemcpyHostToDevice, ss.st) != cudaSuccess ||
            launch_batch(ctx->lazy, uniform_width(descs), P, smem, &grid, ss.st) != cudaSuccess ||
            cudaMemcpyAsync(L->status_host, P.status, sizeof(int), cudaMemcpyDeviceToHost, ss.st) != cudaSuccess) {
            cudaFreeAsync(dbuf, ss.st);
            delete L;
            return POLY_ECUDA;
        }
    }
    for (auto &r : plain) {
        const int rc = run_product(r.p, 0, r.a, r.za, r.b, r.zb, r.c, ceil_log2(r.n), true, ss.st, nullptr, -1,
                                   SMALL_MAX_LOG_L);
        if (rc) {
            if (L->dbuf) cudaFreeAsync(L->dbuf, ss.st);
            delete L;
            return rc;
        }
    }
    for (auto &r : reqs) {
        L->tickets.push_back(r.ticket);
        L->t_submit.push_back(r.t_submit);
        L->bytes += r.bytes;
    }
    if (cudaEventRecord(ss.done, ss.st) != cudaSuccess) {
        if (L->dbuf) cudaFreeAsync(L->dbuf, ss.st);
        delete L;
        return POLY_ECUDA;
    }
    ss.busy = true;
    s->inflight.push_back(L);
    return POLY_OK;
}

// Before the first request: every kernel a request can meet is made
// resident on the device (one zero product per transform length and prime,
// one batched launch of the tile width the server's groups use), so no
// request waits for a module to load, and the stream-ordered pool is grown
// once to a part of the budget, so admissions do not map memory.
static int srv_warm_up(polymul_server *s) {
    keep_pool_memory();
    const int max_l = BATCH_SIGMA + LARGE_MAX_LOG_T;
    const int64_t half = (int64_t)1 << (max_l - 1);
    cudaStream_t st = s->streams[0].st;
    u32 *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)4 * half * sizeof(u32)) != cudaSuccess) return POLY_ENOMEM;
    u32 *a = buf, *b = buf + half, *c = buf + 2 * half;
    int rc = cudaMemsetAsync(buf, 0, (size_t)4 * half * sizeof(u32), st) == cudaSuccess ? POLY_OK : POLY_ECUDA;
    for (auto &kv : s->ctx) {
        const u32 p = kv.first;
        for (int l = 1; l <= max_l && !rc; ++l) {
            const int64_t z = (int64_t)1 << (l - 1);  // n = 2z - 1 needs L = 2^l
            rc = run_product(p, 0, a, z, b, z, c, l, true, st, nullptr, -1, SMALL_MAX_LOG_L);
        }
        if (!rc) {  // the batched kernel of the groups' tile width (all batched requests have L <= 2^17)
            const int64_t z = (int64_t)1 << (SRV_BATCH_MAX_L - 2), off[2] = {0, z}, coff[2] = {0, 2 * z - 1};
            rc = polymul_mod_batched(p, 1, a, off, b, off, c, coff, st);
        }
    }
    // grow the pool to min(budget, 1 GiB) once
    void *big = nullptr;
    const size_t reserve = std::min<size_t>(s->budget, (size_t)1 << 30);
    if (!rc && cudaMallocAsync(&big, reserve, st) == cudaSuccess) cudaFreeAsync(big, st);
    cudaGetLastError();
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = POLY_ECUDA;
    cudaFree(buf);
    return rc;
}

// Whether request r may run on stream lane ss (POLY_SERVE_BATCH lanes).
static bool lane_takes(const SrvStream &ss, const SrvReq &r) {
    return !ss.small_only || ceil_log2(r.n) <= SRV_BATCH_MAX_L;
}

static void srv_loop(polymul_server *s) {
    cudaSetDevice(s->dev);
    double last_activity = now_us();
    for (;;) {
        uint64_t seq0;
        {
            std::lock_guard<std::mutex> lk(s->wake_mu);
            seq0 = s->wake_seq;
        }
        bool progress = false;
        // 1. retire finished launches (the in-flight list belongs to this thread)
        for (size_t i = 0; i < s->inflight.size();) {
            SrvLaunch *L = s->inflight[i];
            const cudaError_t q = cudaEventQuery(s->streams[L->stream].done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const double t_done = now_us();
            int st = L->status_host ? *L->status_host : POLY_OK;
            if (q != cudaSuccess) st = POLY_ECUDA;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (size_t j = 0; j < L->tickets.size(); ++j) {
                    s->state[L->tickets[j]] = 2;
                    s->result[L->tickets[j]] = st;
                    s->lat_us.push_back(t_done - L->t_submit[j]);
                    s->latency[L->tickets[j]] = t_done - L->t_submit[j];
                }
                s->in_use -= L->bytes;
            }
            s->cv.notify_all();
            if (L->dbuf) cudaFreeAsync(L->dbuf, s->streams[L->stream].st);
            s->streams[L->stream].busy = false;
            delete L;
            s->inflight.erase(s->inflight.begin() + i);
            progress = true;
        }
        // 2. admit queued requests onto free streams and launch them: in
        // POLY_SERVE_BATCH the small-request lanes first, and the other lanes
        // take large requests before small ones
        for (int pass = 0; pass < 2; ++pass) {
            for (size_t si = 0; si < s->streams.size(); ++si) {
                SrvStream &ss = s->streams[si];
                if (ss.busy || (pass == 0) != ss.small_only) continue;
                std::vector<SrvReq> take;
                uint64_t bytes = 0;
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    if (s->pending.empty()) break;
                    // the group's prime: that of the first request this lane may take
                    // (large ones first on a general lane in the serving mode)
                    const SrvReq *first = nullptr;
                    if (s->mode == POLY_SERVE_BATCH && !ss.small_only)
                        for (auto &r : s->pending)
                            if (ceil_log2(r.n) > SRV_BATCH_MAX_L) {
                                first = &r;
                                break;
                            }
                    if (!first)
                        for (auto &r : s->pending)
                            if (lane_takes(ss, r)) {
                                first = &r;
                                break;
                            }
                    if (!first) continue;
                    const u32 p = first->p;
                    const bool large_first = s->mode == POLY_SERVE_BATCH && !ss.small_only &&
                                             ceil_log2(first->n) > SRV_BATCH_MAX_L;
                    size_t staged = 4096;
                    for (auto it = s->pending.begin(); it != s->pending.end() && take.size() < 8192;) {
                        const bool large = ceil_log2(it->n) > SRV_BATCH_MAX_L;
                        if (it->p != p || !lane_takes(ss, *it) || (large_first && !large)) {
                            ++it;
                            continue;
                        }
                        if (s->in_use + bytes + it->bytes > s->budget) break;
                        const size_t sb = request_stage_bytes(it->n) + 1024;
                        if (staged + sb > ss.pinned_bytes) break;
                        staged += sb;
                        bytes += it->bytes;
                        s->state[it->ticket] = 1;
                        take.push_back(*it);
                        it = s->pending.erase(it);
                    }
                    s->in_use += bytes;
                }
                if (take.empty()) continue;
                const int rc = srv_launch(s, (int)si, take);
                if (rc) {
                    {
                        std::lock_guard<std::mutex> lk(s->mu);
                        s->in_use -= bytes;
                        for (auto &r : take) {
                            s->state[r.ticket] = 2;
                            s->result[r.ticket] = rc;
                        }
                    }
                    s->cv.notify_all();
                }
                progress = true;
            }
        }
        bool idle;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop && s->pending.empty() && s->inflight.empty()) break;
            idle = s->pending.empty() && s->inflight.empty();
        }
        const double now = now_us();
        if (progress || !idle) last_activity = now;
        if (progress) continue;
        if (!idle || now - last_activity < 2000.0) {
            // work in flight, or recent activity: keep polling (completions
            // and new requests are then seen within about a microsecond)
            std::this_thread::yield();
            continue;
        }
        std::unique_lock<std::mutex> lk(s->wake_mu);
        s->wake_cv.wait_for(lk, std::chrono::microseconds(500), [&] { return s->wake_seq != seq0; });
    }
}

}  // namespace pm

extern "C" {

int polymul_server_create(size_t mem_budget_bytes, int n_streams, int mode, polymul_server **out) {
    if (!out) return POLY_ENULL;
    *out = nullptr;
    if (mem_budget_bytes == 0 || n_streams < 1 || n_streams > 64) return POLY_EINVAL;
    if (mode != POLY_SERVE_BATCH && mode != POLY_SERVE_PLAIN) return POLY_EINVAL;
    polymul_server *s = new polymul_server();
    s->budget = mem_budget_bytes;
    s->mode = mode;
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        delete s;
        return POLY_ECUDA;
    }
    const int max_l = BATCH_SIGMA + LARGE_MAX_LOG_T;
    for (u32 p : {469762049u, 2013265921u}) {
        PrimeCtx *c = nullptr;
        int rc = get_prime(p, 0, max_l, &c, nullptr);
        if (rc) {
            delete s;
            return rc;
        }
        s->ctx[p] = c;
        // Step lists for every (T, k) a request can meet are made resident now,
        // so admission never builds one while launches are in flight.
        const ItftStep *st;
        int ns;
        for (int logT = 0; logT <= SMALL_MAX_LOG_T; ++logT)
            for (int64_t k = 1; k <= ((int64_t)1 << logT); ++k) get_steps(c, (int64_t)1 << logT, k, &st, &ns);
        for (int t = SMALL_MAX_LOG_L + 1 - BATCH_SIGMA; t <= LARGE_MAX_LOG_T; ++t) {
            const int64_t T = (int64_t)1 << t;
            for (int64_t k = T / 2 + 1; k <= T; ++k) get_steps(c, T, k, &st, &ns);
        }
        // and for the plain products' schedules
        for (int l = SMALL_MAX_LOG_L + 1; l <= max_l; ++l) {
            const int64_t T = (int64_t)1 << (l - schedule_for(l).sigma);
            for (int64_t k = T / 2 + 1; k <= T; ++k) get_steps(c, T, k, &st, &ns);
        }
    }
    s->streams.resize(n_streams);
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
        delete s;
        return POLY_ECUDA;
    }
    for (size_t si = 0; si < s->streams.size(); ++si) {
        SrvStream &ss = s->streams[si];
        // serving form: one lane in four (at least one) is a high-priority small-request lane
        ss.small_only = mode == POLY_SERVE_BATCH && n_streams >= 2 && (int)si < std::max(1, n_streams / 4);
        if (cudaStreamCreateWithPriority(&ss.st, cudaStreamNonBlocking, ss.small_only ? prio_greatest : prio_least) !=
                cudaSuccess ||
            cudaEventCreateWithFlags(&ss.done, cudaEventDisableTiming) != cudaSuccess) {
            delete s;
            return POLY_ECUDA;
        }
        ss.pinned_bytes = SRV_STAGE_BYTES;
        if (cudaMallocHost(&ss.pinned, ss.pinned_bytes) != cudaSuccess) {
            ss.pinned = nullptr;
            delete s;
            return POLY_ENOMEM;
        }
    }
    int rc = srv_warm_up(s);
    if (rc) {
        for (auto &ss : s->streams) {
            if (ss.st) cudaStreamDestroy(ss.st);
            if (ss.done) cudaEventDestroy(ss.done);
            if (ss.pinned) cudaFreeHost(ss.pinned);
        }
        delete s;
        return rc;
    }
    s->th = std::thread(srv_loop, s);
    *out = s;
    return POLY_OK;
}

int polymul_server_submit(polymul_server *s, uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                          uint32_t *c, uint64_t *ticket) {
    if (!s || !a || !b || !c || !ticket) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    if (s->ctx.find(p) == s->ctx.end()) return POLY_EINVAL_PRIME;
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    if (ceil_log2(n) > BATCH_SIGMA + LARGE_MAX_LOG_T) return POLY_ETOO_LONG;
    const uint64_t bytes = request_bytes(za, zb);
    if (bytes > s->budget) return POLY_EBUSY;
    if (validation_on()) {  // synchronous check on the legacy default stream before the request is queued
        int rc = validate_coeffs(p, a, za, b, zb, nullptr);
        if (rc) return rc;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return POLY_EINVAL;
        SrvReq r{s->next_ticket++, p, a, b, c, za, zb, n, bytes, now_us()};
        s->state[r.ticket] = 0;
        s->pending.push_back(r);
        *ticket = r.ticket;
    }
    srv_wake(s);
    return POLY_OK;
}

int polymul_server_poll(polymul_server *s, uint64_t ticket, int *done) {
    if (!s || !done) return POLY_ENULL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return POLY_ENOTFOUND;
    *done = it->second == 2;
    return *done ? s->result[ticket] : POLY_OK;
}

int polymul_server_wait(polymul_server *s, uint64_t ticket, int64_t timeout_ms) {
    if (!s) return POLY_ENULL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return POLY_ENOTFOUND;
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return s->state[ticket] == 2; });
    if (!ok) return POLY_ETIMEOUT;
    return s->result[ticket];
}

int polymul_server_latency(polymul_server *s, uint64_t ticket, double *us) {
    if (!s || !us) return POLY_ENULL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return POLY_ENOTFOUND;
    auto lt = s->latency.find(ticket);
    if (lt == s->latency.end()) return POLY_EINVAL;  // not done yet (or failed before a launch)
    *us = lt->second;
    return POLY_OK;
}

int polymul_server_stats(polymul_server *s, double *out6) {
    if (!s || !out6) return POLY_ENULL;
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        v = s->lat_us;
    }
    for (int i = 0; i < 6; ++i) out6[i] = 0;
    if (v.empty()) return POLY_OK;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
        return v[std::min(i, v.size() - 1)];
    };
    double sum = 0;
    for (double x : v) sum += x;
    out6[0] = (double)v.size();
    out6[1] = pct(0.50);
    out6[2] = pct(0.90);
    out6[3] = pct(0.99);
    out6[4] = v.back();
    out6[5] = sum / (double)v.size();
    return POLY_OK;
}

int polymul_server_destroy(polymul_server *s) {
    if (!s) return POLY_ENULL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    srv_wake(s);
    if (s->th.joinable()) s->th.join();
    for (auto &ss : s->streams) {
        if (ss.st) {
            cudaStreamSynchronize(ss.st);
            cudaStreamDestroy(ss.st);
        }
        if (ss.done) cudaEventDestroy(ss.done);
        if (ss.pinned) cudaFreeHost(ss.pinned);
    }
    delete s;
    return POLY_OK;
}

}  // extern "C"
