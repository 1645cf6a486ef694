// host.cu -- host runtime of the C ABI: primes and resident twiddle tables,
// ITFT step lists, schedules, and the single-product / transform entry points.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "host.h"
#include "polymul.h"

namespace pm {

cudaError_t launch_build_tw(uint2 *fwd, uint2 *inv, int lmax, u32 p, const u32 *pw_lo, const u32 *pw_hi,
                            cudaStream_t st);

static thread_local char g_last_err[256] = "";

int cuda_fail(cudaError_t e, const char *where) {
    snprintf(g_last_err, sizeof g_last_err, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return POLY_ECUDA;
}

// ------------------------------------------------------------ host math
int aux_streams(AuxStreams **out) {
    static thread_local std::vector<AuxStreams> per_dev;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    for (auto &x : per_dev)
        if (x.dev == dev) {
            *out = &x;
            return POLY_OK;
        }
    AuxStreams x;
    x.dev = dev;
    for (int j = 0; j < AUX_STREAMS && e == cudaSuccess; ++j)
        e = cudaStreamCreateWithFlags(&x.s[j], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming);
    for (int j = 0; j < AUX_STREAMS && e == cudaSuccess; ++j)
        e = cudaEventCreateWithFlags(&x.join[j], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "auxiliary streams");
    per_dev.push_back(x);
    *out = &per_dev.back();
    return POLY_OK;
}

u32 h_powmod(u64 b, u64 e, u32 p) {
    u64 r = 1 % p;
    b %= p;
    while (e) {
        if (e & 1) r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return (u32)r;
}
u32 h_invmod(u32 a, u32 p) { return h_powmod(a, (u64)p - 2, p); }
uint2 shoup_pair(u32 w, u32 p) { return make_uint2(w, (u32)(((u64)w << 32) / p)); }

static u32 pinv32(u32 p) {
    u32 x = p;  // p*x = 1 mod 8 for odd p
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return x;
}

static bool h_is_prime(u32 p) {
    if (p < 2) return false;
    if (p % 2 == 0) return p == 2;
    for (u64 d = 3; d * d <= p; d += 2)
        if (p % d == 0) return false;
    return true;
}

static bool h_is_primitive_root(u32 g, u32 p) {
    u32 n = p - 1;
    for (u32 d = 2; (u64)d * d <= n; ++d) {
        if (n % d == 0) {
            if (h_powmod(g, (p - 1) / d, p) == 1) return false;
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1 && h_powmod(g, (p - 1) / n, p) == 1) return false;
    return true;
}

static u32 h_bitrev(u32 i, int bits) {
    u32 r = 0;
    for (int b = 0; b < bits; ++b) {
        r = (r << 1) | (i & 1u);
        i >>= 1;
    }
    return r;
}

int ceil_log2(int64_t n) {
    int l = 0;
    while (((int64_t)1 << l) < n) ++l;
    return l;
}

static u32 default_root(u32 p) {
    if (p == 469762049u) return 3;
    if (p == 2013265921u) return 31;
    for (u32 g = 2; g < p; ++g)
        if (h_is_primitive_root(g, p)) return g;
    return 0;
}

// ------------------------------------------------------------ device status
// One word per device that kernels set when a bounded wait expires (or, in
// validating runs, when an input is out of range).  A static device variable,
// so fetching it never allocates.
static __device__ int g_pm_status;

int *device_status_ptr() {
    static std::mutex mu;
    static std::map<int, int *> ptrs;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = ptrs.find(dev);
    if (it != ptrs.end()) return it->second;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pm_status) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ptrs[dev] = (int *)p;
    return (int *)p;
}

// ------------------------------------------------------------ validation
// With validation on, the entry points check that their inputs are residues
// (below p) with one pass over them before any product work, and return
// POLY_EINVAL_COEF otherwise.  The check synchronises the caller's stream.
static std::atomic<int> g_validate{0};
static __device__ int g_pm_badcoef;

__global__ void k_check_range(const u32 *__restrict__ x, int64_t n, u32 p, int *bad) {
    bool any = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        any |= x[i] >= p;
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicExch(bad, 1);
}

bool validation_on() { return g_validate.load(std::memory_order_relaxed) != 0; }

int validate_coeffs(u32 p, const u32 *a, int64_t za, const u32 *b, int64_t zb, cudaStream_t st) {
    if (!validation_on()) return POLY_OK;
    static std::mutex mu;  // one flag per device, one check at a time
    static std::map<int, int *> flags;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLY_ECUDA;
    auto it = flags.find(dev);
    if (it == flags.end()) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_pm_badcoef);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(validation flag)");
        it = flags.emplace(dev, (int *)ptr).first;
    }
    int *flag = it->second;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    const int threads = 256;
    for (int o = 0; o < 2 && e == cudaSuccess; ++o) {
        const u32 *x = o ? b : a;
        const int64_t n = o ? zb : za;
        if (!x || n <= 0) continue;
        const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 1216);
        k_check_range<<<blocks, threads, 0, st>>>(x, n, p, flag);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "coefficient validation");
    return h ? POLY_EINVAL_COEF : POLY_OK;
}

// ------------------------------------------------------------ prime registry
static std::mutex g_mu;
static std::map<std::tuple<int, u32, u32>, PrimeCtx *> g_primes;
static std::map<u32, bool> g_prime_ok;

int validate_prime(u32 p, u32 *root) {
    if (p < 3 || (p & 1u) == 0 || p >= (1u << 31)) return POLY_EINVAL_PRIME;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_prime_ok.find(p);
        if (it == g_prime_ok.end()) it = g_prime_ok.emplace(p, h_is_prime(p)).first;
        if (!it->second) return POLY_EINVAL_PRIME;
    }
    if (*root == 0) *root = default_root(p);
    if (*root == 0 || *root >= p || !h_is_primitive_root(*root, p)) return POLY_EINVAL_PRIME;
    return POLY_OK;
}

static int build_tables(PrimeCtx *ctx, int lmax, cudaStream_t st) {
    const u32 p = ctx->p;
    const u32 psi = h_powmod(ctx->root, (u64)(p - 1) >> lmax, p);
    std::vector<u32> lo(4096), hi(((size_t)1 << lmax) / 4096 + 2);
    u64 x = 1;
    for (size_t a = 0; a < lo.size(); ++a) {
        lo[a] = (u32)x;
        x = x * psi % p;
    }
    const u32 step = h_powmod(psi, 4096, p);
    x = 1;
    for (size_t b = 0; b < hi.size(); ++b) {
        hi[b] = (u32)x;
        x = x * step % p;
    }
    const size_t entries = (size_t)1 << lmax;
    uint2 *fwd = nullptr, *inv = nullptr;
    u32 *dlo = nullptr, *dhi = nullptr;
    if (cudaMalloc(&fwd, entries * sizeof(uint2)) != cudaSuccess) return POLY_ENOMEM;
    if (cudaMalloc(&inv, entries * sizeof(uint2)) != cudaSuccess) {
        cudaFree(fwd);
        return POLY_ENOMEM;
    }
    if (cudaMalloc(&dlo, lo.size() * 4) != cudaSuccess || cudaMalloc(&dhi, hi.size() * 4) != cudaSuccess) {
        cudaFree(fwd);
        cudaFree(inv);
        if (dlo) cudaFree(dlo);
        return POLY_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(dlo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dhi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_build_tw(fwd, inv, lmax, p, dlo, dhi, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dlo);
    cudaFree(dhi);
    if (e != cudaSuccess) {
        cudaFree(fwd);
        cudaFree(inv);
        return POLY_ECUDA;
    }
    // Kernels already queued may still read the old tables: keep them alive.
    if (ctx->fwd) ctx->retired.push_back(const_cast<uint2 *>(ctx->tw.fwd));
    if (ctx->inv) ctx->retired.push_back(const_cast<uint2 *>(ctx->tw.inv));
    ctx->fwd = fwd;
    ctx->inv = inv;
    ctx->tw.fwd = fwd;
    ctx->tw.inv = inv;
    ctx->tw.lmax = lmax;
    return POLY_OK;
}

int get_prime(u32 p, u32 root, int need_l, PrimeCtx **out, cudaStream_t st) {
    int rc = validate_prime(p, &root);
    if (rc) return rc;
    const int v2 = __builtin_ctz(p - 1);
    if (need_l > v2 || need_l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLY_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(dev, p, root);
    auto it = g_primes.find(key);
    PrimeCtx *ctx;
    if (it == g_primes.end()) {
        ctx = new PrimeCtx();
        ctx->p = p;
        ctx->root = root;
        ctx->v2 = v2;
        ctx->lazy = p < (1u << 30);
        ctx->m.p = p;
        ctx->m.pinv = pinv32(p);
        ctx->tw = TwTables{nullptr, nullptr, 0, nullptr};
        const std::vector<uint2> ps = pscale_table(p);
        if (cudaMalloc(&ctx->pscale, ps.size() * sizeof(uint2)) != cudaSuccess) {
            delete ctx;
            return POLY_ENOMEM;
        }
        if (cudaMemcpy(ctx->pscale, ps.data(), ps.size() * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(ctx->pscale);
            delete ctx;
            return POLY_ECUDA;
        }
        ctx->tw.pscale = ctx->pscale;
        ctx->tw.status = device_status_ptr();
        g_primes[key] = ctx;
    } else {
        ctx = it->second;
    }
    int want = need_l < 16 ? 16 : need_l;
    if (want > v2) want = v2;
    if (ctx->tw.lmax < need_l || ctx->tw.fwd == nullptr) {
        rc = build_tables(ctx, want, st);
        if (rc) return rc;
    }
    *out = ctx;
    return POLY_OK;
}

// ------------------------------------------------------------ ITFT steps
// ITFT of node (s, i) of size M (rows [base, base+M)) from its first k leaves,
// with the coefficients at rows >= k known (all zero when `zero`).  The node
// splits x^M - r^2 into x^h - r (left, rows [base, base+h)) and x^h + r
// (right); left coefficients are c_j + r c_{j+h}, right ones c_j - r c_{j+h}.
//   k >= h: invert the left child fully (giving h times its coefficients);
//           for j >= m = k-h the upper c_{j+h} are known, so c_j and the right
//           child's coefficient c_j - r c_{j+h} follow (PRE_RIGHT); recurse on
//           the right child with m leaves; combine the halves (POST_RIGHT).
//   k <  h: the left child's coefficients for j >= k are known (PRE_LEFT),
//           recurse on it, then c_j = lo_j - r c_{j+h} (POST_LEFT).
// Every step keeps the scale of its inputs, except a top-level node with all
// M leaves, which is one unscaled full inverse (M times the coefficients).
// A FULL record of size h leaves h times its coefficients, which the next
// record multiplies by h^-1; with `prescaled` the leaves were already
// multiplied by 1/h and h^-1 is recorded as 1.
static void steps_rec(PrimeCtx *ctx, int s, u32 i, int base, int M, int k, bool zero, bool prescaled,
                      std::vector<ItftStep> &out) {
    const u32 p = ctx->p;
    if (k == 0) return;
    ItftStep st{};
    if (k == M) {
        st.kind = ST_FULL;
        st.s = s;
        st.i = i;
        st.base = base;
        st.h = M;
        out.push_back(st);
        return;
    }
    const int h = M / 2;
    const u32 psi = h_powmod(ctx->root, (u64)(p - 1) >> (s + 1), p);
    const u32 rev = h_bitrev(i, s);
    const u32 r = h_powmod(psi, rev, p);
    st.s = s;
    st.i = i;
    st.base = base;
    st.h = h;
    st.r = shoup_pair(r, p);
    st.hinv = shoup_pair(prescaled ? 1u : h_invmod((u32)(h % p), p), p);
    st.inv2 = shoup_pair(h_invmod(2, p), p);
    st.i2r = shoup_pair(h_invmod((u32)((u64)2 * r % p), p), p);
    if (k >= h) {
        const int m = k - h;
        ItftStep f{};
        f.kind = ST_FULL;
        f.s = s + 1;
        f.i = 2 * i;
        f.base = base;
        f.h = h;
        out.push_back(f);
        st.kind = ST_PRE_RIGHT;
        st.m = m;
        st.zero = zero ? 1 : 0;
        out.push_back(st);
        steps_rec(ctx, s + 1, 2 * i + 1, base + h, h, m, false, prescaled, out);
        st.kind = ST_POST_RIGHT;
        st.zero = 0;
        out.push_back(st);
    } else {
        st.m = k;
        if (!zero) {
            st.kind = ST_PRE_LEFT;
            out.push_back(st);
        }
        steps_rec(ctx, s + 1, 2 * i, base, h, k, zero, prescaled, out);
        if (!zero) {
            st.kind = ST_POST_LEFT;
            out.push_back(st);
        }
    }
}

std::vector<ItftStep> itft_steps(PrimeCtx *ctx, int64_t M, int64_t k, bool prescaled) {
    std::vector<ItftStep> out;
    steps_rec(ctx, 0, 0, 0, (int)M, (int)k, true, prescaled, out);
    return out;
}

std::vector<uint2> pscale_table(u32 p) {
    std::vector<uint2> t(32);
    for (int e = 0; e < 32; ++e) t[e] = scale_const(p, (u64)1 << e);
    return t;
}

// Device copy of the step list for (T, k), cached per prime context.
int get_steps(PrimeCtx *ctx, int64_t T, int64_t k, const ItftStep **d_steps, int *nsteps) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(T, k);
    auto it = ctx->steps.find(key);
    if (it != ctx->steps.end()) {
        *d_steps = it->second.first;
        *nsteps = it->second.second;
        return POLY_OK;
    }
    std::vector<ItftStep> v = itft_steps(ctx, T, k, true);
    if (!ctx->upload && cudaStreamCreateWithFlags(&ctx->upload, cudaStreamNonBlocking) != cudaSuccess)
        return POLY_ECUDA;
    if (ctx->arena_used + v.size() > ctx->arena_cap) {
        const size_t cap = std::max<size_t>(v.size(), (size_t)1 << 15);
        ItftStep *a = nullptr;
        if (cudaMalloc(&a, cap * sizeof(ItftStep)) != cudaSuccess) return POLY_ENOMEM;
        ctx->arenas.push_back(a);
        ctx->arena_used = 0;
        ctx->arena_cap = cap;
    }
    ItftStep *d = ctx->arenas.back() + ctx->arena_used;
    if (cudaMemcpyAsync(d, v.data(), v.size() * sizeof(ItftStep), cudaMemcpyHostToDevice, ctx->upload) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->upload) != cudaSuccess)
        return POLY_ECUDA;
    ctx->arena_used += v.size();
    ctx->steps[key] = std::make_pair((const ItftStep *)d, (int)v.size());
    *d_steps = d;
    *nsteps = (int)v.size();
    return POLY_OK;
}

// ------------------------------------------------------------ schedules
static std::mutex g_sched_mu;
static std::map<int, Schedule> g_sched;  // autotuned, by log2 L
static std::atomic<uint64_t> g_sched_version{1};  // bumped by every schedule change

// Defaults from timing every valid (sigma, C) on GB300 with back-to-back
// products mod 469762049 (polymul_autotune measures the same way); the row
// kernel and the column ITFT start early under programmatic dependent
// launch, so the best split differs from one that isolated launches would
// pick.  C = 32 selects the TMA-fed column kernels.
Schedule default_schedule(int l) {
    switch (l) {
        case 10:
        case 11:
        case 12: return Schedule{9, 128};
        case 13: return Schedule{10, 128};
        case 14: return Schedule{9, 8};
        case 15:
        case 16: return Schedule{10, 8};
        case 17:
        case 18: return Schedule{11, 8};
        case 19: return Schedule{10, 8};
        case 20: return Schedule{11, 8};
        case 21: return Schedule{12, 8};
        case 22: return Schedule{12, 32};
        case 23: return Schedule{13, 32};
        default: return l < 10 ? Schedule{9, 8} : Schedule{13, 8};
    }
}

// Column tiles are double-buffered: 2 * T * C words must fit 128 KB.  The
// TMA-fed kernels of 32-column tiles also take t = 10 (one 128 KB stage).
bool schedule_valid(int l, Schedule s) {
    if (s.sigma < 9 || s.sigma > 13 || s.sigma > l) return false;
    if (s.C != 8 && s.C != 32 && s.C != 128) return false;
    const int t = l - s.sigma;
    if (t < 1 || t > 11) return false;
    if (((int64_t)2 << t) * s.C * 4 > 128 * 1024 && !(s.C == 32 && t == 10)) return false;
    if (((int64_t)1 << s.sigma) < s.C) return false;
    return true;
}

Schedule schedule_for(int l) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched.find(l);
    if (it != g_sched.end() && schedule_valid(l, it->second)) return it->second;
    return default_schedule(l);
}

void set_schedule(int l, Schedule s) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched[l] = s;
    g_sched_version.fetch_add(1);
}

std::map<int, Schedule> all_schedules() {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    return g_sched;
}

Geometry make_geometry(int64_t n, int l, int sigma) {
    Geometry g;
    g.l = l;
    g.L = (int64_t)1 << l;
    g.sigma = sigma < l ? sigma : l;
    g.S = (int64_t)1 << g.sigma;
    g.t = l - g.sigma;
    g.T = (int64_t)1 << g.t;
    g.n = n;
    // Relaxed truncation (Section 5's relaxed parallel algorithms): the
    // ceil(n/S) rows the product needs are rounded up to a multiple of
    // T / 2^RELAX_LOG_T, so the truncated inverse has at most RELAX_LOG_T
    // levels of bookkeeping records instead of t.  The extra rows hold true
    // spectral values, and the product (degree < n) is unchanged.
    const int64_t need = (n + g.S - 1) / g.S;
    const int64_t gran = g.t > RELAX_LOG_T ? g.T >> RELAX_LOG_T : 1;
    g.k = (need + gran - 1) / gran * gran;
    if (g.k > g.T) g.k = g.T;
    return g;
}

uint2 scale_const(u32 p, u64 scale) {
    const u32 r32 = (u32)((((u64)1) << 32) % p);
    const u32 c = (u32)((u64)r32 * h_invmod((u32)(scale % p), p) % p);
    return shoup_pair(c, p);
}

// ------------------------------------------------------------ profiling
// While enabled, every product records CUDA events around its kernels.
static std::mutex g_prof_mu;
static bool g_prof_on = false;
struct ProfRec {
    int kind;  // 0 small, 1 large
    cudaEvent_t ev[4];
};
static std::vector<ProfRec> g_prof;

static cudaEvent_t *prof_events(int kind) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return nullptr;
    ProfRec r;
    r.kind = kind;
    for (int i = 0; i < 4; ++i) cudaEventCreate(&r.ev[i]);
    g_prof.push_back(r);
    return g_prof.back().ev;
}

// ------------------------------------------------------------ products
// Fills a product descriptor for the small (one CTA) path.
int prepare_small(PrimeCtx *ctx, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                  SmallDesc *d, int64_t n_out) {
    const int lp = l < SMALL_LOG_S ? SMALL_LOG_S : l;
    const int logT = lp - SMALL_LOG_S;
    const int64_t T = (int64_t)1 << logT, S = (int64_t)1 << SMALL_LOG_S;
    const int64_t n = n_out < 0 ? za + zb - 1 : n_out;
    const int64_t k = prune ? (n + S - 1) / S : T;
    const ItftStep *st = nullptr;
    int ns = 0;
    int rc = get_steps(ctx, T, k, &st, &ns);
    if (rc) return rc;
    d->a = a;
    d->b = b;
    d->c = c;
    d->za = za;
    d->zb = zb;
    d->n = n;
    d->logT = logT;
    d->k = (int32_t)k;
    d->steps = st;
    d->nsteps = ns;
    d->prune = prune ? 1 : 0;
    return POLY_OK;
}

int prepare_large(PrimeCtx *ctx, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                  Schedule sch, LargeDesc *d, int64_t n_out) {
    const int64_t n = n_out < 0 ? za + zb - 1 : n_out;
    Geometry g = make_geometry(n, l, sch.sigma);
    if (!prune) g.k = g.T;
    const ItftStep *st = nullptr;
    int ns = 0;
    int rc = get_steps(ctx, g.T, g.k, &st, &ns);
    if (rc) return rc;
    d->a = a;
    d->b = b;
    d->c = c;
    d->wa = d->wb = nullptr;
    d->za = za;
    d->zb = zb;
    d->n = n;
    d->g = g;
    d->steps = st;
    d->nsteps = ns;
    d->prune = prune ? 1 : 0;
    return POLY_OK;
}

int64_t large_workspace_words(int64_t n, int l, Schedule sch, bool prune) {
    Geometry g = make_geometry(n, l, sch.sigma);
    if (!prune) g.k = g.T;
    return 2 * g.k * g.S;
}

// Per-thread cache of recently prepared product shapes: a repeated shape
// (the common case of a caller looping over same-size products) skips the
// prime validation, the mutex-guarded context, step-list and schedule
// lookups.  An entry stays valid because prime contexts and step lists live
// until the process exits and twiddle tables only grow (retired ones stay
// allocated); a schedule change (autotuning, a loaded table) bumps
// g_sched_version and so misses every entry.

struct PlanEntry {
    uint64_t ver = 0;
    int dev = -1, l = 0, small_max_l = 0;
    u32 p = 0, root = 0;
    int64_t n = 0;
    bool prune = false;
    PrimeCtx *ctx = nullptr;
    Schedule sch{0, 0};
    Geometry g{};
    const ItftStep *steps = nullptr;
    int nsteps = 0;
    int logT = 0;
    int64_t k = 0;
};
constexpr int PLAN_CACHE = 8;

static PlanEntry *plan_lookup(int dev, u32 p, u32 root, int l, int64_t n, bool prune, int small_max_l) {
    static thread_local PlanEntry cache[PLAN_CACHE];
    const uint64_t ver = g_sched_version.load(std::memory_order_acquire);
    const uint64_t h = ((uint64_t)p * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)n * 0xC2B2AE3D27D4EB4Full) ^
                       ((uint64_t)l << 7) ^ ((uint64_t)prune << 5) ^ (uint64_t)dev ^ ((uint64_t)small_max_l << 11);
    PlanEntry &e = cache[(h >> 29) % PLAN_CACHE];
    if (e.ver == ver && e.dev == dev && e.p == p && e.root == root && e.l == l && e.n == n && e.prune == prune &&
        e.small_max_l == small_max_l)
        return &e;
    e.ver = 0;  // filled by the caller after a miss
    e.dev = dev;
    e.p = p;
    e.root = root;
    e.l = l;
    e.n = n;
    e.prune = prune;
    e.small_max_l = small_max_l;
    return &e;
}

int run_product(u32 p, u32 root, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                cudaStream_t st, u32 *workspace, int64_t n_out, int small_max_l) {
    if (!a || !b || !c) return POLY_ENULL;
    PrimeCtx *ctx = nullptr;
    // Small products run with L padded to at least 512 (the product does not
    // depend on L), so their tables must reach depth 9.
    const bool small = l <= std::min(small_max_l, SMALL_MAX_LOG_L);
    const int need = (small && l < SMALL_LOG_S) ? SMALL_LOG_S : l;
    const int64_t n = n_out < 0 ? za + zb - 1 : n_out;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLY_ECUDA;
    PlanEntry *pe = plan_lookup(dev, p, root, l, n, prune, small_max_l);
    const bool hit = pe->ver != 0;
    int rc;
    if (hit) {
        ctx = pe->ctx;
    } else {
        rc = get_prime(p, root, need, &ctx, st);
        if (rc) return rc;
    }
    if (small) {
        SmallDesc d;
        if (hit) {
            d.a = a;
            d.b = b;
            d.c = c;
            d.za = za;
            d.zb = zb;
            d.n = n;
            d.logT = pe->logT;
            d.k = (int32_t)pe->k;
            d.steps = pe->steps;
            d.nsteps = pe->nsteps;
            d.prune = prune ? 1 : 0;
        } else {
            rc = prepare_small(ctx, a, za, b, zb, c, l, prune, &d, n_out);
            if (rc) return rc;
            pe->ctx = ctx;
            pe->logT = d.logT;
            pe->k = d.k;
            pe->steps = d.steps;
            pe->nsteps = d.nsteps;
            pe->ver = g_sched_version.load(std::memory_order_acquire);
        }
        cudaEvent_t *ev = prof_events(0);
        if (ev) cudaEventRecord(ev[0], st);
        cudaError_t e = launch_small(ctx->lazy, d.logT, nullptr, &d, 1, ctx->m, ctx->tw, st);
        if (ev) cudaEventRecord(ev[1], st);
        return e == cudaSuccess ? POLY_OK : cuda_fail(e, "one-CTA product launch");
    }
    LargeDesc d;
    Schedule sch;
    if (hit) {
        sch = pe->sch;
        d.a = a;
        d.b = b;
        d.c = c;
        d.wa = d.wb = nullptr;
        d.za = za;
        d.zb = zb;
        d.n = n;
        d.g = pe->g;
        d.steps = pe->steps;
        d.nsteps = pe->nsteps;
        d.prune = prune ? 1 : 0;
    } else {
        const uint64_t ver = g_sched_version.load(std::memory_order_acquire);
        sch = schedule_for(l);
        rc = prepare_large(ctx, a, za, b, zb, c, l, prune, sch, &d, n_out);
        if (rc) return rc;
        pe->ctx = ctx;
        pe->sch = sch;
        pe->g = d.g;
        pe->steps = d.steps;
        pe->nsteps = d.nsteps;
        pe->ver = ver;
    }
    const size_t bytes = (size_t)2 * d.g.k * d.g.S * sizeof(u32);
    u32 *ws = workspace;
    if (!ws) {
        cudaError_t e = cudaMallocAsync((void **)&ws, bytes, st);
        if (e != cudaSuccess) {
            cuda_fail(e, "workspace cudaMallocAsync");
            return POLY_ENOMEM;
        }
    }
    d.wa = ws;
    d.wb = ws + d.g.k * d.g.S;
    cudaError_t e = launch_large(ctx->lazy, d, sch, ctx->m, ctx->tw, st, prof_events(1));
    if (!workspace) {
        cudaError_t ef = cudaFreeAsync(ws, st);
        if (e == cudaSuccess) e = ef;
    }
    return e == cudaSuccess ? POLY_OK : cuda_fail(e, "three-kernel product launch");
}

void keep_pool_memory() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();  // an unsupported pool attribute must not surface at the next launch
    });
}

// Whether kernels on device `dev` may read and write ordinary host memory in
// place: the device walks the host's page tables (address translation
// services; on Grace systems over the coherent NVLink-C2C link), so every
// host address the process can use is also valid in a kernel.  Then the host
// entry point needs no staging buffers or copies.
// Host-buffer products with n <= 2^19 words run on the host buffers in place
// when the device can address them: measured on GB300 (Grace host) end to end
// 22 / 52 us at n = 2^10 / 2^19 in place against 29 / 57 us with copy kernels
// and 36 / 65 us with copy engines.  Larger ones are staged: the column
// kernels' 32-byte row segments use the link poorly (217 against 141 us at
// n = 2^21), while the copy kernels move it in 16-byte vectors.
constexpr int64_t HOST_IN_PLACE_MAX_N = (int64_t)1 << 19;

// Copies of up to two segments (src0 -> dst0, n0 words; src1 -> dst1, n1
// words) by all SMs, 16-byte accesses where both sides allow them; either
// side may be host memory the device can address.  Four independent
// accesses per thread keep the link's latency covered.
__global__ void __launch_bounds__(512) k_copy_words(const u32 *__restrict__ s0, u32 *__restrict__ d0, int64_t n0,
                                                    const u32 *__restrict__ s1, u32 *__restrict__ d1, int64_t n1) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int seg = 0; seg < 2; ++seg) {
        const u32 *s = seg ? s1 : s0;
        u32 *d = seg ? d1 : d0;
        const int64_t n = seg ? n1 : n0;
        if (n <= 0) continue;
        const int64_t head = ((((uintptr_t)s) | ((uintptr_t)d)) & 15) == 0 ? 0 : n;  // words before the vector part
        const int64_t n4 = (n - head) / 4;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(s + head);
        uint4 *d4 = reinterpret_cast<uint4 *>(d + head);
        for (int64_t i = t; i < n4; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * stride < n4) v[u] = s4[i + u * stride];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * stride < n4) d4[i + u * stride] = v[u];
        }
        for (int64_t i = t; i < head; i += stride) d[i] = s[i];
        for (int64_t i = head + 4 * n4 + t; i < n; i += stride) d[i] = s[i];
    }
}

static cudaError_t launch_copy_words(const u32 *s0, u32 *d0, int64_t n0, const u32 *s1, u32 *d1, int64_t n1,
                                     cudaStream_t st) {
    const int64_t vec = (std::max(n0, n1) + 3) / 4;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((vec + 511) / 512, 152 * 4));
    k_copy_words<<<blocks, 512, 0, st>>>(s0, d0, n0, s1, d1, n1);
    return cudaGetLastError();
}

static bool host_memory_in_place(int dev) {
    static std::mutex mu;
    static std::map<int, bool> known;
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find(dev);
    if (it != known.end()) return it->second;
    int ats = 0;
    if (cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
        cudaGetLastError();
        ats = 0;
    }
    return known[dev] = (ats == 1);
}

}  // namespace pm

using namespace pm;

// ================================================================ C ABI
extern "C" {

const char *polymul_strerror(int s) {
    switch (s) {
        case POLY_OK: return "ok";
        case POLY_EINVAL_PRIME: return "p is not an odd prime below 2^31, or root is not a primitive root";
        case POLY_ETOO_LONG: return "transform length exceeds the prime's 2-adic order or the library limit";
        case POLY_ENULL: return "a required pointer is NULL";
        case POLY_ENOMEM: return "allocation failed";
        case POLY_ECUDA: return "a CUDA runtime call failed";
        case POLY_ETIMEOUT: return "a bounded wait expired";
        case POLY_EINVAL: return "argument out of range";
        case POLY_EBUSY: return "request exceeds the server memory budget";
        case POLY_ENOTFOUND: return "unknown ticket";
        case POLY_EINVAL_COEF: return "an input coefficient is outside [0, p)";
        case POLY_EDEBUG_CHECK: return "a range or index check of the debug build failed in a kernel";
        default: return "unknown status";
    }
}

const char *polymul_version(void) { return "gb300-polymul 0.1 (sm_103a)"; }

const char *polymul_last_error(void) { return g_last_err; }

int polymul_device_status(int clear) {
    int *p = device_status_ptr();
    if (!p) return POLY_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return POLY_ECUDA;
    if (clear && v != 0) {
        const int zero = 0;
        if (cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return POLY_ECUDA;
    }
    return v;
}

int polymul_set_validate(int on) {
    g_validate.store(on ? 1 : 0);
    return POLY_OK;
}

int polymul_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = true;
    return POLY_OK;
}

int polymul_profile_end(double *ms4, int64_t *launches4) {
    if (!ms4 || !launches4) return POLY_ENULL;
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_on = false;
        recs.swap(g_prof);
    }
    for (int i = 0; i < 4; ++i) {
        ms4[i] = 0;
        launches4[i] = 0;
    }
    int rc = POLY_OK;
    for (auto &r : recs) {
        float t[3] = {0, 0, 0};
        const int nk = r.kind == 0 ? 1 : 3;
        for (int j = 0; j < nk; ++j) {
            if (cudaEventSynchronize(r.ev[j + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&t[j], r.ev[j], r.ev[j + 1]) != cudaSuccess)
                rc = POLY_ECUDA;
        }
        if (r.kind == 0) {
            ms4[0] += t[0];
            launches4[0] += 1;
        } else {
            for (int j = 0; j < 3; ++j) {
                ms4[1 + j] += t[j];
                launches4[1 + j] += 1;
            }
        }
        for (int j = 0; j < 4; ++j) cudaEventDestroy(r.ev[j]);
    }
    return rc;
}

int polymul_mod_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                      void *stream) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    keep_pool_memory();
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    const int l = ceil_log2(n);
    if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    if (validation_on()) {
        u32 root = 0;
        int rc = validate_prime(p, &root);
        if (!rc) rc = validate_coeffs(p, a, za, b, zb, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return run_product(p, 0, a, za, b, zb, c, l, true, (cudaStream_t)stream, nullptr);
}

int polymul_mod(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c) {
    int rc = polymul_mod_async(p, a, da, b, db, c, nullptr);
    if (rc) return rc;
    return cudaStreamSynchronize(nullptr) == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

int polymul_mod_padded_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                             int64_t Lp, void *stream) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    if (Lp < n || (Lp & (Lp - 1))) return POLY_EINVAL;
    const int l = ceil_log2(Lp);
    if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    keep_pool_memory();
    if (validation_on()) {
        u32 root = 0;
        int rc = validate_prime(p, &root);
        if (!rc) rc = validate_coeffs(p, a, za, b, zb, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return run_product(p, 0, a, za, b, zb, c, l, false, (cudaStream_t)stream, nullptr);
}

// Host-buffer products on `st`, asynchronous: small ones in place where the
// device walks the host page tables, the others staged through a
// stream-ordered device buffer.  Pinned host buffers move by the copy
// engines (they leave every SM to the products that run meanwhile on other
// streams); pageable ones by the all-SM copy kernels where the device can
// address them, else by the runtime's staged copies.
static int host_product_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                              cudaStream_t st) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    keep_pool_memory();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLY_ECUDA;
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    const bool in_place = host_memory_in_place(dev);
    if (in_place && n <= HOST_IN_PLACE_MAX_N) return polymul_mod_async(p, a, da, b, db, c, st);
    auto pinned = [](const void *ptr) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeHost;
    };
    const bool pin_in = pinned(a) && pinned(b), pin_out = pinned(c);
    // staging buffers at 16-byte boundaries (vector copies)
    const int64_t za4 = (za + 3) & ~(int64_t)3, zb4 = (zb + 3) & ~(int64_t)3;
    u32 *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, (size_t)(za4 + zb4 + n) * 4, st) != cudaSuccess) return POLY_ENOMEM;
    u32 *da_ = buf, *db_ = buf + za4, *dc_ = buf + za4 + zb4;
    int rc = POLY_OK;
    if (in_place && !pin_in) {
        if (launch_copy_words(a, da_, za, b, db_, zb, st) != cudaSuccess) rc = POLY_ECUDA;
    } else if (cudaMemcpyAsync(da_, a, (size_t)za * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
               cudaMemcpyAsync(db_, b, (size_t)zb * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = POLY_ECUDA;
    }
    if (!rc) rc = polymul_mod_async(p, da_, da, db_, db, dc_, st);
    if (!rc) {
        if (in_place && !pin_out) {
            if (launch_copy_words(dc_, c, n, nullptr, nullptr, 0, st) != cudaSuccess) rc = POLY_ECUDA;
        } else if (cudaMemcpyAsync(c, dc_, (size_t)n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = POLY_ECUDA;
        }
    }
    if (cudaFreeAsync(buf, st) != cudaSuccess && !rc) rc = POLY_ECUDA;
    return rc;
}

int polymul_mod_host_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                           void *stream) {
    return host_product_async(p, a, da, b, db, c, (cudaStream_t)stream);
}

int polymul_mod_host(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    static thread_local cudaStream_t st = nullptr;
    static thread_local int st_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLY_ECUDA;
    if (!st || st_dev != dev) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return POLY_ECUDA;
        st_dev = dev;
    }
    int rc = host_product_async(p, a, da, b, db, c, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = POLY_ECUDA;
    return rc;
}

// ---------------------------------------------------------------- TFT plans
struct tft_plan {
    uint32_t p, root;
    int64_t z, n, L;
    int l;
    PrimeCtx *ctx;
    std::vector<ItftStep> steps;  // element-level ITFT(L, n, n)
};

int tft_plan_create(uint32_t p, uint32_t root, int64_t z, int64_t n, tft_plan **out) {
    if (!out) return POLY_ENULL;
    *out = nullptr;
    if (z < 1 || n < z) return POLY_EINVAL;
    const int l = ceil_log2(n);
    if (l > POLY_MAX_LOG_L) return POLY_ETOO_LONG;
    int rc = validate_prime(p, &root);
    if (rc) return rc;
    PrimeCtx *ctx = nullptr;
    rc = get_prime(p, root, l, &ctx, nullptr);
    if (rc) return rc;
    tft_plan *pl = new tft_plan();
    pl->p = p;
    pl->root = root;
    pl->z = z;
    pl->n = n;
    pl->l = l;
    pl->L = (int64_t)1 << l;
    pl->ctx = ctx;
    pl->steps = itft_steps(ctx, pl->L, n, false);
    *out = pl;
    return POLY_OK;
}

int64_t tft_plan_length(const tft_plan *plan) { return plan ? plan->L : 0; }

void tft_plan_destroy(tft_plan *plan) { delete plan; }

int tft_exec(const tft_plan *pl, const uint32_t *in, uint32_t *out, void *stream) {
    if (!pl || !in || !out) return POLY_ENULL;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_memory();
    PrimeCtx *ctx = pl->ctx;
    u32 *x = nullptr;
    if (cudaMallocAsync((void **)&x, (size_t)pl->L * 4, st) != cudaSuccess) return POLY_ENOMEM;
    cudaError_t e = launch_copy_pad(in, pl->z, x, pl->L, st);
    for (int s = 0; s < pl->l && e == cudaSuccess; ++s)
        e = launch_fwd_level(ctx->lazy, x, pl->L, s, pl->n, pl->z, ctx->m, ctx->tw, st);
    if (e == cudaSuccess) e = launch_finish(ctx->lazy, x, out, pl->n, make_uint2(0, 0), 0, ctx->m, st);
    cudaFreeAsync(x, st);
    return e == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

int itft_exec(const tft_plan *pl, const uint32_t *in, uint32_t *out, int scale, void *stream) {
    if (!pl || !in || !out) return POLY_ENULL;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_memory();
    PrimeCtx *ctx = pl->ctx;
    u32 *x = nullptr;
    if (cudaMallocAsync((void **)&x, (size_t)pl->L * 4, st) != cudaSuccess) return POLY_ENOMEM;
    cudaError_t e = launch_copy_pad(in, pl->n, x, pl->L, st);
    for (size_t i = 0; i < pl->steps.size() && e == cudaSuccess; ++i) {
        const ItftStep &sp = pl->steps[i];
        if (sp.kind == ST_FULL) {
            const int lm = ceil_log2(sp.h);
            for (int s = sp.s + lm - 1; s >= sp.s && e == cudaSuccess; --s)
                e = launch_inv_level(ctx->lazy, x, s, sp.base, sp.h, sp.s, sp.i, ctx->m, ctx->tw, st);
        } else {
            e = launch_step(ctx->lazy, sp, x, ctx->m, st);
        }
    }
    // n == L: one unscaled full inverse (L times g); otherwise g itself.
    const u32 p = pl->p;
    const bool full = pl->n == pl->L;
    uint2 sc = make_uint2(1, 0);
    int apply = 0;
    if (full && scale) {
        sc = shoup_pair(h_invmod((u32)(pl->L % p), p), p);
        apply = 1;
    } else if (!full && !scale) {
        sc = shoup_pair((u32)(pl->L % p), p);
        apply = 1;
    }
    if (e == cudaSuccess) e = launch_finish(ctx->lazy, x, out, pl->n, sc, apply, ctx->m, st);
    cudaFreeAsync(x, st);
    return e == cudaSuccess ? POLY_OK : POLY_ECUDA;
}

}  // extern "C"
