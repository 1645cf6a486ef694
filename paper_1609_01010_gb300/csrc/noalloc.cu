// noalloc.cu -- polymul_mod_noalloc_async: the product for callers that must
// not have the library allocate device memory.
//
// Everything this entry point touches on the device lives in file-scope
// static __device__ arrays, which the CUDA runtime allocates when it loads
// the library's module on a device and keeps until the process exits:
//   g_na_scratch  the workspace of the three-kernel path (rows of both
//                 operands' column stages, then the product's rows);
//   g_na_tw       the twiddle tables of the two built-in primes;
//   g_na_steps    the ITFT step lists of every (T, k) the entry point can meet;
//   g_na_pow      power tables used once to build the twiddles;
//   g_na_pscale   the pointwise scale constants of the two primes.
// In host code a static __device__ array's name is only a host-side
// stand-in, so the device addresses are fetched once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "host.h"
#include "polymul.h"

namespace pm {

cudaError_t launch_build_tw(uint2 *fwd, uint2 *inv, int lmax, u32 p, const u32 *pw_lo, const u32 *pw_hi,
                            cudaStream_t st);

constexpr int NA_MAX_LOG_L = 17;                       // n <= 2^17 coefficients
constexpr int NA_SIGMA = 10;                           // rows of 1024 words above L = 8192
constexpr int NA_C = 32;                               // column tiles of 32 words
constexpr size_t NA_SCRATCH_WORDS = (size_t)2 << NA_MAX_LOG_L;  // 2 k S <= 2 L words (1 MiB)
constexpr size_t NA_TW_ENTRIES = (size_t)1 << NA_MAX_LOG_L;      // per prime and direction
constexpr size_t NA_MAX_STEPS = 8192;
constexpr int NA_POW_HI = (int)(((size_t)1 << NA_MAX_LOG_L) / 4096 + 2);
constexpr u32 NA_PRIMES[2] = {469762049u, 2013265921u};

static __device__ __align__(256) uint32_t g_na_scratch[NA_SCRATCH_WORDS];
static __device__ __align__(256) uint2 g_na_tw[2 * 2 * NA_TW_ENTRIES];  // prime x {fwd, inv}
static __device__ __align__(256) ItftStep g_na_steps[NA_MAX_STEPS];
static __device__ __align__(256) uint32_t g_na_pow[2 * (4096 + NA_POW_HI)];
static __device__ __align__(256) uint2 g_na_pscale[2 * 32];

struct NaDevice {
    bool ready = false;
    u32 *scratch = nullptr;
    uint2 *tw = nullptr;
    ItftStep *steps = nullptr;
    uint2 *pscale = nullptr;
    std::map<std::pair<int64_t, int64_t>, std::pair<int, int>> lists[2];  // (T, k) -> (offset, count)
};

static std::mutex g_na_mu;
static std::map<int, NaDevice> g_na_dev;

static ModParams na_params(u32 p) {
    ModParams m;
    m.p = p;
    u32 x = p;
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    m.pinv = x;
    return m;
}

// One-time set-up on the current device: symbol addresses, twiddle tables and
// step lists written into the static arrays.  No allocation of any kind.
static int na_setup(int dev, NaDevice &D) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    D.scratch = (u32 *)ptr;
    e = cudaGetSymbolAddress(&ptr, g_na_tw);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(twiddles)");
    D.tw = (uint2 *)ptr;
    e = cudaGetSymbolAddress(&ptr, g_na_steps);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(steps)");
    D.steps = (ItftStep *)ptr;
    e = cudaGetSymbolAddress(&ptr, g_na_pow);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(powers)");
    u32 *pow_dev = (u32 *)ptr;
    e = cudaGetSymbolAddress(&ptr, g_na_pscale);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scales)");
    D.pscale = (uint2 *)ptr;

    std::vector<ItftStep> all;
    for (int pi = 0; pi < 2; ++pi) {
        const u32 p = NA_PRIMES[pi];
        u32 root = 0;
        if (validate_prime(p, &root)) return POLY_EINVAL_PRIME;
        // twiddles: psi = root^((p-1)/2^lmax), powers psi^a (a < 4096), psi^(4096 b)
        const int lmax = NA_MAX_LOG_L;
        const u32 psi = h_powmod(root, (u64)(p - 1) >> lmax, p);
        std::vector<u32> pw(4096 + NA_POW_HI);
        u64 x = 1;
        for (int a = 0; a < 4096; ++a) {
            pw[a] = (u32)x;
            x = x * psi % p;
        }
        const u32 step = h_powmod(psi, 4096, p);
        x = 1;
        for (int b = 0; b < NA_POW_HI; ++b) {
            pw[4096 + b] = (u32)x;
            x = x * step % p;
        }
        u32 *pw_dev = pow_dev + (size_t)pi * (4096 + NA_POW_HI);
        e = cudaMemcpy(pw_dev, pw.data(), pw.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "power tables");
        uint2 *fwd = D.tw + (size_t)pi * 2 * NA_TW_ENTRIES, *inv = fwd + NA_TW_ENTRIES;
        e = launch_build_tw(fwd, inv, lmax, p, pw_dev, pw_dev + 4096, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "twiddle build");
        const std::vector<uint2> ps = pscale_table(p);
        e = cudaMemcpy(D.pscale + pi * 32, ps.data(), 32 * sizeof(uint2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "scale table");
        // step lists: one-CTA path (T = 1..16 rows of 512) and three-kernel path
        // (rows of 2^NA_SIGMA, T = 16..128)
        PrimeCtx tmp;
        tmp.p = p;
        tmp.root = root;
        auto add = [&](int64_t T, int64_t k) {
            std::vector<ItftStep> v = itft_steps(&tmp, T, k, true);
            D.lists[pi][std::make_pair(T, k)] = std::make_pair((int)all.size(), (int)v.size());
            all.insert(all.end(), v.begin(), v.end());
        };
        for (int logT = 0; logT <= SMALL_MAX_LOG_T; ++logT)
            for (int64_t k = 1; k <= ((int64_t)1 << logT); ++k) add((int64_t)1 << logT, k);
        for (int l = SMALL_MAX_LOG_L + 1; l <= NA_MAX_LOG_L; ++l) {
            const int64_t T = (int64_t)1 << (l - NA_SIGMA);
            for (int64_t k = T / 2 + 1; k <= T; ++k) add(T, k);
        }
    }
    if (all.size() > NA_MAX_STEPS) return POLY_ENOMEM;
    e = cudaMemcpy(D.steps, all.data(), all.size() * sizeof(ItftStep), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "step lists");
    // A copy from pageable host memory may return once the data is staged,
    // before it has landed in g_na_steps; the caller's stream may be a
    // non-blocking one that does not wait for the legacy stream.  Wait here.
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "step lists");
    (void)dev;
    D.ready = true;
    return POLY_OK;
}

// The step list recorded for (T, k) of prime pi, or false if set-up did not
// record one (a geometry outside the ranges na_setup enumerates).
static bool na_list(const NaDevice &D, int pi, int64_t T, int64_t k, std::pair<int, int> *out) {
    auto it = D.lists[pi].find(std::make_pair(T, k));
    if (it == D.lists[pi].end()) return false;
    *out = it->second;
    return true;
}

}  // namespace pm

using namespace pm;

static int noalloc_body(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                        void *stream) {
    if (!a || !b || !c) return POLY_ENULL;
    if (da < 0 || db < 0) return POLY_EINVAL;
    const int pi = p == NA_PRIMES[0] ? 0 : (p == NA_PRIMES[1] ? 1 : -1);
    if (pi < 0) return POLY_EINVAL_PRIME;
    // da + db + 1 <= 2^17 checked before any addition (no signed overflow)
    if (da >= ((int64_t)1 << NA_MAX_LOG_L) || db >= ((int64_t)1 << NA_MAX_LOG_L) - da) return POLY_ETOO_LONG;
    const int64_t za = da + 1, zb = db + 1, n = za + zb - 1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    NaDevice *D;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        D = &g_na_dev[dev];
        if (!D->ready) {
            int rc = na_setup(dev, *D);
            if (rc) return rc;
        }
    }
    const ModParams m = na_params(p);
    const bool lazy = p < (1u << 30);
    TwTables tw;
    tw.fwd = D->tw + (size_t)pi * 2 * NA_TW_ENTRIES;
    tw.inv = tw.fwd + NA_TW_ENTRIES;
    tw.lmax = NA_MAX_LOG_L;
    tw.pscale = D->pscale + pi * 32;
    tw.status = device_status_ptr();
    const int l = ceil_log2(n);
    cudaStream_t st = (cudaStream_t)stream;
    if (l <= SMALL_MAX_LOG_L) {
        const int lp = l < SMALL_LOG_S ? SMALL_LOG_S : l;
        const int logT = lp - SMALL_LOG_S;
        const int64_t T = (int64_t)1 << logT, S = (int64_t)1 << SMALL_LOG_S;
        const int64_t k = (n + S - 1) / S;
        std::pair<int, int> ls;
        if (!na_list(*D, pi, T, k, &ls)) return POLY_EINVAL;
        SmallDesc d;
        d.a = a;
        d.b = b;
        d.c = c;
        d.za = za;
        d.zb = zb;
        d.n = n;
        d.logT = logT;
        d.k = (int32_t)k;
        d.steps = D->steps + ls.first;
        d.nsteps = ls.second;
        d.prune = 1;
        e = launch_small(lazy, logT, nullptr, &d, 1, m, tw, st);
        return e == cudaSuccess ? POLY_OK : cuda_fail(e, "one-CTA product launch");
    }
    const Geometry g = make_geometry(n, l, NA_SIGMA);
    std::pair<int, int> ls;
    if (!na_list(*D, pi, g.T, g.k, &ls)) return POLY_EINVAL;
    LargeDesc d;
    d.a = a;
    d.b = b;
    d.c = c;
    d.wa = D->scratch;
    d.wb = D->scratch + g.k * g.S;
    d.za = za;
    d.zb = zb;
    d.n = n;
    d.g = g;
    d.steps = D->steps + ls.first;
    d.nsteps = ls.second;
    d.prune = 1;
    e = launch_large(lazy, d, Schedule{NA_SIGMA, NA_C}, m, tw, st);
    return e == cudaSuccess ? POLY_OK : cuda_fail(e, "three-kernel product launch");
}

extern "C" int polymul_mod_noalloc_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                                         uint32_t *c, void *stream) {
    // No C++ exception may leave an extern "C" function: the host-side maps
    // of the first call's set-up can throw std::bad_alloc.
    try {
        return noalloc_body(p, a, da, b, db, c, stream);
    } catch (const std::bad_alloc &) {
        return POLY_ENOMEM;
    } catch (...) {
        return POLY_EINVAL;
    }
}
