// host.h -- host-side runtime state shared by the C ABI translation units.
#pragma once
#include <map>
#include <utility>
#include <vector>

#include "internal.h"

namespace pm {

// Single products (polymul_mod_async and the entry points built on
// run_product) with L <= 2^SINGLE_SMALL_MAX_LOG_L run on the one-CTA kernel;
// longer ones on the three-kernel path, which spreads even a 1024-point
// product over the whole GPU and measured faster than the one-cluster kernel
// from L = 1024 up (CUDA graph of back-to-back products: 4.7 against 6.6 us
// at L = 2048, 5.7 against 8.6 us at L = 8192).  Where many products
// overlap on the GPU, one launch on a few SMs per small product leaves the
// rest of the GPU to the others: batches keep one CTA per product and the
// server one cluster per product up to SMALL_MAX_LOG_L.
constexpr int SINGLE_SMALL_MAX_LOG_L = SMALL_LOG_S;

// Per (device, prime, primitive root): resident twiddle tables and cached
// ITFT step lists.  Created on first use, never freed before process exit.
struct PrimeCtx {
    u32 p = 0, root = 0;
    int v2 = 0;  // 2-adic order of p-1
    bool lazy = false;
    ModParams m{};
    TwTables tw{};
    uint2 *fwd = nullptr, *inv = nullptr;
    uint2 *pscale = nullptr;  // 32 Shoup pairs of 2^32 * 2^-e
    std::vector<uint2 *> retired;
    std::map<std::pair<int64_t, int64_t>, std::pair<const ItftStep *, int>> steps;
    // Step lists live in device arenas filled through a private stream, so
    // building one never synchronises the device.
    std::vector<ItftStep *> arenas;
    size_t arena_used = 0, arena_cap = 0;
    cudaStream_t upload = nullptr;
};

// Records the last failing CUDA call of this thread (see polymul_last_error)
// and returns POLY_ECUDA.
int cuda_fail(cudaError_t e, const char *where);

// Auxiliary streams of the calling host thread on the current device, for
// entry points that fork independent products off the caller's stream and
// join them back (the three primes algorithm, the general radix): non-
// blocking streams, a fork event and one join event per stream.  Created on
// first use, kept until the process exits.
constexpr int AUX_STREAMS = 3;
struct AuxStreams {
    int dev = -1;
    cudaStream_t s[AUX_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[AUX_STREAMS] = {};
};
int aux_streams(AuxStreams **out);

// The device's default stream-ordered pool keeps memory it has grown to
// (release threshold = unlimited), so a transient allocation does not map
// and unmap memory at every synchronisation.  Once per process.
void keep_pool_memory();

u32 h_powmod(u64 b, u64 e, u32 p);
u32 h_invmod(u32 a, u32 p);
uint2 shoup_pair(u32 w, u32 p);
int ceil_log2(int64_t n);

int validate_prime(u32 p, u32 *root);
// Validation mode (polymul_set_validate): whether it is on, and the check of
// a[0..za) and b[0..zb) against p on stream st (synchronous; POLY_OK when
// validation is off).  Null operands are skipped.
bool validation_on();
int validate_coeffs(u32 p, const u32 *a, int64_t za, const u32 *b, int64_t zb, cudaStream_t st);
int get_prime(u32 p, u32 root, int need_l, PrimeCtx **out, cudaStream_t st);
// prescaled: the spectral rows arrive multiplied by 1/h for their FULL
// record (the product paths fold that into the pointwise constant), so the
// records carry h^-1 = 1; otherwise (tft plans) h^-1 is the true inverse.
std::vector<ItftStep> itft_steps(PrimeCtx *ctx, int64_t M, int64_t k, bool prescaled);
// The pointwise constants 2^32 * 2^-e mod p, e = 0..31.
std::vector<uint2> pscale_table(u32 p);
int get_steps(PrimeCtx *ctx, int64_t T, int64_t k, const ItftStep **d_steps, int *nsteps);

Schedule default_schedule(int l);
bool schedule_valid(int l, Schedule s);
Schedule schedule_for(int l);
void set_schedule(int l, Schedule s);
std::map<int, Schedule> all_schedules();

Geometry make_geometry(int64_t n, int l, int sigma);
uint2 scale_const(u32 p, u64 scale);

// n_out: the number of output coefficients; < 0 for the linear product's
// za + zb - 1.  n_out = L (with za, zb <= L) gives the product mod x^L - 1
// (the full transform, Eq. 11).
int prepare_small(PrimeCtx *ctx, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                  SmallDesc *d, int64_t n_out = -1);
int prepare_large(PrimeCtx *ctx, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                  Schedule sch, LargeDesc *d, int64_t n_out = -1);
int64_t large_workspace_words(int64_t n, int l, Schedule sch, bool prune);
// small_max_l: the largest log2 L that runs on the one-CTA / one-cluster
// kernel (the public single-product entry points use SINGLE_SMALL_MAX_LOG_L;
// the server, whose requests overlap on the GPU, SMALL_MAX_LOG_L).
int run_product(u32 p, u32 root, const u32 *a, int64_t za, const u32 *b, int64_t zb, u32 *c, int l, bool prune,
                cudaStream_t st, u32 *workspace, int64_t n_out = -1, int small_max_l = SINGLE_SMALL_MAX_LOG_L);

}  // namespace pm
