/*
 * polymul.h -- C ABI of the GB300 (sm_103a) library for exact univariate
 * polynomial multiplication over Z/pZ through the truncated Fourier transform.
 *
 * The method (Meng, "Automatic Library Generation for Modular Polynomial
 * Multiplication", Section 3, Eq. (14)): with z1 = da+1, z2 = db+1,
 * n = z1+z2-1 and L = 2^l >= n,
 *     g^ = TFT(L, z1, n) g,   h^ = TFT(L, z2, n) h,   u^_i = g^_i h^_i (i < n),
 *     (L u_0, ..., L u_{n-1}) = ITFT(L, n, n) u^,
 * and u = g h (Definition 2, Eq. (2)).  This library returns u (it multiplies
 * by L^-1 mod p); itft_exec can return the paper's L*u instead.
 *
 * Conventions shared by every entry point:
 *  - Coefficients are uint32 residues, canonical in [0, p), a_i at index i
 *    (Definition 1's dense representation).  Degrees are int64 (length =
 *    degree + 1).  Inputs outside [0, p) give undefined (but memory-safe)
 *    results; outputs are always canonical.
 *  - p must be an odd prime below 2^31 with 2^k | p-1; the transform length L
 *    must divide p-1 and not exceed 2^POLY_MAX_LOG_L.  root is a primitive
 *    root of p, or 0 for the built-in table (469762049 -> 3, 2013265921 -> 31).
 *    The principal L-th root used is w = root^((p-1)/L).
 *  - L is the smallest power of two >= n (the paper only requires n <= L).
 *  - TFT outputs are in van der Hoeven's bit-reversed order:
 *    out_i = g(w^{rev_l(i)}) for i < n.
 *  - Pointers marked "device" are CUDA device (or managed) memory owned by the
 *    caller; "host" pointers are ordinary or pinned host memory.  Buffers must
 *    not alias unless stated.  Plans, twiddle tables and workspaces are owned
 *    by the library and stay resident until their destroy call (tables: until
 *    the process exits).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  *_async calls only enqueue work and return; results are valid
 *    once the stream reaches that point.
 *  - Every call returns POLY_OK (0) or a negative error code; nothing traps.
 *    Device-side waits are bounded and report POLY_ETIMEOUT.
 */
#ifndef POLYMUL_H
#define POLYMUL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define POLY_OK 0
#define POLY_EINVAL_PRIME (-1) /* p even, >= 2^31, or root not usable */
#define POLY_ETOO_LONG (-2)    /* L does not divide p-1, or L > 2^POLY_MAX_LOG_L */
#define POLY_ENULL (-3)        /* a required pointer is NULL */
#define POLY_ENOMEM (-4)       /* device or host allocation failed */
#define POLY_ECUDA (-5)        /* a CUDA runtime call failed */
#define POLY_ETIMEOUT (-6)     /* a bounded device or host wait expired */
#define POLY_EINVAL (-7)       /* a size or argument is out of range */
#define POLY_EBUSY (-8)        /* request larger than the server's memory budget */
#define POLY_ENOTFOUND (-9)    /* unknown server ticket */
#define POLY_EINVAL_COEF (-10) /* a validating call found an input coefficient outside [0, p) */
#define POLY_EDEBUG_CHECK (-11) /* debug build only: a range or index check inside a kernel failed */

#define POLY_MAX_LOG_L 24

/* Human-readable text for a status code (static storage). */
const char *polymul_strerror(int status);

/* Text of the last failing CUDA call made by this thread ("" if none). */
const char *polymul_last_error(void);

/*
 * The device status word of the current device: POLY_OK, or the first error
 * a kernel recorded since it was last cleared.  POLY_ETIMEOUT: a bounded
 * wait inside a kernel expired (that kernel skipped the work whose data
 * never arrived, so its output is not valid).  POLY_EDEBUG_CHECK: a range
 * or index check of the debug build (libpolymul_debug.so, built with
 * python -m paper_1609_01010_gb300.build --debug) failed -- a residue a
 * kernel stored outside its stated range, or an index outside its buffer.
 * clear != 0 resets it to POLY_OK after reading.  Synchronous (a
 * device-to-host copy on the legacy default stream).  POLY_ECUDA if the
 * word cannot be read.
 */
int polymul_device_status(int clear);

/*
 * Validation mode (off by default).  While on, every entry point that takes
 * modular operands -- polymul_mod[_async], polymul_mod_padded_async,
 * polymul_mod_host, polymul_cyclic_async, polymul_negacyclic_async,
 * polymul_mod_radix_async, polymul_batch_exec[_nograph],
 * polymul_mod_batched[_plain] and polymul_server_submit -- first checks with
 * one pass over a and b that every coefficient lies in [0, p), and returns
 * POLY_EINVAL_COEF (computing nothing, c untouched) if one does not.  The
 * check synchronises the caller's stream (the server's submit: the legacy
 * default stream), so it is meant for debugging and for callers whose inputs
 * are untrusted.  polymul_mod_noalloc_async and polymul_crt3_async (whose
 * inputs are arbitrary 32-bit words) are never checked.  Process-wide.
 */
int polymul_set_validate(int on);

/* Library version string. */
const char *polymul_version(void);

/*
 * c = a * b mod p (Section 3, Eq. (14)).
 *   a: device, da+1 words; b: device, db+1 words; c: device, da+db+1 words.
 * polymul_mod is synchronous on the legacy default stream.
 * polymul_mod_async enqueues on `stream`; its workspace comes from the
 * stream-ordered allocator and is released on the same stream.
 */
int polymul_mod(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c);
int polymul_mod_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                      uint32_t *c, void *stream);

/*
 * The zero-padded comparator of Eq. (12): both operands zero-padded to Lp
 * (a power of two >= da+db+1), full size-Lp modular DFTs (no pruning of zero
 * inputs or of outputs), pointwise product, full inverse.  c as above.
 */
int polymul_mod_padded_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                             uint32_t *c, int64_t Lp, void *stream);

/*
 * Host-buffer form: a, b, c are host pointers (pinned or pageable).
 * Synchronous, on an internal stream.  Where the device walks the host's
 * page tables (address translation services; GB300 with a Grace host, over
 * NVLink-C2C), products with da+db+1 <= 2^19 are computed on the host
 * buffers in place.  Larger ones are staged through a stream-ordered device
 * buffer: pinned buffers by the copy engines, pageable ones by copy kernels
 * on all SMs where the device can address them, else by the runtime's
 * staged copies.
 */
int polymul_mod_host(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c);

/*
 * The host-buffer product enqueued on `stream` without waiting: the same
 * paths as polymul_mod_host.  a and b must stay valid and unchanged, and c
 * untouched, until the stream has passed this call's work (synchronise the
 * stream or an event recorded after the call).  A caller with many products
 * spreads them over a few streams so that one product's host-link copies run
 * while another computes.
 */
int polymul_mod_host_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c,
                           void *stream);

/*
 * Allocation-free product for callers that cannot let a library allocate
 * device memory: applications that reserve all device memory up front in
 * their own pool (a library cudaMalloc would fail or bypass their
 * accounting), and latency-critical callers that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.  The paper has
 * no counterpart; it is a deployment variant of polymul_mod_async.
 *
 * Same result as polymul_mod_async (a, b, c: device buffers of da+1, db+1,
 * da+db+1 words), computed with the same kernels, but the three-kernel
 * path's workspace is a 1 MiB static device array inside the library (and the
 * twiddle tables and step lists it needs are static arrays too: about 5.5 MiB
 * in total, held by every GPU that loads the library until the process
 * exits).  This call makes no device allocation: it never calls
 * cudaMalloc, cudaMallocAsync, cudaFree or a library routine that allocates
 * device memory.  (Its first call on a device fills small host-side lookup
 * tables; that is ordinary host memory.)  It records no profile events
 * (polymul_profile_begin/end do not see its kernels).
 *  - p must be 469762049 or 2013265921 (else POLY_EINVAL_PRIME).
 *  - n = da+db+1 must not exceed 131072 = 2^17 (else POLY_ETOO_LONG).
 *  - The first call on a device sets the static tables up (with that device
 *    current, synchronising the legacy default stream); make it before any
 *    stream capture.
 *  - All calls share the one workspace, which keeps the last call's
 *    contents (nothing in it needs to start at zero): calls whose work
 *    overlaps on the GPU (e.g. on different streams) race and give wrong
 *    results.  Serialise them on one stream.
 */
int polymul_mod_noalloc_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                              uint32_t *c, void *stream);

/*
 * Measurement helpers.  Between polymul_profile_begin and polymul_profile_end
 * every single-product call (except polymul_mod_noalloc_async) records CUDA
 * events around its kernels on its
 * stream.  polymul_profile_end synchronises those events and returns the
 * summed device time in milliseconds and the number of launches per kernel:
 * index 0 the one-CTA product kernel (L <= 512), 1 the TFT column stage,
 * 2 the row stage (forward, pointwise, inverse), 3 the ITFT column stage.
 */
int polymul_profile_begin(void);
int polymul_profile_end(double *ms4, int64_t *launches4);

/*
 * Measured integer-pipe peak of the current device (a diagnostic with no
 * counterpart in the paper: the denominator of the transform kernels'
 * roofline).  Runs one probe kernel of `iters` loop iterations at full
 * occupancy: 16 independent register accumulators per thread, no memory
 * traffic in the loop.  kind 0: the lazy forward butterfly (the transform
 * kernels' instruction mix, 3 multiplies per butterfly); 1: the lazy inverse
 * butterfly; 2: mul.lo.u32; 3: mul.hi.u32; 4: add.u32; 5: min.u32.
 * *ops_per_s: butterflies per second (kinds 0, 1) or instructions per second
 * (2..5), from CUDA events around the timed launch (after one warm-up
 * launch); *ms: that launch's duration.  Allocates and frees a small output
 * buffer.  POLY_EINVAL for an unknown kind or iters outside [1, 2^24].
 */
int polymul_probe_int(int kind, int iters, double *ops_per_s, double *ms);

/*
 * Cyclic convolution: c = a * b mod (x^N - 1), c_k = sum over i + j = k mod N
 * of a_i b_j (Definition 4, Eq. 5), N >= 1 words in c.  a and b are given by
 * their lengths za, zb (1 <= za, zb <= N), device buffers owned by the caller;
 * coefficients in [0, p).  A power-of-two N >= 512 runs as Eq. 11 (transform
 * of length N, pointwise product, inverse); any other N computes the linear
 * product and folds it (a transient workspace of za + zb - 1 words from the
 * stream-ordered pool).  POLY_EINVAL for lengths outside [1, N].
 */
int polymul_cyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb, uint32_t *c,
                         int64_t N, void *stream);

/*
 * Negacyclic convolution: c = a * b mod (x^N + 1) (x^N = -1), the second
 * factor of Eq. 13's splitting of x^{2N} - 1.  Arguments as
 * polymul_cyclic_async.  A power-of-two N >= 512 with 2N dividing p - 1 runs
 * as a twisted cyclic convolution of length N: a_i and b_i times psi^i (psi a
 * primitive 2N-th root of unity, so x = psi y maps x^N + 1 to -(y^N - 1)),
 * the length-N transform product, and the result times psi^-i (a transient
 * workspace of za + zb words from the stream-ordered pool).  Any other N
 * computes the linear product and folds it with a sign.
 */
int polymul_negacyclic_async(uint32_t p, const uint32_t *a, int64_t za, const uint32_t *b, int64_t zb,
                             uint32_t *c, int64_t N, void *stream);

/*
 * Exact integer product of two polynomials with unsigned 32-bit coefficients,
 * by the three primes algorithm that Section 1 names as the route from
 * modular polynomial multiplication to multiplication over the integers:
 * the product modulo q0 = 469762049, q1 = 2013265921 and q2 = 754974721
 * (three TFT products, Eq. 14), recombined by the Chinese remainder theorem
 * (Garner's mixed-radix form).
 *   a: device, da+1 words, any value in [0, 2^32); b likewise (db+1 words).
 *   c: device, 3*(da+db+1) words: coefficient k of a*b over the integers is
 *      c[3k] + 2^32 c[3k+1] + 2^64 c[3k+2] (little-endian 32-bit words).
 * Exact for n = da+db+1 <= 2^24: every coefficient is below
 * min(da+1, db+1) (2^32-1)^2 < 2^87 < q0 q1 q2 (about 2^89.2).
 * POLY_ETOO_LONG beyond 2^24, POLY_EINVAL for negative degrees, POLY_ENULL for
 * null pointers.  Workspace: 3 (da+db+2) + 3 n words from the stream-ordered
 * pool, released on `stream`; the three products also take their own.
 */
int polymul_crt3_async(const uint32_t *a, int64_t da, const uint32_t *b, int64_t db, uint32_t *c, void *stream);

/*
 * c = a * b mod p with a transform length L = m 2^k that is not a power of
 * two: the general-radix TFT that Section 1 cites ([25, 27]) against the
 * power-of-two stair-case, truncated at the radix-m level as Section 5's
 * relaxed algorithms truncate.  With N = 2^k the smallest power of two
 * >= 512 with m N >= n (n = da+db+1) and zeta a primitive m-th root of
 * unity, x^L - 1 splits into the m factors x^N - zeta^j; the product is
 * computed from its residues modulo the first ceil(n / N) of them, each a
 * twisted cyclic convolution of length N (Eq. 11) on the power-of-two
 * kernels, and recombined by the inverse Vandermonde (for all m factors: the
 * inverse m-point DFT).  The result equals polymul_mod_async's exactly.
 *   a, b, c: device buffers of da+1, db+1, da+db+1 words, as polymul_mod.
 *   m: odd radix in [1, 15] dividing p-1 (for 2013265921 = 15 2^27 + 1:
 *      3, 5, 15; for 469762049 = 7 2^26 + 1: 7); m = 1 is polymul_mod_async.
 * POLY_EINVAL for an even m, m > 15 or m not dividing p-1; POLY_ETOO_LONG if
 * m 2^k does not divide p-1 or N > 2^23.  Workspace: 3 ceil(n/N) N words
 * from the stream-ordered pool, plus twist tables resident per (p, m, k).
 */
int polymul_mod_radix_async(uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b, int64_t db,
                            uint32_t *c, int m, void *stream);

/* ---------------------------------------------------------------- TFT plans */
typedef struct tft_plan tft_plan;

/*
 * Plan for TFT(L, z, n) / ITFT(L, n, n) with L = smallest power of two >= n
 * (Section 3).  Requires 1 <= z <= n.  One plan owns both directions, so the
 * inverse mirrors the forward decomposition.
 */
int tft_plan_create(uint32_t p, uint32_t root, int64_t z, int64_t n, tft_plan **out);

/* Transform length L of a plan (0 for NULL). */
int64_t tft_plan_length(const tft_plan *plan);

/* out[0..n) = TFT(L, z, n) in[0..z).  in, out: device; must not alias. */
int tft_exec(const tft_plan *plan, const uint32_t *in, uint32_t *out, void *stream);

/*
 * out[0..n) = ITFT(L, n, n) in[0..n): the g of degree < n with
 * TFT(L, g, n) = in.  scale = 1 returns g; scale = 0 returns L*g, the form
 * Section 3 states.  in, out: device; must not alias.
 */
int itft_exec(const tft_plan *plan, const uint32_t *in, uint32_t *out, int scale, void *stream);

void tft_plan_destroy(tft_plan *plan);

/* ---------------------------------------------------------------- batched */
typedef struct polymul_batch polymul_batch;

/*
 * Plan for `count` independent products mod p packed back to back:
 * operand i of a occupies a[a_off[i] .. a_off[i+1]) (length = degree+1 >= 1),
 * likewise b with b_off, and product i is written to c[c_off[i] ..
 * c_off[i] + len_a + len_b - 1).  The offset arrays are HOST arrays of
 * count+1 int64 entries; the plan copies them.  A product with L <= 8192 is
 * one work item; a longer one is split into column, row and ITFT items with
 * rows of 2^12 words (one 256-thread CTA per row, fixed by the kernel's CTA
 * shape) and column tiles of the width its size class (log2 L) has in the
 * tuned table -- polymul_autotune times a batch of each length at every
 * width, polymul_load_schedules reads it back ("batch_C") -- or, untuned, a
 * built-in rule (polymul_get_batch_width).
 */
int polymul_batch_create(uint32_t p, int64_t count, const int64_t *a_off, const int64_t *b_off,
                         const int64_t *c_off, polymul_batch **out);

/*
 * Run the batch on device buffers a, b, c as one persistent kernel launch,
 * replayed from a CUDA graph instantiated for this (a, b, c, stream) and
 * cached in the plan.  Asynchronous on `stream`.
 */
int polymul_batch_exec(polymul_batch *batch, const uint32_t *a, const uint32_t *b, uint32_t *c, void *stream);

/* Same work without the graph: the persistent kernel launched directly. */
int polymul_batch_exec_nograph(polymul_batch *batch, const uint32_t *a, const uint32_t *b, uint32_t *c,
                               void *stream);

/* Status of the last finished run (POLY_ETIMEOUT if a bounded wait expired).
 * Synchronises with the batch's last launch. */
int polymul_batch_status(polymul_batch *batch);

void polymul_batch_destroy(polymul_batch *batch);

/*
 * Test hook for the bounded waits: removes the first work item of `kind`
 * (0 one-CTA product, 1 column item, 2 row item, 3 ITFT column item) from the
 * batch's device work list and sets the wait limit to spin_limit polls of
 * ~128 ns.  The next exec then has an item whose wait cannot be met; it must
 * return POLY_ETIMEOUT through polymul_batch_status, not hang.  kind < 0
 * restores the list and the default limit.  Use only on a non-graph exec
 * (polymul_batch_exec_nograph).
 */
int polymul_batch_test_withhold(polymul_batch *batch, int kind, long long spin_limit);

/*
 * One-shot convenience: create, exec and destroy (synchronous on `stream`).
 * Offsets are host arrays as in polymul_batch_create.
 */
int polymul_mod_batched(uint32_t p, int64_t count, const uint32_t *a, const int64_t *a_off, const uint32_t *b,
                        const int64_t *b_off, uint32_t *c, const int64_t *c_off, void *stream);

/*
 * The plain comparator for a batch: one polymul_mod_async call (its own
 * launches) per product, in order, on `stream`.
 */
int polymul_mod_batched_plain(uint32_t p, int64_t count, const uint32_t *a, const int64_t *a_off,
                              const uint32_t *b, const int64_t *b_off, uint32_t *c, const int64_t *c_off,
                              void *stream);

/* ---------------------------------------------------------------- autotuner */
/*
 * Time the candidate schedules (row block, column tile) for every
 * transform length 2^lo_log .. 2^hi_log on the current device and prime p,
 * and the batched kernel's column-tile widths for the lengths a batch splits
 * into items (2^14 .. 2^22), keep the fastest per length, and write the
 * table as JSON to `json_path` (NULL: keep in memory only).  Subsequent
 * plans use the table.
 */
int polymul_autotune(uint32_t p, int lo_log, int hi_log, const char *json_path);

/* Load a table written by polymul_autotune. */
int polymul_load_schedules(const char *json_path);

/*
 * The schedule the three-kernel path uses for L = 2^l (l in 10..24): row
 * length 2^(*sigma) and column-tile width *C (autotuned or default).  The
 * paper's counterpart is the DP search's chosen breakdown (Section 4).
 * POLY_EINVAL outside that range, POLY_ENULL for null outputs.
 */
int polymul_get_schedule(int l, int *sigma, int *C);

/*
 * Column-tile width (8, 32, 128, 256, 512, 1024 or 2048 words) of a product of length
 * L = 2^l inside a batch (l in 14..22): tuned or built-in (the widest tile
 * of T x C words that fits 64 KB).  POLY_EINVAL outside that range.
 */
int polymul_get_batch_width(int l, int *C);

/* ---------------------------------------------------------------- serving */
typedef struct polymul_server polymul_server;

/* Dispatch modes of the server. */
#define POLY_SERVE_BATCH 0 /* serving form: small requests (L <= 2^17) on a high-priority lane, batched in one persistent launch when 2 or more, the rest plain */
#define POLY_SERVE_PLAIN 1 /* every request as its own plain product (the comparator) */

/*
 * A continuous-batching server on the current device (the paper has no
 * serving layer).  Requests are admitted while the bytes they hold (inputs,
 * output and workspace) fit in mem_budget_bytes; the rest wait in arrival
 * order.  A free stream (of `n_streams`) takes admissible queued requests
 * of one prime as a group and runs them as `mode` says, so work admitted while
 * other work runs overlaps on the GPU.  In POLY_SERVE_BATCH one stream in four
 * (at least one) is a high-priority lane for small requests (L <= 2^17); the
 * others take large requests first.  A scheduler thread polls the groups'
 * completion events (spinning while work is in flight or arrived within the
 * last 2 ms, so it holds a host core busy meanwhile).  Twiddle tables and plans for
 * 469762049 and 2013265921 are made resident at creation, every kernel a
 * request can meet is loaded by running zero-input products of every length
 * on the device, and the stream-ordered pool is grown to min(budget, 1 GiB)
 * (creation takes some tens of milliseconds).  POLY_EINVAL for a zero budget,
 * n_streams outside [1, 64] or an unknown mode.
 */
int polymul_server_create(size_t mem_budget_bytes, int n_streams, int mode, polymul_server **out);

/*
 * Submit c = a * b mod p.  a, b, c: device buffers owned by the caller, which
 * must stay valid and untouched until the ticket is done.  Returns at once
 * with a ticket.  POLY_EBUSY if the request alone exceeds the budget.
 */
int polymul_server_submit(polymul_server *srv, uint32_t p, const uint32_t *a, int64_t da, const uint32_t *b,
                          int64_t db, uint32_t *c, uint64_t *ticket);

/* *done = 1 once the product is in c (and its status is returned), else 0. */
int polymul_server_poll(polymul_server *srv, uint64_t ticket, int *done);

/* Block until the ticket is done or timeout_ms passes (POLY_ETIMEOUT). */
int polymul_server_wait(polymul_server *srv, uint64_t ticket, int64_t timeout_ms);

/*
 * Latency statistics of completed requests (submit -> GPU completion), in
 * microseconds: out[0..5] = {count, p50, p90, p99, max, mean}.
 */
int polymul_server_stats(polymul_server *srv, double *out6);

/* Latency (submit -> completion seen by the server, microseconds) of one done
 * ticket; POLY_EINVAL while it is not done, POLY_ENOTFOUND for an unknown one. */
int polymul_server_latency(polymul_server *srv, uint64_t ticket, double *us);

int polymul_server_destroy(polymul_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* POLYMUL_H */
