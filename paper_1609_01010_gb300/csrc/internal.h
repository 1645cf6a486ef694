// internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace pm {

typedef uint64_t u64;

// ---------------------------------------------------------------- twiddles
// One table per prime, shared by every transform length L <= 2^lmax.
// Node i (0 <= i < 2^s) at depth s of the merged Cooley-Tukey tree of any
// power-of-two length splits x^M - r^2 into (x^{M/2} - r)(x^{M/2} + r) with
//     r = psi_{s+1}^{rev_s(i)},   psi_k = g^((p-1)/2^k),
// independent of L.  Entry 2^s + i holds (r, floor(r 2^32/p)); the inverse
// table holds r^-1.  Leaves of a length-L tree are then g(w^{rev_l(i)}) with
// w = g^((p-1)/L): the TFT's bit-reversed output order.
struct TwTables {
    const uint2 *fwd;
    const uint2 *inv;
    int lmax;             // entries [1, 2^lmax) are valid
    const uint2 *pscale;  // pscale[e] = Shoup pair of 2^32 * 2^-e mod p, e < 32
    int *status = nullptr;  // the device status word (bounded waits record POLY_ETIMEOUT)
};

// The device status word of the current device (a static device variable of
// the library; its address is fetched once per device).  NULL on failure.
int *device_status_ptr();

__host__ __device__ inline uint32_t tw_index(int level, uint32_t node) { return (1u << level) + node; }

// ------------------------------------------------------------- ITFT steps
// In-place truncated inverse of one node of size M (in rows) given the first
// k leaves (spectral values) and known coefficients beyond k; see
// itft_steps() in host.cu for the recursion these records encode.
enum StepKind : int32_t {
    ST_FULL = 0,       // unscaled inverse of subtree (s, i) over rows [base, base+h)
    ST_PRE_RIGHT = 1,  // j in [m, h): c_j = X_j/h - r X_{j+h}; X_j = c_j; X_{j+h} = c_j - r X_{j+h}
    ST_POST_RIGHT = 2, // j < m: u = X_j/h; X_j = (u + X_{j+h})/2; X_{j+h} = (u - X_{j+h})/(2r)
    ST_PRE_LEFT = 3,   // j in [m, h): X_j += r X_{j+h}
    ST_POST_LEFT = 4,  // j < m: X_j -= r X_{j+h}
};

struct ItftStep {
    int32_t kind;
    int32_t zero;  // PRE_RIGHT only: the known upper coefficients are all zero
    int32_t s;     // depth of the node (for ST_FULL: of the subtree root)
    uint32_t i;    // node index at depth s
    int32_t base;  // first row of the node
    int32_t h;     // half size (ST_FULL: subtree size)
    int32_t m;     // range bound (see kinds)
    int32_t pad;
    uint2 r;       // node twiddle psi_{s+1}^{rev_s(i)}
    uint2 hinv;    // h^-1
    uint2 inv2;    // 2^-1
    uint2 i2r;     // (2r)^-1
};

// ------------------------------------------------------------ geometry
// Block-relaxed decomposition of a length-L transform: L = T * S, rows of S
// words.  The top t = log2 T tree levels act on whole rows (the column
// stage); the bottom sigma = log2 S levels act inside one row (row stage).
// Truncation is applied at row granularity: k >= ceil(n / S) rows are computed.
struct Geometry {
    int l, t, sigma;
    int64_t L, S, T, k, n;
};

// Small products: one CTA, rows of 512 words, T <= 16 (L <= 8192).
constexpr int SMALL_LOG_S = 9;
constexpr int SMALL_MAX_LOG_T = 4;
constexpr int SMALL_MAX_LOG_L = SMALL_LOG_S + SMALL_MAX_LOG_T;

// Large products: rows of S = 2^sigma (9..13) words handled by one CTA each,
// column tiles of C words handled by one CTA each, T <= 1024 rows.
constexpr int LARGE_MAX_LOG_T = 10;
// Rows computed by the three-kernel path: ceil(n/S) rounded up to a multiple
// of T / 2^RELAX_LOG_T (see make_geometry).
constexpr int RELAX_LOG_T = 3;

// Shared memory of one row of the row stage held E words per thread: one
// exchange buffer (S words), the row's twiddles (S entries of 8 bytes, entry
// 0 unused) and, for sigma <= 12, the 2^UL inverse twiddles of the sub-levels
// before its last pass (UL = log2(E) times the passes before the last).
inline size_t row_smem_bytes(int sigma, int E = 16) {
    const int le = E >= 16 ? 4 : (E >= 8 ? 3 : 2);
    const int ul = le * ((sigma + le - 1) / le - 1);
    return ((size_t)1 << sigma) * 4 + ((size_t)1 << sigma) * 8 + (sigma <= 12 ? ((size_t)8 << ul) : 0);
}

struct Schedule {
    int sigma;  // row-block log size
    int C;      // column tile width
};

// Raises a kernel's dynamic shared-memory limit once per (kernel, device):
// the attribute is per function and device, and setting it on every launch
// would cost a driver call per product.
cudaError_t ensure_smem_ptr(const void *kern, size_t bytes);
template <typename K>
inline cudaError_t ensure_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return ensure_smem_ptr((const void *)kern, bytes);
}

// Grid of a persistent kernel: all CTAs that fit on the device at once, at
// most `items`.
cudaError_t persistent_grid(const void *kern, int threads, size_t smem, int items, int *grid);

// ------------------------------------------------------------ launchers
// Kernels are launched only through these (defined in k_small.cu /
// k_large.cu / k_generic.cu); all return a cudaError_t of the launch.

// One CTA (or, for one product of T >= 2 rows, one cluster) per product; used
// for the products that take the small path (l < 9 is padded to 9).
struct SmallDesc {
    const uint32_t *a, *b;
    uint32_t *c;
    int64_t za, zb, n;
    int32_t logT, k;
    const ItftStep *steps;
    int32_t nsteps;
    int32_t prune;  // 0: compute every butterfly (the zero-padded comparator)
};
// d_desc: device array of `count` descriptors, or NULL to use *h_one (count 1).
cudaError_t launch_small(bool lazy, int logT, const SmallDesc *d_desc, const SmallDesc *h_one, int count,
                         ModParams m, TwTables tw, cudaStream_t st);

struct LargeDesc {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t *wa, *wb;  // workspace rows: k * S words each
    int64_t za, zb, n;
    Geometry g;
    const ItftStep *steps;
    int32_t nsteps;
    int32_t prune;  // 0: compute every butterfly (the zero-padded comparator)
};
// ev: NULL, or 4 events recorded before the column stage, after it, after
// the row stage and after the ITFT column stage (profiling).
cudaError_t launch_large(bool lazy, const LargeDesc &d, Schedule sch, ModParams m, TwTables tw, cudaStream_t st,
                         cudaEvent_t *ev = nullptr);

// Generic per-level kernels (any L): used by tft_exec / itft_exec.
cudaError_t launch_copy_pad(const uint32_t *in, int64_t z, uint32_t *x, int64_t L, cudaStream_t st);
cudaError_t launch_fwd_level(bool lazy, uint32_t *x, int64_t L, int s, int64_t n, int64_t z, ModParams m,
                             TwTables tw, cudaStream_t st);
cudaError_t launch_inv_level(bool lazy, uint32_t *x, int s, int64_t base, int64_t M, int s_root, uint32_t i_root,
                             ModParams m, TwTables tw, cudaStream_t st);
cudaError_t launch_step(bool lazy, const ItftStep &stp, uint32_t *x, ModParams m, cudaStream_t st);
cudaError_t launch_finish(bool lazy, const uint32_t *x, uint32_t *out, int64_t n, uint2 scale, int apply_scale,
                          ModParams m, cudaStream_t st);

}  // namespace pm
