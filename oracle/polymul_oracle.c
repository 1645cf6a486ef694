/*
 * polymul_oracle.c -- plain, slow, obviously-correct CPU oracle for polynomial
 * multiplication over Z/pZ through the truncated Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) links, loads or calls this file.  It is used by tests/,
 * by __graft_entry__.smoke() and by bench.py's CPU-baseline leg, and it shares
 * no code, table or constant generator with the GPU path.
 *
 * Every routine works on canonical residues in [0, p) and reduces each
 * product with a 64-bit `%`; nothing is lazy, blocked, fused or reordered
 * beyond what the definition or the algorithm states.
 *
 * What follows from the paper (Meng, "Automatic Library Generation for
 * Modular Polynomial Multiplication"):
 *   - or_schoolbook:  Definition 2, Eq. (2): c_k = sum_{i+j=k} a_i b_j.
 *   - or_tft / or_itft: the TFT(L, z, n) and ITFT(L, n, n) of Section 3
 *     (TFT-based convolution, Eq. (14)), in van der Hoeven's bit-reversed
 *     output order.  The paper does not print the transforms; they are the
 *     recursive radix-2 forms written out from their definitions:
 *       TFT(L, g, n): h = L/2; a_j = g_j + g_{j+h}; b_j = (g_j - g_{j+h}) w^j;
 *                     outputs = TFT(h, a, min(n,h)) ++ TFT(h, b, n-h)
 *       so out_i = g(w^{rev_l(i)}) for i < n.
 *       ITFT(L, x, n): recover g (deg g < n) from out_0..out_{n-1}; see
 *       itft_rec for the steps.
 *   - or_polymul_tft: Section 3, "TFT-based polynomial multiplication":
 *     g^ = TFT(L,z1,n) g, h^ = TFT(L,z2,n) h, u^_i = g^_i h^_i (i < n),
 *     u = ITFT(L,n,n) u^ (this oracle returns u itself; the paper's
 *     ITFT gives L*u, which is exposed through or_itft's `paper_scale`).
 *   - or_polymul_ntt: Eq. (12), linear convolution through a zero-padded
 *     power-of-two modular DFT of size Lp >= n.
 *   - or_cyclic / or_negacyclic: Eq. (11) and the x^N + 1 factor of Eq. (13),
 *     by definition (folding the schoolbook product), for invariant tests.
 *
 * Readings where the paper is silent: L is the smallest power of two >= n;
 * w = g0^((p-1)/L) for the prime's primitive root g0; the inverse uses w^-1.
 *
 * Parity pins: every exported routine here is checked in tests/test_oracle.py
 * against values fixed by the mathematics (Kronecker substitution through
 * Python big integers, Horner evaluation at the transform points, closed-form
 * products, round trips, the convolution theorem, Eq. (13)'s CRT identity and
 * the butterfly-count bound of Section 3's complexity paragraph).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef uint32_t u32;

/* A planted-mistake switch for tests that prove the pins can fail.  0 = off. */
static int or_fault_mode = 0;
void or_set_fault(int mode) { or_fault_mode = mode; }

/* Butterfly counter (one per radix-2 butterfly the forward TFT executes). */
static u64 or_bfly_count = 0;
u64 or_get_butterflies(void) { return or_bfly_count; }
void or_reset_butterflies(void) { or_bfly_count = 0; }

static u32 mulm(u32 a, u32 b, u32 p) { return (u32)(((u64)a * b) % p); }
static u32 addm(u32 a, u32 b, u32 p) { return (u32)(((u64)a + b) % p); }
static u32 subm(u32 a, u32 b, u32 p) { return (u32)(((u64)a + p - b) % p); }

u32 or_powmod(u32 b, u64 e, u32 p) {
    u64 r = 1 % p, x = b % p;
    while (e) {
        if (e & 1) r = r * x % p;
        x = x * x % p;
        e >>= 1;
    }
    return (u32)r;
}

/* p is prime, so a^-1 = a^(p-2). */
u32 or_invmod(u32 a, u32 p) { return or_powmod(a, (u64)p - 2, p); }

static u64 next_pow2(u64 n) {
    u64 L = 1;
    while (L < n) L <<= 1;
    return L;
}

static void *xcalloc(u64 n, u64 sz) {
    void *q = calloc(n ? n : 1, sz);
    if (!q) abort();
    return q;
}

/* Definition 2, Eq. (2). */
void or_schoolbook(u32 p, const u32 *a, u64 za, const u32 *b, u64 zb, u32 *c) {
    if (za == 0 || zb == 0) return;
    u64 n = za + zb - 1;
    for (u64 k = 0; k < n; k++) c[k] = 0;
    for (u64 i = 0; i < za; i++)
        for (u64 j = 0; j < zb; j++)
            c[i + j] = addm(c[i + j], mulm(a[i], b[j], p), p);
}

/*
 * TFT(L, g[0..z), n) with principal L-th root w: out[i] = g(w^{rev_l(i)}), i < n.
 * g is read as zero beyond z.
 */
static void tft_rec(u32 p, u64 L, const u32 *g, u64 z, u64 n, u32 w, u32 *out) {
    if (n == 0) return;
    if (L == 1) {
        out[0] = z ? g[0] : 0;
        return;
    }
    u64 h = L / 2;
    u32 *a = xcalloc(h, sizeof(u32)), *b = xcalloc(h, sizeof(u32));
    u32 wj = 1;
    for (u64 j = 0; j < h; j++) {
        u32 lo = j < z ? g[j] : 0;
        u32 hi = (j + h < z) ? g[j + h] : 0;
        if (or_fault_mode == 1) hi = 0; /* planted: drop the upper term */
        a[j] = addm(lo, hi, p);
        b[j] = mulm(subm(lo, hi, p), or_fault_mode == 3 ? mulm(wj, w, p) : wj, p);
        wj = mulm(wj, w, p);
    }
    or_bfly_count += h;
    u32 w2 = mulm(w, w, p);
    tft_rec(p, h, a, h, n < h ? n : h, w2, out);
    if (n > h) tft_rec(p, h, b, h, n - h, w2, out + h);
    free(a);
    free(b);
}

/*
 * ITFT(L, x[0..n)) -> g[0..n) with deg g < n and TFT(L, g, n) = x (true scale).
 *   n <= h : g = ITFT(h, x, n) with root w^2 (g lives in the left half only).
 *   n >  h : A = ITFT(h, x[0..h)) is the full inverse of the left half, i.e.
 *            A_j = g_j + g_{j+h}.  With m = n-h, g_{j+h} = 0 for j >= m, so the
 *            right half B_j = (g_j - g_{j+h}) w^j equals A_j w^j there; its
 *            first m transform values are x[h..n).  Subtracting the transform
 *            of that known tail leaves a polynomial of degree < m, recovered by
 *            ITFT(h, ., m); then g_j = (A_j + D_j)/2, g_{j+h} = (A_j - D_j)/2
 *            with D_j = B_j w^-j.
 */
static void itft_rec(u32 p, u64 L, const u32 *x, u64 n, u32 w, u32 *g) {
    if (n == 0) return;
    if (L == 1) {
        g[0] = x[0];
        return;
    }
    u64 h = L / 2;
    u32 w2 = mulm(w, w, p);
    if (n <= h) {
        itft_rec(p, h, x, n, w2, g);
        return;
    }
    u64 m = n - h;
    u32 *A = xcalloc(h, sizeof(u32));
    u32 *tail = xcalloc(h, sizeof(u32));
    u32 *t = xcalloc(m, sizeof(u32));
    u32 *y = xcalloc(m, sizeof(u32));
    u32 *B = xcalloc(m, sizeof(u32));
    itft_rec(p, h, x, h, w2, A);
    u32 wj = or_powmod(w, m, p);
    for (u64 j = m; j < h; j++) {
        tail[j] = mulm(A[j], or_fault_mode == 4 ? 1 : wj, p);
        wj = mulm(wj, w, p);
    }
    tft_rec(p, h, tail, h, m, w2, t);
    for (u64 i = 0; i < m; i++) y[i] = subm(x[h + i], t[i], p);
    itft_rec(p, h, y, m, w2, B);
    u32 winv = or_invmod(w, p), inv2 = or_invmod(2, p), wmj = 1;
    for (u64 j = 0; j < m; j++) {
        u32 D = mulm(B[j], wmj, p);
        g[j] = mulm(addm(A[j], D, p), inv2, p);
        g[j + h] = mulm(or_fault_mode == 2 ? addm(A[j], D, p) : subm(A[j], D, p), inv2, p);
        wmj = mulm(wmj, winv, p);
    }
    for (u64 j = m; j < h; j++) g[j] = A[j];
    free(A);
    free(tail);
    free(t);
    free(y);
    free(B);
}

/* Checks shared by the entry points: p odd, 1 <= L, L | p-1, root in range. */
static int check_params(u32 p, u32 root, u64 L) {
    if (p < 3 || (p & 1) == 0) return -1;
    if (root == 0 || root >= p) return -1;
    if (L == 0 || ((u64)p - 1) % L != 0) return -2;
    return 0;
}

/* Principal L-th root w = root^((p-1)/L). */
u32 or_root_of_unity(u32 p, u32 root, u64 L) { return or_powmod(root, ((u64)p - 1) / L, p); }

/* TFT(L, z, n): out[0..n) = in(w^{rev_l(i)}). Returns 0, or <0 on bad input. */
int or_tft(u32 p, u32 root, u64 L, const u32 *in, u64 z, u64 n, u32 *out) {
    int e = check_params(p, root, L);
    if (e) return e;
    if (z > L || n > L) return -3;
    tft_rec(p, L, in, z, n, or_root_of_unity(p, root, L), out);
    return 0;
}

/* ITFT(L, n, n): out[0..n) = g with TFT(L, g, n) = in.
 * paper_scale = 1 returns L*g, the form Section 3 states. */
int or_itft(u32 p, u32 root, u64 L, const u32 *in, u64 n, int paper_scale, u32 *out) {
    int e = check_params(p, root, L);
    if (e) return e;
    if (n > L) return -3;
    itft_rec(p, L, in, n, or_root_of_unity(p, root, L), out);
    if (paper_scale)
        for (u64 i = 0; i < n; i++) out[i] = mulm(out[i], (u32)(L % p), p);
    return 0;
}

/* Section 3, Eq. (14): c = ITFT(L,n,n)( TFT(L,za,n) a * TFT(L,zb,n) b ). */
int or_polymul_tft(u32 p, u32 root, const u32 *a, u64 za, const u32 *b, u64 zb, u32 *c) {
    if (za == 0 || zb == 0) return -3;
    u64 n = za + zb - 1, L = next_pow2(n);
    int e = check_params(p, root, L);
    if (e) return e;
    u32 w = or_root_of_unity(p, root, L);
    u32 *A = xcalloc(n, sizeof(u32)), *B = xcalloc(n, sizeof(u32));
    tft_rec(p, L, a, za, n, w, A);
    tft_rec(p, L, b, zb, n, w, B);
    for (u64 i = 0; i < n; i++) A[i] = mulm(A[i], B[i], p);
    itft_rec(p, L, A, n, w, c);
    free(A);
    free(B);
    return 0;
}

/* Eq. (12): zero-pad both operands to Lp (a power of two >= n), full modular
 * DFT of size Lp on each, pointwise product, full inverse, keep c[0..n). */
int or_polymul_ntt(u32 p, u32 root, const u32 *a, u64 za, const u32 *b, u64 zb, u64 Lp, u32 *c) {
    if (za == 0 || zb == 0) return -3;
    u64 n = za + zb - 1;
    if (Lp < n || (Lp & (Lp - 1))) return -3;
    int e = check_params(p, root, Lp);
    if (e) return e;
    u32 w = or_root_of_unity(p, root, Lp);
    u32 *A = xcalloc(Lp, sizeof(u32)), *B = xcalloc(Lp, sizeof(u32)), *U = xcalloc(Lp, sizeof(u32));
    tft_rec(p, Lp, a, za, Lp, w, A);
    tft_rec(p, Lp, b, zb, Lp, w, B);
    for (u64 i = 0; i < Lp; i++) A[i] = mulm(A[i], B[i], p);
    itft_rec(p, Lp, A, Lp, w, U);
    memcpy(c, U, n * sizeof(u32));
    free(A);
    free(B);
    free(U);
    return 0;
}

/* Definition 4, Eq. (5): circular convolution of two length-N vectors
 * (the product reduced mod x^N - 1), by definition. */
void or_cyclic(u32 p, const u32 *u, const u32 *v, u64 N, u32 *out) {
    for (u64 i = 0; i < N; i++) out[i] = 0;
    for (u64 k = 0; k < N; k++)
        for (u64 j = 0; j < N; j++) {
            u64 idx = (k + j) % N;
            out[idx] = addm(out[idx], mulm(u[k], v[j], p), p);
        }
}

/* The x^N + 1 factor of Eq. (13): product reduced mod x^N + 1 (x^N = -1). */
void or_negacyclic(u32 p, const u32 *u, const u32 *v, u64 N, u32 *out) {
    for (u64 i = 0; i < N; i++) out[i] = 0;
    for (u64 k = 0; k < N; k++)
        for (u64 j = 0; j < N; j++) {
            u32 t = mulm(u[k], v[j], p);
            if (k + j < N) out[k + j] = addm(out[k + j], t, p);
            else out[k + j - N] = subm(out[k + j - N], t, p);
        }
}

/* Batch of independent products, each through or_polymul_tft (used for the
 * CPU baseline of the batched workload).  Offsets are element offsets into
 * the packed arrays, off[count] = total length. */
int or_polymul_tft_batch(u32 p, u32 root, u64 count, const u32 *a, const int64_t *a_off,
                         const u32 *b, const int64_t *b_off, u32 *c, const int64_t *c_off) {
    for (u64 i = 0; i < count; i++) {
        int e = or_polymul_tft(p, root, a + a_off[i], (u64)(a_off[i + 1] - a_off[i]),
                               b + b_off[i], (u64)(b_off[i + 1] - b_off[i]), c + c_off[i]);
        if (e) return e;
    }
    return 0;
}
