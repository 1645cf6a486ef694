// modarith.cuh -- word-size modular arithmetic for sm_103a (device side).
//
// Residues are uint32 for an odd prime p < 2^31.  Two regimes:
//   LAZY  (p < 2^30): Harvey's lazy butterflies (D. Harvey, "Faster arithmetic
//          for number-theoretic transforms", J. Symb. Comp. 2014); forward
//          values live in [0, 4p), inverse values in [0, 2p).  Bound B = 2p.
//   !LAZY (2^30 < p < 2^31): 4p overflows a word, so forward values live in
//          [0, 2p) and inverse values in [0, p).  Bound B = p.
// In both regimes forward-butterfly values are in [0, 2B) and inverse-butterfly
// values in [0, B).
//
// Fixed multipliers (twiddles, scale factors) use Shoup's method with the
// precomputed w' = floor(w 2^32 / p): x*w - umulhi(x, w')*p lies in [0, 2p) for
// any 32-bit x and w < p (V. Shoup, NTL).  The pointwise product of two
// data values uses Montgomery's REDC with R = 2^32 (P. Montgomery, Math.
// Comp. 1985), whose 2^-32 factor is cancelled, together with the transform's
// scale, by the Shoup constant that follows it.
#pragma once
#include <stdint.h>

namespace pm {

typedef uint32_t u32;

struct ModParams {
    u32 p;     // the prime
    u32 pinv;  // p^-1 mod 2^32 (for REDC)
};

__device__ __forceinline__ u32 umin32(u32 a, u32 b) { return a < b ? a : b; }

// x mod p in [0, 2p) for any 32-bit x; w = (w, w').
__device__ __forceinline__ u32 shoup(u32 x, uint2 w, u32 p) {
    u32 q = __umulhi(x, w.y);
    return x * w.x - q * p;
}

// [0, 2p) -> [0, p)
__device__ __forceinline__ u32 canon2(u32 x, u32 p) { return umin32(x, x - p); }

// 2p, computed by an opaque (but pure) instruction: the compiler then keeps
// it in a register and folds "x - 2p, min" into one add-min instruction,
// instead of re-deriving 2p from p at every use.
__device__ __forceinline__ u32 twice(u32 p) {
    u32 r;
    asm("add.u32 %0, %1, %1;" : "=r"(r) : "r"(p));
    return r;
}

template <bool LAZY>
struct Arith {
    static constexpr bool lazy = LAZY;
    // The bound B (2p or p).
    __device__ __forceinline__ static u32 bound(u32 p) { return LAZY ? twice(p) : p; }

    // Merged Cooley-Tukey butterfly of one tree node with twiddle w:
    // (a, b) -> (a + w b, a - w b).  Inputs and outputs in [0, 2B).
    __device__ __forceinline__ static void ct(u32& a, u32& b, uint2 w, u32 p) {
        const u32 B = bound(p);
        u32 x = umin32(a, a - B);
        u32 t = shoup(b, w, p);
        if (!LAZY) t = canon2(t, p);
        a = x + t;
        b = x - t + B;
    }

    // ct with twiddle 1 (the first node of every tree level): no multiply,
    // the upper input is only brought below B.  Same ranges as ct.
    __device__ __forceinline__ static void ct_one(u32& a, u32& b, u32 p) {
        const u32 B = bound(p);
        const u32 x = umin32(a, a - B);
        const u32 t = umin32(b, b - B);
        a = x + t;
        b = x - t + B;
    }

    // gs with twiddle 1: (x, y) -> (x + y, x - y).  Same ranges as gs.
    __device__ __forceinline__ static void gs_one(u32& a, u32& b, u32 p) {
        const u32 B = bound(p);
        u32 s = a + b;
        s = umin32(s, s - B);
        const u32 d = a - b + B;
        a = s;
        b = umin32(d, d - B);
    }

    // Gentleman-Sande inverse butterfly with the inverse twiddle w = r^-1:
    // (x, y) -> (x + y, (x - y) w).  Inputs and outputs in [0, B).
    __device__ __forceinline__ static void gs(u32& a, u32& b, uint2 w, u32 p) {
        const u32 B = bound(p);
        u32 s = a + b;
        s = umin32(s, s - B);
        u32 d = a - b + B;
        u32 t = shoup(d, w, p);
        if (!LAZY) t = canon2(t, p);
        a = s;
        b = t;
    }

    // Forward-range value [0, 2B) -> inverse range [0, B).
    __device__ __forceinline__ static u32 fwd_to_inv(u32 x, u32 p) {
        const u32 B = bound(p);
        return umin32(x, x - B);
    }

    // Any value in [0, B) -> canonical [0, p).
    __device__ __forceinline__ static u32 to_canon(u32 x, u32 p) { return LAZY ? canon2(x, p) : x; }

    // Pointwise product of two forward-range values times the constant c:
    // returns a*b*c*2^-32 mod p in [0, B).  The caller folds the transform
    // scale into c = 2^32 * scale mod p.
    __device__ __forceinline__ static u32 pointwise(u32 a, u32 b, uint2 c, const ModParams& m) {
        const u32 p = m.p;
        // LAZY: both to [0, 2p) so a*b < 4p^2 < p*2^32.
        // !LAZY: a to [0, p), b in [0, 2p), so a*b < 2p^2 < p*2^32.
        a = LAZY ? umin32(a, a - bound(p)) : canon2(a, p);
        if (LAZY) b = umin32(b, b - bound(p));
        u32 lo = a * b;
        u32 hi = __umulhi(a, b);
        u32 q = lo * m.pinv;             // q*p = a*b mod 2^32
        u32 t = hi - __umulhi(q, p) + p; // (a*b - q*p)/2^32 + p, in (0, 2p)
        u32 r = shoup(t, c, p);          // [0, 2p)
        return LAZY ? r : canon2(r, p);
    }
};

// Canonical helpers for the ITFT bookkeeping steps (inputs canonical).
__device__ __forceinline__ u32 add_c(u32 a, u32 b, u32 p) { return canon2(a + b, p); }
__device__ __forceinline__ u32 sub_c(u32 a, u32 b, u32 p) { return canon2(a - b + p, p); }
__device__ __forceinline__ u32 mul_c(u32 x, uint2 w, u32 p) { return canon2(shoup(x, w, p), p); }

}  // namespace pm
