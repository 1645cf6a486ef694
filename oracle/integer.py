"""CPU oracle for the exact integer product of polynomials with unsigned
32-bit coefficients (test infrastructure only).

Only tests/ and bench.py's CPU legs may import this module; the CUDA library
never loads it and shares no code with it.

Section 1 of the paper names the route from modular to integer polynomial
multiplication: the three primes algorithm (the product modulo three word-size
primes, recombined by the Chinese remainder theorem).  That algorithm is the
GPU side's business.  Its result has a plain definition, Definition 2 / Eq. (2)
read over the integers instead of Z/pZ,

    c_k = sum_{i + j = k} a_i b_j        (0 <= k <= za + zb - 2),

and this oracle is that definition written out:

  ``int_product(a, b)``: every a_i is split into 16-bit digits,
      a_i = ah_i 2^16 + al_i (likewise b), so that the four digit
      convolutions conv(ah, bh), conv(ah, bl), conv(al, bh), conv(al, bl)
      (numpy's direct convolution on int64: each sum has at most min(za, zb)
      terms below 2^32, so below 2^55 for za, zb <= 2^23) are exact, and
          c_k = conv(ah, bh)_k 2^32 + (conv(ah, bl) + conv(al, bh))_k 2^16
                + conv(al, bl)_k.
      The result is returned as 96-bit little-endian words, an (n, 3) uint32
      array: c_k = w[k, 0] + 2^32 w[k, 1] + 2^64 w[k, 2].
  ``int_coeff(a, b, k)``: one coefficient by the same sum, for sampled
      checks of products too large for ``int_product``.
  ``words_to_ints``: the (n, 3) words as Python integers.

Pins (tests/test_oracle_integer.py): Kronecker substitution through Python big
integers (an independent route to the same product), closed forms (operands of
all-(2^32 - 1) coefficients), the residues modulo each prime against the
modular oracle of ``oracle.polymul_tft``, evaluation at integer points, and
planted mistakes (``set_fault``) that each fail a pin.
"""
from __future__ import annotations

import numpy as np

MAX_TERMS = 1 << 23  # exactness of the int64 digit convolutions (see above)

_fault = 0


def set_fault(mode: int) -> None:
    """Plant a known mistake (tests prove the pins catch it); 0 = off.
    1: the cross term conv(al, bh) is dropped; 2: the middle term is shifted
    by 15 bits instead of 16; 3: the carry out of the low word is lost;
    4: b is reversed (a transposed operand)."""
    global _fault
    _fault = int(mode)


def _digits(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    x = np.ascontiguousarray(x, dtype=np.uint32).astype(np.int64)
    return x >> 16, x & 0xFFFF


def int_product(a, b) -> np.ndarray:
    """c = a * b over the integers (Eq. (2)), as an (n, 3) uint32 array."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    if len(a) == 0 or len(b) == 0:
        raise ValueError("empty operand")
    if min(len(a), len(b)) > MAX_TERMS:
        raise ValueError("operands too long for exact int64 digit sums")
    if _fault == 4:
        b = b[::-1].copy()
    ah, al = _digits(a)
    bh, bl = _digits(b)
    hh = np.convolve(ah, bh)
    mid = np.convolve(ah, bl)
    if _fault != 1:
        mid = mid + np.convolve(al, bh)
    ll = np.convolve(al, bl)
    shift = 15 if _fault == 2 else 16
    # c = hh 2^32 + mid 2^shift + ll, carried into 32-bit words (all < 2^63)
    low = ll + ((mid & ((1 << (32 - shift)) - 1)) << shift)
    w0 = low & 0xFFFFFFFF
    carry = 0 if _fault == 3 else (low >> 32)
    high = hh + (mid >> (32 - shift)) + carry
    w1 = high & 0xFFFFFFFF
    w2 = high >> 32
    return np.stack([w0, w1, w2], axis=1).astype(np.uint32)


def int_coeff(a, b, k: int) -> int:
    """c_k = sum_{i+j=k} a_i b_j exactly (one coefficient of Eq. (2))."""
    a = np.ascontiguousarray(a, dtype=np.uint32).astype(np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint32).astype(np.uint64)
    lo = max(0, k - (len(b) - 1))
    hi = min(k, len(a) - 1)
    if lo > hi:
        return 0
    ai = a[lo:hi + 1]
    bj = b[k - hi:k - lo + 1][::-1]
    prod = ai * bj  # each < 2^64: exact in uint64
    s_lo = int(np.sum(prod & np.uint64(0xFFFFFFFF), dtype=np.uint64))
    s_hi = int(np.sum(prod >> np.uint64(32), dtype=np.uint64))
    return (s_hi << 32) + s_lo


def words_to_ints(w: np.ndarray) -> list[int]:
    w = np.asarray(w, dtype=np.uint32).reshape(-1, 3)
    return [int(x) | (int(y) << 32) | (int(z) << 64) for x, y, z in w]
