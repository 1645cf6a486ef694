"""Pins of the integer-product oracle (oracle/integer.py) against what the
mathematics fixes, on the CPU.

The exact product over the integers is what the three primes algorithm of
Section 1 computes (modular products, then the Chinese remainder theorem).
Every expected value here comes from a route other than the oracle's digit
convolutions: Python big-integer multiplication (Kronecker substitution),
closed forms, the modular oracle (itself pinned in test_oracle.py) for the
residues modulo each prime, and evaluation at integer points.  The last test
plants mistakes in the oracle and checks that a pin catches each.
"""
import random

import numpy as np
import pytest

from oracle import brute
from oracle import integer as I
from paper_1609_01010_gb300 import workloads as W

M32 = (1 << 32) - 1
# The three primes of the GPU path's CRT: 7*2^26+1, 15*2^27+1, 45*2^24+1.
CRT_PRIMES = [(469762049, 3), (2013265921, 31), (754974721, 11)]


def rnd_words(rng, n):
    return np.array([rng.randrange(1 << 32) for _ in range(n)], dtype=np.uint32)


def test_crt_primes_and_exactness_bound():
    """Each prime has the stated primitive root and 2-adic order >= 24, and
    their product exceeds every coefficient of a product of 32-bit operands
    of length <= 2^23 (so the CRT reconstruction is exact up to L = 2^24)."""
    prod = 1
    for p, g in CRT_PRIMES:
        assert len(brute.factor(p)) == 1 and brute.factor(p)[0] == p
        assert brute.is_primitive_root(g, p)
        assert ((p - 1) & -(p - 1)).bit_length() - 1 >= 24
        prod *= p
    assert (1 << 23) * M32 * M32 < prod


def test_int_product_equals_kronecker():
    rng = random.Random(31)
    sizes = [(1, 1), (1, 9), (7, 1), (2, 2), (16, 16), (33, 70), (100, 37), (257, 256)]
    sizes += [(rng.randint(1, 400), rng.randint(1, 400)) for _ in range(10)]
    for za, zb in sizes:
        a, b = rnd_words(rng, za), rnd_words(rng, zb)
        got = I.words_to_ints(I.int_product(a, b))
        assert got == brute.kronecker_int_product(a, b), (za, zb)


def test_int_product_closed_forms():
    # all-(2^32 - 1) operands: c_k = t_k (2^32 - 1)^2, t_k the number of terms
    for za, zb in [(1, 1), (3, 5), (64, 64), (1000, 7), (4096, 4096)]:
        a = np.full(za, M32, dtype=np.uint32)
        b = np.full(zb, M32, dtype=np.uint32)
        n = za + zb - 1
        want = [min(k + 1, za, zb, n - k) * M32 * M32 for k in range(n)]
        assert I.words_to_ints(I.int_product(a, b)) == want
    # x^i * x^j = x^(i+j) with coefficients 2^31 and 2^32 - 1
    a = np.zeros(10, np.uint32)
    a[7] = 1 << 31
    b = np.zeros(4, np.uint32)
    b[3] = M32
    want = [0] * 13
    want[10] = (1 << 31) * M32
    assert I.words_to_ints(I.int_product(a, b)) == want


def test_int_product_residues_match_the_modular_oracle(orc):
    """c mod p == (a mod p)(b mod p) mod p for each of the three primes."""
    a, b = W.workload6(3000, 1234)
    c = I.words_to_ints(I.int_product(a, b))
    for p, g in CRT_PRIMES:
        am = (a.astype(np.uint64) % p).astype(np.uint32)
        bm = (b.astype(np.uint64) % p).astype(np.uint32)
        want = orc.polymul_tft(p, am, bm, root=g).tolist()
        assert [v % p for v in c] == want


def test_int_product_evaluation_at_integer_points():
    a, b = W.workload6(500, 300)
    c = I.words_to_ints(I.int_product(a, b))
    for r in (1, 2, 3, (1 << 40) + 17):
        ev = lambda coeffs: sum(int(v) * r ** i for i, v in enumerate(coeffs))
        assert ev(c) == ev(a) * ev(b)


def test_int_coeff_agrees_at_sampled_indices():
    a, b = W.workload6(2000, 777)
    full = I.words_to_ints(I.int_product(a, b))
    for k in [0, 1, 776, 777, 1000, 1999, 2000, 2774, 2775]:
        assert I.int_coeff(a, b, k) == full[k]
    a = np.full(5000, M32, np.uint32)
    assert I.int_coeff(a, a, 4999) == 5000 * M32 * M32


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mode):
    """A dropped cross term, a wrong shift, a lost carry and a reversed
    operand each fail the Kronecker pin."""
    rng = random.Random(40 + mode)
    a, b = rnd_words(rng, 50), rnd_words(rng, 61)
    want = brute.kronecker_int_product(a, b)
    I.set_fault(mode)
    try:
        got = I.words_to_ints(I.int_product(a, b))
    finally:
        I.set_fault(0)
    assert got != want
    assert I.words_to_ints(I.int_product(a, b)) == want
