"""Pins of the CPU oracle against what the mathematics fixes (no GPU needed).

The paper prints no worked example, so every expected value here comes from
an independent route: Python big-integer multiplication (Kronecker
substitution), Horner evaluation at the transform points, closed-form
products, textbook DFT sums, round trips, the convolution theorem (Theorem 1,
Eq. (8)-(10)), the CRT identity of Eq. (13) and the butterfly bound of
Section 3's complexity paragraph.  The last test plants known mistakes in the
oracle and checks that these pins catch each of them.
"""
import math
import random

import numpy as np
import pytest

from oracle import brute
from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

PRIMES = [(W.P1, 3), (W.P2, 31)]


def rnd(rng, n, p):
    return np.array([rng.randrange(p) for _ in range(n)], dtype=np.uint32)


@pytest.mark.parametrize("p,g", PRIMES)
def test_primitive_roots_and_two_adic_order(p, g):
    assert brute.is_primitive_root(g, p)
    assert sorted(brute.factor(p - 1)) == ([2, 7] if p == W.P1 else [2, 3, 5])
    v = ((p - 1) & -(p - 1)).bit_length() - 1
    assert v == (26 if p == W.P1 else 27)


@pytest.mark.parametrize("p,g", PRIMES)
def test_roots_of_unity_are_principal(orc, p, g):
    for l in range(0, 24):
        L = 1 << l
        w = int(orc.lib().or_root_of_unity(p, g, L))
        assert pow(w, L, p) == 1
        if L > 1:
            assert pow(w, L // 2, p) == p - 1  # principal: w^(L/2) = -1
    # L = 2048: L^-1 * L = 1
    inv = int(orc.lib().or_invmod(2048, p))
    assert inv * 2048 % p == 1


@pytest.mark.parametrize("p,g", PRIMES)
def test_schoolbook_equals_kronecker(orc, p, g):
    rng = random.Random(11)
    for za, zb in [(1, 1), (1, 7), (5, 1), (3, 4), (16, 16), (33, 70), (64, 1), (100, 37)]:
        a, b = rnd(rng, za, p), rnd(rng, zb, p)
        assert orc.schoolbook(p, a, b).tolist() == brute.kronecker_product(a, b, p)
    # maximal coefficients and zeros
    a = np.full(50, p - 1, dtype=np.uint32)
    b = np.full(31, p - 1, dtype=np.uint32)
    assert orc.schoolbook(p, a, b).tolist() == brute.kronecker_product(a, b, p)
    z = np.zeros(9, dtype=np.uint32)
    assert orc.schoolbook(p, z, b).tolist() == [0] * 39


@pytest.mark.parametrize("p,g", PRIMES)
def test_polymul_closed_forms(orc, p, g):
    # (1+x)^m (1+x)^k = (1+x)^(m+k): binomial coefficients
    for m, k in [(10, 7), (100, 155), (300, 301)]:
        a = np.array([math.comb(m, i) % p for i in range(m + 1)], dtype=np.uint32)
        b = np.array([math.comb(k, i) % p for i in range(k + 1)], dtype=np.uint32)
        want = [math.comb(m + k, i) % p for i in range(m + k + 1)]
        assert orc.polymul_tft(p, a, b).tolist() == want
        assert orc.schoolbook(p, a, b).tolist() == want
    # (x - 1)(1 + x + ... + x^(k-1)) = x^k - 1
    for k in [1, 2, 5, 64, 1000, 1025]:
        a = np.array([p - 1, 1], dtype=np.uint32)
        b = np.ones(k, dtype=np.uint32)
        want = [p - 1] + [0] * (k - 1) + [1]
        assert orc.polymul_tft(p, a, b).tolist() == want
    # all-ones of lengths m, k: c_i = min(i+1, m, k, m+k-1-i)
    for m, k in [(1, 1), (7, 3), (64, 64), (1000, 37)]:
        c = orc.polymul_tft(p, np.ones(m, np.uint32), np.ones(k, np.uint32)).tolist()
        assert c == [min(i + 1, m, k, m + k - 1 - i) for i in range(m + k - 1)]


@pytest.mark.parametrize("p,g", PRIMES)
def test_tft_equals_evaluation_at_bit_reversed_roots(orc, p, g):
    rng = random.Random(5)
    for l in range(0, 7):
        L = 1 << l
        for _ in range(6):
            n = rng.randint(1, L)
            z = rng.randint(1, n)
            gg = rnd(rng, z, p)
            assert orc.tft(p, L, gg, n).tolist() == brute.direct_tft(gg, L, n, p, g)
    gg = rnd(rng, 200, p)
    assert orc.tft(p, 256, gg, 233).tolist() == brute.direct_tft(gg, 256, 233, p, g)


@pytest.mark.parametrize("p,g", PRIMES)
def test_full_tft_is_textbook_dft_in_bit_reversed_order(orc, p, g):
    rng = random.Random(9)
    for l in range(0, 7):
        L = 1 << l
        gg = rnd(rng, L, p)
        X = brute.direct_dft(gg, L, p, g)
        out = orc.tft(p, L, gg, L).tolist()
        assert out == [X[brute.bitrev(i, l)] for i in range(L)]


@pytest.mark.parametrize("p,g", PRIMES)
def test_itft_round_trip_every_n_up_to_1024(orc, p, g):
    rng = np.random.default_rng(3)
    for l in range(0, 11):
        L = 1 << l
        for n in range(1, L + 1):
            gg = rng.integers(0, p, size=n, dtype=np.uint32)
            x = orc.tft(p, L, gg, n)
            back = orc.itft(p, L, x)
            assert np.array_equal(back, gg), (L, n)


@pytest.mark.parametrize("p,g", PRIMES)
def test_itft_paper_scale_is_L_times(orc, p, g):
    rng = np.random.default_rng(4)
    for L, n in [(1, 1), (8, 5), (64, 64), (512, 300)]:
        gg = rng.integers(0, p, size=n, dtype=np.uint32)
        x = orc.tft(p, L, gg, n)
        scaled = orc.itft(p, L, x, paper_scale=True)
        assert scaled.tolist() == [int(v) * L % p for v in gg]


def boundary_sizes():
    out = [(1, 1), (1, 2), (2, 1), (2, 2)]
    for k in range(2, 13):
        for n in (2 ** k - 1, 2 ** k, 2 ** k + 1):
            za = max(1, n // 3)
            out.append((za, n + 1 - za))
    return out


@pytest.mark.parametrize("p,g", PRIMES)
def test_polymul_tft_equals_kronecker(orc, p, g):
    rng = random.Random(1)
    sizes = boundary_sizes() + [(rng.randint(1, 700), rng.randint(1, 700)) for _ in range(25)]
    for za, zb in sizes:
        a, b = rnd(rng, za, p), rnd(rng, zb, p)
        assert orc.polymul_tft(p, a, b).tolist() == brute.kronecker_product(a, b, p), (za, zb)


@pytest.mark.parametrize("p,g", PRIMES)
def test_polymul_padded_ntt_matches(orc, p, g):
    rng = random.Random(2)
    for za, zb in [(1, 1), (3, 5), (100, 29), (513, 512), (1024, 1024)]:
        a, b = rnd(rng, za, p), rnd(rng, zb, p)
        n = za + zb - 1
        want = brute.kronecker_product(a, b, p)
        L = 1 << (n - 1).bit_length()
        for Lp in (L, 2 * L):
            assert orc.polymul_ntt(p, a, b, Lp).tolist() == want


def fold(c, N, sign):
    out = [0] * N
    for i, v in enumerate(c):
        q, r = divmod(i, N)
        out[r] += v * (sign ** q)
    return out


@pytest.mark.parametrize("p,g", PRIMES)
def test_convolution_theorem_and_cyclic(orc, p, g):
    """Theorem 1: DFT(u (*) v) = DFT(u) . DFT(v) for the full transform."""
    rng = random.Random(7)
    for N in (1, 2, 8, 64, 256):
        u, v = rnd(rng, N, p), rnd(rng, N, p)
        want = [x % p for x in fold(brute.kronecker_product(u, v, p), N, 1)]
        assert orc.cyclic(p, u, v).tolist() == want
        U, V = orc.tft(p, N, u, N), orc.tft(p, N, v, N)
        prod = (U.astype(np.uint64) * V.astype(np.uint64) % p).astype(np.uint32)
        assert orc.itft(p, N, prod).tolist() == want


@pytest.mark.parametrize("p,g", PRIMES)
def test_crt_identity_eq13(orc, p, g):
    """Z[x]/(x^2N - 1) = Z[x]/(x^N - 1) x Z[x]/(x^N + 1), Eq. (13)."""
    rng = random.Random(8)
    for N in (1, 4, 32, 100):
        u, v = rnd(rng, 2 * N, p), rnd(rng, 2 * N, p)
        big = orc.cyclic(p, u, v).tolist()                    # mod x^2N - 1
        red_minus = [x % p for x in fold(big, N, 1)]
        red_plus = [x % p for x in fold(big, N, -1)]
        um, vm = [x % p for x in fold(u.tolist(), N, 1)], [x % p for x in fold(v.tolist(), N, 1)]
        up, vp = [x % p for x in fold(u.tolist(), N, -1)], [x % p for x in fold(v.tolist(), N, -1)]
        assert orc.cyclic(p, um, vm).tolist() == red_minus
        assert orc.negacyclic(p, up, vp).tolist() == red_plus
        kr = brute.kronecker_product(up, vp, p)
        assert orc.negacyclic(p, up, vp).tolist() == [x % p for x in fold(kr, N, -1)]


@pytest.mark.parametrize("p,g", PRIMES)
def test_random_point_evaluation(orc, p, g):
    rng = random.Random(12)
    for za, zb in [(3000, 5000), (1024, 1024), (4097, 3)]:
        a, b = rnd(rng, za, p), rnd(rng, zb, p)
        c = orc.polymul_tft(p, a, b)
        for _ in range(8):
            r = rng.randrange(p)
            assert brute.horner(c, r, p) == brute.horner(a, r, p) * brute.horner(b, r, p) % p


@pytest.mark.parametrize("p,g", PRIMES)
def test_workload_products_spot_checked(orc, p, g):
    """Workload 1 (full NTT 2048) and 2 (TFT 8001) against schoolbook entries."""
    for wl in (W.workload1, W.workload2):
        pp, a, b = wl()
        c = orc.polymul_tft(pp, a, b)
        assert np.array_equal(c, orc.schoolbook(pp, a, b))
        assert np.array_equal(c, orc.polymul_ntt(pp, a, b, 1 << (len(c) - 1).bit_length()))


def test_butterfly_bound(orc):
    """TFT(L, z, n) uses at most n log2(L) / 2 + L butterflies (Section 3)."""
    p = W.P1
    rng = random.Random(13)
    for l in range(1, 14):
        L = 1 << l
        for n in sorted({1, L // 2 + 1, L - 1, L, rng.randint(1, L)}):
            orc.reset_butterflies()
            orc.tft(p, L, np.ones(n, np.uint32), n)
            assert orc.butterflies() <= n * l / 2 + L, (L, n)
    orc.reset_butterflies()
    orc.tft(p, 1024, np.ones(1024, np.uint32), 1024)
    assert orc.butterflies() == 1024 * 10 // 2  # full transform: (L log L)/2


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(orc, mode):
    """Each planted mistake (dropped term, wrong sign, shifted twiddle, lost
    tail twist) must fail at least one of the pins above."""
    p, g = W.P1, 3
    rng = random.Random(21)
    caught = False
    orc.set_fault(mode)
    try:
        for za, zb in [(5, 9), (300, 211), (513, 600)]:
            a, b = rnd(rng, za, p), rnd(rng, zb, p)
            if orc.polymul_tft(p, a, b).tolist() != brute.kronecker_product(a, b, p):
                caught = True
        gg = rnd(rng, 40, p)
        if orc.tft(p, 64, gg, 50).tolist() != brute.direct_tft(gg, 64, 50, p, g):
            caught = True
    finally:
        orc.set_fault(0)
    assert caught
    a, b = rnd(rng, 33, p), rnd(rng, 20, p)
    assert orc.polymul_tft(p, a, b).tolist() == brute.kronecker_product(a, b, p)


def test_golden_tiny_products(orc):
    """Stored products (tests/golden/tiny_products.json, Def. 2 via big integers)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_products.json")
    with open(path) as f:
        recs = json.load(f)["records"]
    assert len(recs) >= 10
    for r in recs:
        assert orc.polymul_tft(r["p"], r["a"], r["b"]).tolist() == r["c"]
        assert orc.schoolbook(r["p"], r["a"], r["b"]).tolist() == r["c"]


@pytest.mark.parametrize("p,g", PRIMES)
def test_batch_equals_kronecker_per_product(orc, p, g):
    """The batched oracle (the checker of the GPU batch) product by product
    against Kronecker substitution: ragged lengths (1 to a few hundred), a
    non-zero first offset in a, b and c, and gaps in c between products whose
    words must stay untouched."""
    import ctypes
    rng = random.Random(31 + p % 97)
    sizes = [(1, 1), (7, 300), (129, 2), (64, 64), (513, 17), (1, 250), (200, 1), (33, 95)]
    a_off, b_off, c_off = [5], [11], [3]
    for i, (za, zb) in enumerate(sizes):
        a_off.append(a_off[-1] + za)
        b_off.append(b_off[-1] + zb)
        c_off.append(c_off[-1] + za + zb - 1 + (i % 3))  # 0, 1 or 2 unused words after product i
    a = rnd(rng, a_off[-1], p)
    b = rnd(rng, b_off[-1], p)
    sentinel = 0xA5A5A5A5
    c = np.full(c_off[-1] + 4, sentinel, dtype=np.uint32)
    i64 = lambda x: np.ascontiguousarray(x, dtype=np.int64)
    ao, bo, co = i64(a_off), i64(b_off), i64(c_off)
    P = ctypes.POINTER(ctypes.c_uint32)
    Q = ctypes.POINTER(ctypes.c_int64)
    rc = orc.lib().or_polymul_tft_batch(p, g, len(sizes), a.ctypes.data_as(P), ao.ctypes.data_as(Q),
                                        b.ctypes.data_as(P), bo.ctypes.data_as(Q), c.ctypes.data_as(P),
                                        co.ctypes.data_as(Q))
    assert rc == 0
    written = np.zeros(len(c), dtype=bool)
    for i, (za, zb) in enumerate(sizes):
        ai = a[a_off[i]:a_off[i] + za]
        bi = b[b_off[i]:b_off[i] + zb]
        n = za + zb - 1
        assert c[c_off[i]:c_off[i] + n].tolist() == brute.kronecker_product(ai, bi, p), i
        written[c_off[i]:c_off[i] + n] = True
    assert (c[~written] == sentinel).all()  # the first 3 words, the gaps and the tail
    # the wrapper: same products through numpy offsets
    got = orc.polymul_tft_batch(p, a, a_off, b, b_off, c_off)
    assert np.array_equal(got[written[:len(got)]], c[:len(got)][written[:len(got)]])
    # a plausible offset mistake (operand b of product i taken from product
    # i+1's start) is caught by the per-product comparison above
    wrong = orc.polymul_tft(p, a[a_off[1]:a_off[2]], b[b_off[2]:b_off[2] + sizes[1][1]])
    assert wrong.tolist() != brute.kronecker_product(a[a_off[1]:a_off[2]], b[b_off[1]:b_off[2]], p)
