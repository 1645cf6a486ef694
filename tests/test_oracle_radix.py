"""Pins of the general-radix product oracle (oracle/radix.py) on the CPU.

Expected values come from routes other than the oracle's own steps: the
product from Kronecker substitution through Python big integers, the
splitting x^(mN) - 1 = prod_j (x^N - zeta^j) by multiplying the factors out,
each residue by polynomial long division, and the Vandermonde inverse by
multiplying it back.  Planted mistakes in the oracle must each fail a pin.
"""
import random

import pytest

from oracle import brute
from oracle import radix as R

P2, G2 = 2013265921, 31   # p - 1 = 15 * 2^27: radices 3, 5, 15
P1, G1 = 469762049, 3     # p - 1 = 7 * 2^26: radix 7
P3, G3 = 754974721, 11    # p - 1 = 45 * 2^24: radices 3, 5, 9, 15, 45

CASES = [(P2, G2, 3), (P2, G2, 5), (P2, G2, 15), (P1, G1, 7), (P3, G3, 9)]


def rnd(rng, n, p):
    return [rng.randrange(p) for _ in range(n)]


def polymul(u, v, p):
    out = [0] * (len(u) + len(v) - 1)
    for i, x in enumerate(u):
        for j, y in enumerate(v):
            out[i + j] = (out[i + j] + x * y) % p
    return out


def polyrem(g, N, c, p):
    """g mod (x^N - c) by long division (leading term x^d -> c x^(d-N))."""
    g = list(g)
    for d in range(len(g) - 1, N - 1, -1):
        if g[d]:
            g[d - N] = (g[d - N] + g[d] * c) % p
            g[d] = 0
    return (g + [0] * N)[:N]


@pytest.mark.parametrize("p,g,m", CASES)
def test_splitting_identity(p, g, m):
    for N in (1, 2, 8):
        k, NN, m2, w = R.plan(p, g, m * N, m)
        assert NN == N and m2 == m
        zeta = pow(w, N, p)
        assert pow(zeta, m, p) == 1 and all(pow(zeta, d, p) != 1 for d in range(1, m))
        prod = [1]
        for j in range(m):
            f = [0] * (N + 1)
            f[0], f[N] = (-pow(zeta, j, p)) % p, 1
            prod = polymul(prod, f, p)
        want = [0] * (m * N + 1)
        want[0], want[m * N] = p - 1, 1
        assert prod == want


@pytest.mark.parametrize("p,g,m", CASES)
def test_residues_are_polynomial_remainders(p, g, m):
    rng = random.Random(m)
    for N, z in [(4, 11), (8, 8 * m), (16, 3)]:
        _, _, _, w = R.plan(p, g, min(z, m * N), m)
        w = pow(g, (p - 1) // (m * N), p)
        gg = rnd(rng, z, p)
        for j in range(m):
            c = pow(w, N * j, p)
            assert R.residue(gg, N, c, p) == polyrem(gg, N, c, p)


@pytest.mark.parametrize("p,g,m", CASES)
def test_vandermonde_inverse(p, g, m):
    w = pow(g, (p - 1) // m, p)
    for r in range(1, m + 1):
        zs = [pow(w, j, p) for j in range(r)]
        Vi = R.vandermonde_inverse(zs, p)
        for i in range(r):
            for q in range(r):
                s = sum(Vi[i][j] * pow(zs[j], q, p) for j in range(r)) % p
                assert s == int(i == q)


@pytest.mark.parametrize("p,g,m", CASES)
def test_radix_product_equals_kronecker(p, g, m):
    rng = random.Random(1000 + m)
    shapes = [(1, 1), (1, 2), (2, 2), (3, 7), (17, 5), (m * 4, m * 4), (33, 40), (60, 61)]
    for za, zb in shapes:
        a, b = rnd(rng, za, p), rnd(rng, zb, p)
        got = R.radix_product(p, a, b, m, g)
        assert got == brute.kronecker_product(a, b, p), (za, zb)
    # truncated (fewer than m factors) and untruncated splits both occur
    used = {R.plan(p, g, za + zb - 1, m)[2] for za, zb in shapes}
    assert max(used) == m or m > 9
    assert any(u < m for u in used)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_planted_mistakes_are_caught(mode):
    rng = random.Random(70 + mode)
    a, b = rnd(rng, 40, P2), rnd(rng, 37, P2)
    want = brute.kronecker_product(a, b, P2)
    R.set_fault(mode)
    try:
        bad = R.radix_product(P2, a, b, 5, G2)
    finally:
        R.set_fault(0)
    assert bad != want
    assert R.radix_product(P2, a, b, 5, G2) == want
