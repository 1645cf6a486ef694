"""Seeded synthetic inputs for the polynomial-multiplication workloads.

This module draws random numbers only; it holds none of the method's
arithmetic and is shared by the tests, the benchmark and the oracle checks.

Generator: splitmix64 over the counter stream seed + k*GOLDEN (k = 1, 2, ...),
Steele, Lea and Flood, "Fast splittable pseudorandom number generators" (2014).
A coefficient uniform in [0, p) is ((x >> 32) * p) >> 32 of one output x
(multiply-shift; bias below 2^-32 per value).  Product i of a batch draws from
seed ^ (i * GOLDEN), and its two operands from that seed + 1 and + 2.

Workloads (seeds 0x16090000 + k for workload k):
  1. one product mod 469762049, two degree-1023 operands (full NTT size 2048);
  2. one TFT product mod 2013265921, degrees 3000 and 5000 (n = 8001, L = 8192),
     compared with the zero-padded NTTs of size 8192 and 16384;
  3. single products mod 469762049 with equal degrees d, d+1 in
     {2^16, 2^20, 2^22, 100000, 1500000, 3000001};
  4. 4096 independent products mod 2013265921, each operand degree
     log-uniform in [64, 65536];
  5. a Poisson request stream (20 000 req/s) of products mod 469762049 or
     2013265921 (fair coin), degrees log-uniform in [256, 2^20];
  6. exact integer products (the three primes algorithm): two operands of
     equal length z with coefficients uniform over all 32-bit words.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
P1 = 469762049   # 7 * 2^26 + 1, primitive root 3
P2 = 2013265921  # 15 * 2^27 + 1, primitive root 31
PRIMES = {P1: 3, P2: 31}

SEED_BASE = 0x16090000
LARGE_SIZES = (1 << 16, 1 << 20, 1 << 22, 100000, 1500000, 3000001)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+count of splitmix64 seeded with `seed` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def coeffs(seed: int, count: int, p: int) -> np.ndarray:
    """`count` values uniform in [0, p) as uint32."""
    x = splitmix64(seed, count) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((x * np.uint64(p)) >> np.uint64(32)).astype(np.uint32)


def words(seed: int, count: int) -> np.ndarray:
    """`count` values uniform in [0, 2^32) as uint32 (the top half of each output)."""
    return (splitmix64(seed, count) >> np.uint64(32)).astype(np.uint32)


def subseed(seed: int, i: int) -> int:
    return (seed ^ ((i * GOLDEN) & MASK64)) & MASK64


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles uniform in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def loguniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(ln lo + U (ln hi - ln lo))) clamped to [lo, hi], int64."""
    u = uniform01(seed, count)
    d = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(d, lo, hi)


def operands(seed: int, da: int, db: int, p: int) -> tuple[np.ndarray, np.ndarray]:
    """Two operands of degrees da and db with uniform coefficients."""
    return coeffs(seed + 1, da + 1, p), coeffs(seed + 2, db + 1, p)


# ----------------------------------------------------------------- workloads
def workload1():
    """(p, a, b): one product of two degree-1023 polynomials mod 469762049."""
    a, b = operands(SEED_BASE + 1, 1023, 1023, P1)
    return P1, a, b


def workload2():
    """(p, a, b): degrees 3000 and 5000 mod 2013265921 (n = 8001)."""
    a, b = operands(SEED_BASE + 2, 3000, 5000, P2)
    return P2, a, b


def workload3(z: int):
    """(p, a, b): equal operand lengths z (degree z-1) mod 469762049."""
    a, b = operands(subseed(SEED_BASE + 3, z), z - 1, z - 1, P1)
    return P1, a, b


def workload6(z: int, zb: int | None = None):
    """(a, b): operands of lengths z and zb (default z), uniform 32-bit coefficients."""
    zb = z if zb is None else zb
    s = subseed(SEED_BASE + 6, z * 7919 + zb)
    return words(s + 1, z), words(s + 2, zb)


def batch_degrees(count: int = 4096, lo: int = 64, hi: int = 65536, seed: int = SEED_BASE + 4):
    """Per-product operand degrees (da, db), drawn independently."""
    da = loguniform_int(seed, count, lo, hi)
    db = loguniform_int(seed ^ 0x5A5A5A5A, count, lo, hi)
    return da, db


def workload4(count: int = 4096, lo: int = 64, hi: int = 65536, seed: int = SEED_BASE + 4):
    """Packed batch: (p, a, a_off, b, b_off, c_off), offsets int64 of length count+1."""
    p = P2
    da, db = batch_degrees(count, lo, hi, seed)
    za, zb = da + 1, db + 1
    a_off = np.zeros(count + 1, dtype=np.int64)
    b_off = np.zeros(count + 1, dtype=np.int64)
    c_off = np.zeros(count + 1, dtype=np.int64)
    a_off[1:] = np.cumsum(za)
    b_off[1:] = np.cumsum(zb)
    c_off[1:] = np.cumsum(za + zb - 1)
    a = np.empty(int(a_off[-1]), dtype=np.uint32)
    b = np.empty(int(b_off[-1]), dtype=np.uint32)
    for i in range(count):
        s = subseed(seed, i)
        a[a_off[i]:a_off[i + 1]] = coeffs(s + 1, int(za[i]), p)
        b[b_off[i]:b_off[i + 1]] = coeffs(s + 2, int(zb[i]), p)
    return p, a, a_off, b, b_off, c_off


def request_stream(rate: float = 20000.0, seconds: float = 60.0, lo: int = 256, hi: int = 1 << 20,
                   seed: int = SEED_BASE + 5):
    """Poisson arrivals: (t_arrival[s], prime[], da[], db[]) for rate*seconds requests."""
    count = int(rate * seconds)
    gaps = -np.log1p(-uniform01(seed, count)) / rate
    t = np.cumsum(gaps)
    coin = uniform01(seed ^ 0x1111, count) < 0.5
    prime = np.where(coin, P1, P2).astype(np.int64)
    da = loguniform_int(seed ^ 0x2222, count, lo, hi)
    db = loguniform_int(seed ^ 0x3333, count, lo, hi)
    keep = t < seconds
    return t[keep], prime[keep], da[keep], db[keep]
