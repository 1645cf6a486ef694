"""Pure-Python brute force used to pin the C oracle (test infrastructure only).

Each function computes its result by a route other than the oracle's:
 - ``kronecker_product``: the polynomial product through Python's big-integer
   multiplication (Kronecker substitution), then reduced mod p.  It is the
   product of Definition 2 / Eq. (2) computed by an independent library routine.
 - ``kronecker_int_product``: the same product over the integers (no reduction),
   for the exact integer product of the three primes algorithm (Section 1).
 - ``horner``: evaluation of a polynomial at a point.
 - ``direct_tft``: the TFT outputs by definition, g(w^{rev_l(i)}) for i < n
   (Section 3; van der Hoeven's bit-reversed order), each by Horner.
 - ``direct_dft``: the textbook DFT sum X_k = sum_j g_j w^{jk}, natural order.
 - ``factor`` / ``is_primitive_root``: trial division and the order test.
"""
from __future__ import annotations


def kronecker_product(a, b, p: int) -> list[int]:
    """(sum a_i x^i)(sum b_j x^j) mod p, via one big-integer multiplication."""
    a = [int(v) for v in a]
    b = [int(v) for v in b]
    n = len(a) + len(b) - 1
    # every coefficient of the integer product is < min(len) * p^2
    bits = (min(len(a), len(b)) * p * p).bit_length() + 1
    A = 0
    for v in reversed(a):
        A = (A << bits) | v
    B = 0
    for v in reversed(b):
        B = (B << bits) | v
    C = A * B
    mask = (1 << bits) - 1
    out = []
    for _ in range(n):
        out.append((C & mask) % p)
        C >>= bits
    return out


def kronecker_int_product(a, b) -> list[int]:
    """(sum a_i x^i)(sum b_j x^j) over the integers, via one big-integer
    multiplication; coefficients must be non-negative."""
    a = [int(v) for v in a]
    b = [int(v) for v in b]
    n = len(a) + len(b) - 1
    top = max(a) * max(b) * min(len(a), len(b))
    bits = max(top.bit_length(), 1) + 1
    A = 0
    for v in reversed(a):
        A = (A << bits) | v
    B = 0
    for v in reversed(b):
        B = (B << bits) | v
    C = A * B
    mask = (1 << bits) - 1
    out = []
    for _ in range(n):
        out.append(C & mask)
        C >>= bits
    return out


def horner(coeffs, x: int, p: int) -> int:
    r = 0
    for v in reversed(list(coeffs)):
        r = (r * x + int(v)) % p
    return r


def bitrev(i: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


def direct_tft(g, L: int, n: int, p: int, root: int) -> list[int]:
    l = L.bit_length() - 1
    w = pow(root, (p - 1) // L, p)
    return [horner(g, pow(w, bitrev(i, l), p), p) for i in range(n)]


def direct_dft(g, L: int, p: int, root: int) -> list[int]:
    w = pow(root, (p - 1) // L, p)
    g = list(g) + [0] * (L - len(g))
    return [sum(int(g[j]) * pow(w, j * k, p) for j in range(L)) % p for k in range(L)]


def factor(n: int) -> list[int]:
    out, d = [], 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        out.append(n)
    return out


def is_primitive_root(g: int, p: int) -> bool:
    return all(pow(g, (p - 1) // q, p) != 1 for q in factor(p - 1))
