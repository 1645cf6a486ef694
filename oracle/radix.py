"""CPU oracle for the general-radix truncated product (test infrastructure
only; tests/ may import it, the CUDA library never does).

Section 1 of the paper cites general-radix TFT/ITFT algorithms ([25, 27]) as
what smooths the power-of-two "stair-case", and Section 5 applies them with
relaxed truncation at the library level.  This file writes out, in plain
Python integers, the product over Z/pZ with a transform length
L = m 2^k that is not a power of two (m odd, m 2^k dividing p - 1), truncated
at the radix-m level:

  1. w = g^((p-1)/L) (g the primitive root), zeta = w^(2^k) (a primitive
     m-th root of unity), so  x^L - 1 = prod_{j<m} (x^(2^k) - zeta^j).
  2. With N = 2^k and m2 = ceil(n / N) <= m factors (n = z1 + z2 - 1), the
     product u (degree < n <= m2 N) is determined by its residues modulo the
     first m2 factors, since their product has degree m2 N >= n.
  3. Residue j of an operand g:  g_j[i] = sum_q g[i + qN] zeta^(jq)  (i < N),
     i.e. g mod (x^N - zeta^j) with x^N replaced by zeta^j.
  4. Twist by beta_j = w^j (beta_j^N = zeta^j): gt_j[i] = g_j[i] beta_j^i,
     so g_j(beta_j y) mod (y^N - 1) is a plain cyclic problem; the residue
     of the product is the cyclic convolution ut_j = gt_j (*) ht_j of length
     N (Definition 4, Eq. 5), untwisted: u_j[i] = ut_j[i] beta_j^(-i).
  5. u = sum_q U_q(x) x^(qN) with deg U_q < N; u_j = sum_{q<m2} U_q zeta^(jq),
     so U = V^-1 (u_0 .. u_{m2-1}) position by position, V the m2 x m2
     Vandermonde matrix V[j][q] = zeta^(jq) (for m2 = m its inverse is the
     inverse m-point DFT).

``radix_product(p, a, b, m)`` returns u (canonical residues).  Every product
reduces its 64-bit result with %; cyclic convolutions are the O(N^2)
definition.  ``vandermonde_inverse`` is Gauss-Jordan elimination mod p.
Pins (tests/test_oracle_radix.py): the product equals Kronecker substitution,
the splitting identity of step 1, the residues of step 3 equal u mod
(x^N - zeta^j) by polynomial division, and planted mistakes each fail.
"""
from __future__ import annotations

_fault = 0


def set_fault(mode: int) -> None:
    """0 = off; 1: wrong twist exponent (beta_j^(i+1)); 2: residue sum drops
    the last block; 3: recombination at the conjugate nodes zeta^-j (the sign
    of the exponent flipped)."""
    global _fault
    _fault = int(mode)


def plan(p: int, g: int, n: int, m: int) -> tuple[int, int, int, int]:
    """(k, N, m2, w) for the smallest N = 2^k with m N >= n."""
    k = 0
    while m * (1 << k) < n:
        k += 1
    N = 1 << k
    L = m * N
    if (p - 1) % L:
        raise ValueError(f"L = {L} does not divide p - 1")
    w = pow(g, (p - 1) // L, p)
    m2 = -(-n // N)
    return k, N, m2, w


def vandermonde_inverse(zs: list[int], p: int) -> list[list[int]]:
    """Inverse of V[j][q] = zs[j]^q mod p by Gauss-Jordan elimination."""
    r = len(zs)
    A = [[pow(zs[j], q, p) for q in range(r)] + [int(i == j) for i in range(r)] for j in range(r)]
    for col in range(r):
        piv = next(i for i in range(col, r) if A[i][col] % p)
        A[col], A[piv] = A[piv], A[col]
        inv = pow(A[col][col], p - 2, p)
        A[col] = [x * inv % p for x in A[col]]
        for i in range(r):
            if i != col and A[i][col]:
                f = A[i][col]
                A[i] = [(x - f * y) % p for x, y in zip(A[i], A[col])]
    return [row[r:] for row in A]


def residue(g: list[int], N: int, zeta_j: int, p: int) -> list[int]:
    """g mod (x^N - zeta_j): sum over blocks q of g[i + qN] zeta_j^q."""
    out = [0] * N
    blocks = -(-len(g) // N)
    if _fault == 2 and blocks > 1:
        blocks -= 1
    for q in range(blocks):
        f = pow(zeta_j, q, p)
        for i in range(N):
            if i + q * N < len(g):
                out[i] = (out[i] + g[i + q * N] * f) % p
    return out


def cyclic(u: list[int], v: list[int], p: int) -> list[int]:
    N = len(u)
    out = [0] * N
    for i in range(N):
        if u[i]:
            for j in range(N):
                out[(i + j) % N] = (out[(i + j) % N] + u[i] * v[j]) % p
    return out


def radix_product(p: int, a, b, m: int, g: int) -> list[int]:
    a = [int(x) for x in a]
    b = [int(x) for x in b]
    n = len(a) + len(b) - 1
    k, N, m2, w = plan(p, g, n, m)
    zeta = pow(w, N, p)
    res = []
    for j in range(m2):
        zj = pow(zeta, j, p)
        beta = pow(w, j, p)
        shift = 1 if _fault == 1 else 0
        tw = [pow(beta, i + shift, p) for i in range(N)]
        at = [x * t % p for x, t in zip(residue(a, N, zj, p), tw)]
        bt = [x * t % p for x, t in zip(residue(b, N, zj, p), tw)]
        ut = cyclic(at, bt, p)
        binv = pow(beta, p - 2, p)
        res.append([x * pow(binv, i, p) % p for i, x in enumerate(ut)])
    node = pow(zeta, p - 2, p) if _fault == 3 else zeta
    Vi = vandermonde_inverse([pow(node, j, p) for j in range(m2)], p)
    u = [0] * (m2 * N)
    for q in range(m2):
        for i in range(N):
            u[q * N + i] = sum(Vi[q][j] * res[j][i] for j in range(m2)) % p
    return u[:n]
