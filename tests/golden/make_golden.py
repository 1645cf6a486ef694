"""Writes tests/golden/tiny_products.json from the oracle alone.

Each record is a small product mod one of the two primes whose expected
coefficients were computed by Python big-integer multiplication (Kronecker
substitution, oracle/brute.py) and checked equal to the C oracle's TFT
product before being stored.  Run: python tests/golden/make_golden.py
"""
import json
import os
import random
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import brute  # noqa: E402

P1, P2 = 469762049, 2013265921


def main():
    rng = random.Random(0x1609)
    recs = []
    for p in (P1, P2):
        for za, zb in [(1, 1), (2, 3), (5, 4), (17, 16), (33, 32), (64, 65)]:
            a = [rng.randrange(p) for _ in range(za)]
            b = [rng.randrange(p) for _ in range(zb)]
            c = brute.kronecker_product(a, b, p)
            assert oracle.polymul_tft(p, a, b).tolist() == c
            recs.append({"p": p, "a": a, "b": b, "c": c})
        # maximal coefficients: every operand entry p-1
        a, b = [p - 1] * 31, [p - 1] * 7
        c = brute.kronecker_product(a, b, p)
        assert oracle.polymul_tft(p, a, b).tolist() == c
        recs.append({"p": p, "a": a, "b": b, "c": c})
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_products.json")
    with open(out, "w") as f:
        json.dump({"source": "Kronecker substitution via Python big integers (Def. 2, Eq. 2)",
                   "records": recs}, f, indent=0)
    print(out, len(recs))


if __name__ == "__main__":
    main()
