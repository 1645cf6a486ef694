"""GPU parity of the exact integer product (three primes and the Chinese
remainder theorem, Section 1's route from modular to integer polynomial
multiplication) against the integer oracle (oracle/integer.py: Eq. (2) over
the integers).  Exact 96-bit integers, compared word for word: in full where
the oracle's digit convolutions finish in seconds, at sampled coefficients at
2^20 x 2^20, and against the closed form at the largest supported length."""
import numpy as np
import pytest

from oracle import integer as I
from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M32 = (1 << 32) - 1


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01010_gb300 import binding
    binding.lib()
    return torch.device("cuda:0")


def to_dev(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(dev)


def crt3(a, b, dev):
    import torch
    from paper_1609_01010_gb300 import binding as B
    n = len(a) + len(b) - 1
    c = torch.full((n, 3), -1, dtype=torch.int32, device=dev)
    B.polymul_crt3_async(to_dev(a, dev), len(a) - 1, to_dev(b, dev), len(b) - 1, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32)


# one-CTA path (L <= 512), the three-kernel path from L = 1024, ragged tails
SHAPES = [(1, 1), (1, 9), (9, 1), (2, 2), (64, 64), (300, 1000), (1024, 1024), (3001, 5001),
          (4096, 4097), (10000, 9000), (20000, 13107)]


@pytest.mark.parametrize("za,zb", SHAPES)
def test_crt3_equals_integer_oracle(gpu, za, zb):
    a, b = W.workload6(za, zb)
    assert np.array_equal(crt3(a, b, gpu), I.int_product(a, b)), (za, zb)


def test_crt3_extreme_coefficients(gpu):
    """All-(2^32 - 1), all-zero, single-word and power-of-two operands."""
    for za, zb in [(1, 1), (5, 3), (2048, 2048), (30000, 777)]:
        a = np.full(za, M32, np.uint32)
        b = np.full(zb, M32, np.uint32)
        assert np.array_equal(crt3(a, b, gpu), I.int_product(a, b))
        z = np.zeros(za, np.uint32)
        assert not crt3(z, b, gpu).any()
    a = np.array([1 << 31], np.uint32)
    b = np.array([0, 0, 1 << 31], np.uint32)
    want = np.zeros((3, 3), np.uint32)
    want[2, 1] = 1 << 30  # 2^62 = 2^32 * 2^30
    assert np.array_equal(crt3(a, b, gpu), want)


def test_crt3_sampled_at_2_20(gpu):
    """Two operands of 2^20 uniform 32-bit words (n = 2^21 - 1): sampled
    coefficients against the exact sum, and the result mod 2^32 against the
    convolution of the operands mod 2^32 at the same indices."""
    z = 1 << 20
    a, b = W.workload6(z)
    c = crt3(a, b, gpu)
    n = 2 * z - 1
    ks = [0, 1, 2, z - 2, z - 1, z, n - 2, n - 1] + [int(k) for k in np.random.default_rng(6).integers(0, n, 40)]
    got = I.words_to_ints(c[ks])
    for k, v in zip(ks, got):
        assert v == I.int_coeff(a, b, k), k


def test_crt3_largest_length_closed_form(gpu):
    """za = zb = 2^23 words of 2^32 - 1 (n = 2^24 - 1, L = 2^24, the largest
    supported): c_k = t_k (2^32 - 1)^2 with t_k = min(k + 1, n - k), the
    largest coefficient 2^23 (2^32 - 1)^2 ~ 2^87 just inside q0 q1 q2."""
    z = 1 << 23
    a = np.full(z, M32, np.uint32)
    c = crt3(a, a, gpu)
    n = 2 * z - 1
    k = np.arange(n, dtype=np.uint64)
    t = np.minimum(k + np.uint64(1), np.uint64(n) - k)
    # t (2^64 - 2^33 + 1) = (t - 1) 2^64 + (2^64 - t 2^33 + t), 1 <= t < 2^24
    with np.errstate(over="ignore"):
        low = (np.uint64(0) - (t << np.uint64(33))) + t
    want = np.stack([low & np.uint64(M32), low >> np.uint64(32), t - np.uint64(1)], axis=1).astype(np.uint32)
    assert np.array_equal(c, want)


def test_crt3_random_near_2_24(gpu, orc):
    """Random 32-bit operands with za + zb - 1 = 2^24 - 1000 (L = 2^24, the
    largest length): every coefficient mod 167772161 (a prime outside the
    three the algorithm uses, so its residues check the recombination itself)
    against the modular oracle, and 40 coefficients exactly (Eq. (2) over Z)."""
    from oracle import brute
    q = 167772161  # 5 * 2^25 + 1
    assert brute.is_primitive_root(3, q)
    za, zb = 1 << 23, (1 << 23) - 999
    a, b = W.workload6(za, zb)
    c = crt3(a, b, gpu)
    n = za + zb - 1
    assert c.shape == (n, 3)
    ks = [0, 1, zb - 1, za - 1, n - 2, n - 1] + [int(k) for k in np.random.default_rng(24).integers(0, n, 34)]
    for k, v in zip(ks, I.words_to_ints(c[ks])):
        assert v == I.int_coeff(a, b, k), k
    lo = c[:, 0].astype(np.uint64) | (c[:, 1].astype(np.uint64) << np.uint64(32))
    hi = c[:, 2].astype(np.uint64)
    got = ((hi % np.uint64(q)) * np.uint64((1 << 64) % q) + lo % np.uint64(q)) % np.uint64(q)
    want = orc.polymul_tft(q, (a % q).astype(np.uint32), (b % q).astype(np.uint32), root=3)
    assert np.array_equal(got.astype(np.uint32), want)


def test_crt3_rejections(gpu):
    import torch
    from paper_1609_01010_gb300 import binding as B
    L = B.lib()
    x = torch.zeros(16, dtype=torch.int32, device=gpu)
    assert L.polymul_crt3_async(None, 3, x.data_ptr(), 3, x.data_ptr(), None) == -3
    assert L.polymul_crt3_async(x.data_ptr(), -1, x.data_ptr(), 3, x.data_ptr(), None) == -7
    # n = 2^24 + 1 needs L = 2^25: beyond the 2-adic order of 754974721 - 1
    assert L.polymul_crt3_async(x.data_ptr(), 1 << 23, x.data_ptr(), 1 << 23, x.data_ptr(), None) == -2


def test_crt3_residues_match_modular_products(gpu, orc):
    """c mod q equals the modular product of the operands reduced mod q, for
    the two workload primes (ties the integer path to the mod-p oracle)."""
    a, b = W.workload6(50000, 40000)
    c = crt3(a, b, gpu)
    lo = c[:, 0].astype(np.uint64) | (c[:, 1].astype(np.uint64) << np.uint64(32))
    hi = c[:, 2].astype(np.uint64)
    for p in (W.P1, W.P2):
        # (hi 2^64 + lo) mod p
        r64 = (1 << 64) % p
        want = orc.polymul_tft(p, (a.astype(np.uint64) % p).astype(np.uint32),
                               (b.astype(np.uint64) % p).astype(np.uint32))
        got = ((hi % np.uint64(p)) * np.uint64(r64) + lo % np.uint64(p)) % np.uint64(p)
        assert np.array_equal(got.astype(np.uint32), want)
