"""GPU parity of the general-radix product (transform length m 2^k, odd m,
truncated at the radix-m level; polymul_mod_radix_async) against the oracle.
The product is unique, so every result is compared bit for bit with the
pinned TFT oracle; one small case is also checked against the oracle that
follows the general-radix steps (oracle/radix.py)."""
import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P3, G3 = 754974721, 11  # p - 1 = 45 * 2^24
RADICES = [(W.P2, 31, 3), (W.P2, 31, 5), (W.P2, 31, 15), (W.P1, 3, 7), (P3, G3, 9)]


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


def radix(p, a, b, m, dev):
    import torch
    from paper_1609_01010_gb300 import binding as B
    n = len(a) + len(b) - 1
    c = torch.full((n,), -1, dtype=torch.int32, device=dev)
    B.polymul_mod_radix_async(p, to_dev(a, dev), len(a) - 1, to_dev(b, dev), len(b) - 1, c, m)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32)


def shapes(m):
    """N = 512 (one-CTA convolutions) and N >= 1024 (three-kernel ones), with
    fewer than m factors (truncated) and all m, ragged lengths."""
    out = [(1, 1), (7, 3), (300, 200), (256 * m, 256 * m), (512 * m - 700, 350)]
    for N in (1024, 4096, 1 << 15):
        out.append((N * m // 2, N * m // 2 - 1))        # n = m N - 2: all m factors
        out.append((N + 17, N // 2 + 5))                 # n ~ 1.5 N + 21: two factors
        out.append((N * (m - 1) // 2 + 3, N * (m - 1) // 2))
    return out


@pytest.mark.parametrize("p,g,m", RADICES)
def test_radix_product_equals_oracle(gpu, orc, p, g, m):
    for i, (za, zb) in enumerate(shapes(m)):
        a, b = W.operands(W.SEED_BASE + 300 + 17 * m + i, za - 1, zb - 1, p)
        want = orc.polymul_tft(p, a, b, root=g)
        assert np.array_equal(radix(p, a, b, m, gpu), want), (m, za, zb)


def test_radix_large_against_oracle(gpu, orc):
    """n = 1.5 * 2^20 + 1: radix 3 (N = 2^19, all 3 factors) and radix 15
    (N = 2^17, 13 of 15 factors) against the TFT oracle."""
    p = W.P2
    a, b = W.operands(W.SEED_BASE + 333, 786431, 786432, p)
    want = orc.polymul_tft(p, a, b)
    for m in (3, 5, 15):
        assert np.array_equal(radix(p, a, b, m, gpu), want), m


def test_radix_matches_the_stepwise_oracle(gpu):
    """One case against oracle/radix.py, which follows the algorithm's steps."""
    from oracle import radix as R
    p = W.P2
    a, b = W.operands(W.SEED_BASE + 334, 700, 500, p)
    want = np.array(R.radix_product(p, a, b, 3, 31), dtype=np.uint32)
    assert np.array_equal(radix(p, a, b, 3, gpu), want)


def test_radix_one_is_the_tft_product_and_rejections(gpu, orc):
    import torch
    from paper_1609_01010_gb300 import binding as B
    p = W.P2
    a, b = W.operands(W.SEED_BASE + 335, 5000, 3000, p)
    assert np.array_equal(radix(p, a, b, 1, gpu), orc.polymul_tft(p, a, b))
    L = B.lib()
    x = torch.zeros(64, dtype=torch.int32, device=gpu)
    ptr = x.data_ptr()
    for m in (0, 2, 4, 17, -3):
        assert L.polymul_mod_radix_async(p, ptr, 3, ptr, 3, ptr, m, None) == -7  # POLY_EINVAL
    assert L.polymul_mod_radix_async(W.P1, ptr, 3, ptr, 3, ptr, 3, None) == -7  # 3 does not divide p1 - 1
    assert L.polymul_mod_radix_async(p, None, 3, ptr, 3, ptr, 3, None) == -3     # POLY_ENULL
    # 7 2^26 > 2^23-word convolutions: POLY_ETOO_LONG
    assert L.polymul_mod_radix_async(W.P1, ptr, 7 << 22, ptr, 7 << 22, ptr, 7, None) == -2
