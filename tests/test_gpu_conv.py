"""GPU parity of the cyclic (mod x^N - 1, Definition 4 / Eq. 11) and
negacyclic (mod x^N + 1, Eq. 13's second factor) convolutions against the
oracle: its O(N^2) definitions for small N, and its linear TFT product
reduced mod x^N -/+ 1 for large N.  Exact integers, compared bit for bit."""
import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def run(kind, p, a, b, N, dev):
    import torch
    from paper_1609_01010_gb300 import binding as B
    c = torch.full((N,), -1, dtype=torch.int32, device=dev)
    fn = B.polymul_cyclic_async if kind == "cyclic" else B.polymul_negacyclic_async
    fn(p, to_dev(a, dev), len(a), to_dev(b, dev), len(b), c, N)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32)


def fold(u, N, p, sign):
    out = np.zeros(N, dtype=np.int64)
    u = np.asarray(u, dtype=np.int64)
    out[:min(N, len(u))] += u[:N]
    if len(u) > N:
        out[:len(u) - N] += sign * u[N:]
    return (out % p).astype(np.uint32)


@pytest.mark.parametrize("kind", ["cyclic", "negacyclic"])
@pytest.mark.parametrize("p", [W.P1, W.P2])
@pytest.mark.parametrize("N", [1, 2, 7, 100, 512, 1000, 1024, 4096])
def test_small_against_definition(gpu, orc, kind, p, N):
    rng = np.random.default_rng(N + (p & 0xff))
    for za, zb in [(N, N), (max(1, N // 3), N), (1, max(1, N - 1))]:
        a = rng.integers(0, p, za, dtype=np.uint32)
        b = rng.integers(0, p, zb, dtype=np.uint32)
        A = np.zeros(N, dtype=np.uint32)
        Bv = np.zeros(N, dtype=np.uint32)
        A[:za], Bv[:zb] = a, b
        want = orc.cyclic(p, A, Bv) if kind == "cyclic" else orc.negacyclic(p, A, Bv)
        assert np.array_equal(run(kind, p, a, b, N, gpu), want), (za, zb)


@pytest.mark.parametrize("kind", ["cyclic", "negacyclic"])
@pytest.mark.parametrize("N,za,zb", [(1 << 14, 1 << 14, 1 << 14), (1 << 16, 40000, 1 << 16), (100003, 100003, 77777),
                                     (1 << 20, 1 << 20, 1 << 20)])
def test_large_against_folded_product(gpu, orc, kind, N, za, zb):
    p = W.P1
    a = W.coeffs(W.SEED_BASE + 70, za, p)
    b = W.coeffs(W.SEED_BASE + 71, zb, p)
    u = orc.polymul_tft(p, a, b)
    want = fold(u, N, p, 1 if kind == "cyclic" else -1)
    assert np.array_equal(run(kind, p, a, b, N, gpu), want)


def test_extreme_values_and_argument_checks(gpu, orc):
    import torch
    from paper_1609_01010_gb300 import binding as B
    p = W.P2
    N = 2048
    a = np.full(N, p - 1, dtype=np.uint32)
    assert np.array_equal(run("cyclic", p, a, a, N, gpu), orc.cyclic(p, a, a))
    assert np.array_equal(run("negacyclic", p, a, a, N, gpu), orc.negacyclic(p, a, a))
    c = torch.empty(8, dtype=torch.int32, device=gpu)
    x = to_dev(np.ones(9, dtype=np.uint32), gpu)
    with pytest.raises(B.PolymulError):
        B.polymul_cyclic_async(p, x, 9, x, 9, c, 8)  # za > N
    with pytest.raises(B.PolymulError):
        B.polymul_negacyclic_async(p, x, 0, x, 4, c, 8)  # empty operand


@pytest.mark.parametrize("N,za,zb", [(1 << 17, 5000, 1 << 17), (1 << 21, 1 << 21, 1234567)])
def test_negacyclic_twisted_second_prime(gpu, orc, N, za, zb):
    """Power-of-two N (the twisted length-N path) mod 2013265921, unequal and
    ragged operand lengths, against the folded oracle product."""
    p = W.P2
    a = W.coeffs(W.SEED_BASE + 72, za, p)
    b = W.coeffs(W.SEED_BASE + 73, zb, p)
    want = fold(orc.polymul_tft(p, a, b), N, p, -1)
    assert np.array_equal(run("negacyclic", p, a, b, N, gpu), want)
