"""GPU parity: every product through the C ABI must equal the CPU oracle bit for
bit (exact integer arithmetic, so the tolerance is zero)."""
import random

import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P1, P2 = W.P1, W.P2


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


def from_dev(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_product(p, a, b, dev, padded_L=None):
    import torch
    from paper_1609_01010_gb300 import binding as B
    n = len(a) + len(b) - 1
    da, db = to_dev(a, dev), to_dev(b, dev)
    dc = torch.full((n,), -1, dtype=torch.int32, device=dev)
    if padded_L:
        B.polymul_mod_padded_async(p, da, len(a) - 1, db, len(b) - 1, dc, padded_L)
    else:
        B.polymul_mod_async(p, da, len(a) - 1, db, len(b) - 1, dc)
    torch.cuda.synchronize()
    return from_dev(dc)


def rnd(rng, n, p):
    return rng.integers(0, p, size=n, dtype=np.uint32)


def check(p, a, b, dev, orc, **kw):
    got = gpu_product(p, a, b, dev, **kw)
    want = orc.polymul_tft(p, a, b)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"p={p} z1={len(a)} z2={len(b)} {kw}: {len(bad)} mismatches, first at {bad[0]}")


@pytest.mark.parametrize("p", [P1, P2])
def test_workload1_full_ntt_2048(gpu, orc, p):
    _, a, b = W.workload1()
    check(p, a % p, b % p, gpu, orc)


def test_workload2_tft_8001_and_padded_comparators(gpu, orc):
    p, a, b = W.workload2()
    check(p, a, b, gpu, orc)
    for Lp in (8192, 16384):
        check(p, a, b, gpu, orc, padded_L=Lp)


@pytest.mark.parametrize("p", [P1, P2])
def test_exhaustive_small_shapes(gpu, orc, p):
    """Every (z1, z2) with z1, z2 <= 64 (launched together, checked after one sync)."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    rng = np.random.default_rng(p)
    jobs = []
    for z1 in range(1, 65):
        for z2 in range(1, 65):
            a, b = rnd(rng, z1, p), rnd(rng, z2, p)
            da, db = to_dev(a, gpu), to_dev(b, gpu)
            dc = torch.full((z1 + z2 - 1,), -1, dtype=torch.int32, device=gpu)
            B.polymul_mod_async(p, da, z1 - 1, db, z2 - 1, dc)
            jobs.append((a, b, da, db, dc))
    torch.cuda.synchronize()
    for a, b, _, _, dc in jobs:
        assert np.array_equal(from_dev(dc), orc.schoolbook(p, a, b)), (len(a), len(b))


@pytest.mark.parametrize("p", [P1, P2])
def test_boundary_lengths(gpu, orc, p):
    """n in {2^k - 1, 2^k, 2^k + 1} across the small/large kernel boundary."""
    rng = np.random.default_rng(7)
    for k in range(1, 19):
        for n in (2 ** k - 1, 2 ** k, 2 ** k + 1):
            if n < 1:
                continue
            for z1 in sorted({1, max(1, n // 2), n}):
                z2 = n + 1 - z1
                if z2 < 1:
                    continue
                check(p, rnd(rng, z1, p), rnd(rng, z2, p), gpu, orc)


@pytest.mark.parametrize("p", [P1, P2])
def test_random_shapes(gpu, orc, p):
    rng = np.random.default_rng(11)
    pyr = random.Random(11)
    for _ in range(24):
        z1 = int(np.exp(pyr.uniform(0, np.log(200000))))
        z2 = int(np.exp(pyr.uniform(0, np.log(200000))))
        check(p, rnd(rng, z1, p), rnd(rng, z2, p), gpu, orc)


@pytest.mark.parametrize("p", [P1, P2])
def test_extreme_values(gpu, orc, p):
    for z1, z2 in [(1, 1), (513, 700), (5000, 3001), (40000, 40001)]:
        a = np.full(z1, p - 1, dtype=np.uint32)
        b = np.full(z2, p - 1, dtype=np.uint32)
        check(p, a, b, gpu, orc)
        check(p, np.zeros(z1, np.uint32), b, gpu, orc)
        a[::3] = 0
        check(p, a, b, gpu, orc)


def test_workload3_sizes_full_oracle(gpu, orc):
    """Large single products mod 469762049, checked element by element
    against the oracle up to d+1 = 1500000 (n ~ 3e6)."""
    for z in (1 << 16, 100000, 1 << 20, 1500000):
        p, a, b = W.workload3(z)
        check(p, a, b, gpu, orc)


def sampled_coeffs(a, b, p, ks):
    """c_k = sum_i a_i b_{k-i} mod p, one k at a time (Definition 2)."""
    out = []
    A = a.astype(np.uint64)
    B_ = b.astype(np.uint64)
    for k in ks:
        lo = max(0, k - (len(b) - 1))
        hi = min(k, len(a) - 1)
        ai = A[lo:hi + 1]
        bj = B_[k - hi:k - lo + 1][::-1]
        out.append(int(((ai * bj) % p).sum() % p))
    return out


def eval_at(c, r, p):
    """c(r) mod p with vectorised powers r^i = r^(i & 4095) r^(4096 (i >> 12))."""
    lo = np.empty(4096, dtype=np.uint64)
    x = 1
    for i in range(4096):
        lo[i] = x
        x = x * r % p
    step = x
    nh = (len(c) >> 12) + 1
    hi = np.empty(nh, dtype=np.uint64)
    x = 1
    for i in range(nh):
        hi[i] = x
        x = x * step % p
    idx = np.arange(len(c), dtype=np.int64)
    pw = lo[idx & 4095] * hi[idx >> 12] % p
    return int(((c.astype(np.uint64) * pw) % p).sum() % p)


@pytest.mark.parametrize("z", [1 << 22, 3000001])
def test_workload3_largest_full_oracle(gpu, orc, z):
    """d+1 in {2^22, 3000001} (L = 2^23: the rows of 2^13 words, the only row
    kernel that stages its inverse twiddles over the forward ones).  A fast
    pre-check first (64 coefficients by Definition 2 and 8 random points
    c(r) = a(r) b(r)), then every coefficient against the oracle."""
    p, a, b = W.workload3(z)
    c = gpu_product(p, a, b, gpu)
    n = len(c)
    rng = random.Random(z)
    ks = [0, 1, n // 2, n - 2, n - 1] + [rng.randrange(n) for _ in range(59)]
    assert [int(c[k]) for k in ks] == sampled_coeffs(a, b, p, ks)
    for _ in range(8):
        r = rng.randrange(1, p)
        assert eval_at(c, r, p) == eval_at(a, r, p) * eval_at(b, r, p) % p
    want = orc.polymul_tft(p, a, b)
    if not np.array_equal(c, want):
        bad = np.flatnonzero(c != want)
        raise AssertionError(f"z={z}: {len(bad)} mismatches, first at {bad[0]}")


def test_unequal_lengths_at_2_23(gpu, orc):
    """Unequal random operands whose product needs L = 2^23, both primes, in
    full against the oracle (a permutation of inputs or rows would show)."""
    rng = np.random.default_rng(23)
    for p, z1, z2 in [(P1, 5000000, 1000003), (P2, 4194305, 2)]:
        check(p, rnd(rng, z1, p), rnd(rng, z2, p), gpu, orc)


@pytest.mark.parametrize("p", [P1, P2])
def test_tft_and_itft_exec(gpu, orc, p):
    import torch
    from paper_1609_01010_gb300 import binding as B
    rng = np.random.default_rng(5)
    cases = [(1, 1), (1, 2), (3, 5), (7, 8), (100, 257), (513, 1000), (4096, 4096), (5000, 8001),
             (30000, 65536), (70000, 100001)]
    for z, n in cases:
        plan = B.TftPlan(p, z, n)
        L = plan.L
        assert L == 1 << (n - 1).bit_length()
        g = rnd(rng, z, p)
        out = torch.full((n,), -1, dtype=torch.int32, device=gpu)
        plan.tft(to_dev(g, gpu), out)
        torch.cuda.synchronize()
        want = orc.tft(p, L, g, n)
        assert np.array_equal(from_dev(out), want), ("tft", z, n)
        # ITFT of n spectral values of a degree < n polynomial
        h = rnd(rng, n, p)
        x = orc.tft(p, L, h, n)
        back = torch.full((n,), -1, dtype=torch.int32, device=gpu)
        plan.itft(to_dev(x, gpu), back, scale=1)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(back), h), ("itft", z, n)
        plan.itft(to_dev(x, gpu), back, scale=0)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(back), orc.itft(p, L, x, paper_scale=True)), ("itft L*u", z, n)
        plan.close()


def test_errors_are_returned(gpu):
    import torch
    from paper_1609_01010_gb300 import binding as B
    # buffers large enough for every call below, so no check depends on them
    a = torch.zeros(8192, dtype=torch.int32, device=gpu)
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod(469762051, a, 3, a, 3, a)  # not prime
    assert e.value.status == -1
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod(2 ** 31 + 11, a, 3, a, 3, a)
    assert e.value.status == -1
    with pytest.raises(B.PolymulError) as e:  # 97: 2-adic order 5, L = 8192 too long
        B.polymul_mod(97, a, 3000, a, 3000, a)
    assert e.value.status == -2
    with pytest.raises(B.PolymulError) as e:
        B.TftPlan(P1, 1, 1 << 25)  # beyond the library's 2^24 limit
    assert e.value.status == -2


def test_host_buffer_entry_point(gpu, orc):
    """polymul_mod_host on pageable numpy buffers, on pinned buffers, on
    buffers at odd word offsets (no 16-byte alignment), one-CTA and
    three-kernel sizes, twice in a row on the same buffers."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    # n up to 2^19 - 1 runs in place where the device walks the host page
    # tables; n = 2^20 - 1 is staged by copy kernels (copy engines elsewhere)
    cases = [W.workload2(), W.workload1(), (W.P1,) + W.operands(W.SEED_BASE + 90, 100, 37, W.P1),
             W.workload3(1 << 18), W.workload3(1 << 19)]
    for p, a, b in cases:
        n = len(a) + len(b) - 1
        want = orc.polymul_tft(p, a, b)
        c = np.zeros(n, dtype=np.uint32)
        B.polymul_mod_host(p, a, len(a) - 1, b, len(b) - 1, c)
        assert np.array_equal(c, want)
        ha = torch.from_numpy(a.view(np.int32)).pin_memory()
        hb = torch.from_numpy(b.view(np.int32)).pin_memory()
        hc = torch.zeros(n + 1, dtype=torch.int32).pin_memory()
        for _ in range(2):
            B.polymul_mod_host(p, ha.data_ptr(), len(a) - 1, hb.data_ptr(), len(b) - 1, hc.data_ptr() + 4)
            assert np.array_equal(hc.numpy()[1:].view(np.uint32), want)
        # odd offsets: a and b one word into larger buffers
        a2 = np.concatenate([[7], a]).astype(np.uint32)
        b2 = np.concatenate([[9], b]).astype(np.uint32)
        c2 = np.zeros(n + 3, dtype=np.uint32)
        B.polymul_mod_host(p, a2.ctypes.data + 4, len(a) - 1, b2.ctypes.data + 4, len(b) - 1, c2.ctypes.data + 12)
        assert np.array_equal(c2[3:], want) and not c2[:3].any()


def test_host_async_on_several_streams(gpu, orc):
    """polymul_mod_host_async: products on pinned and pageable host buffers
    enqueued on three streams without waiting (in-place and staged sizes);
    after the streams are synchronised every product equals the oracle."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    streams = [torch.cuda.Stream() for _ in range(3)]
    jobs = []
    rng = np.random.default_rng(41)
    for i, (z1, z2) in enumerate([(1000, 3000), (300000, 400000), (1 << 19, 1 << 19), (5, 7), (600000, 99999),
                                  (1 << 20, 1 << 20)]):
        p = P1 if i % 2 else P2
        a = rnd(rng, z1, p)
        b = rnd(rng, z2, p)
        if i % 3 == 0:  # pageable numpy buffers
            c = np.zeros(z1 + z2 - 1, dtype=np.uint32)
            ha, hb, hc = a, b, c
        else:  # pinned
            ha = torch.from_numpy(a.view(np.int32)).pin_memory()
            hb = torch.from_numpy(b.view(np.int32)).pin_memory()
            hc = torch.zeros(z1 + z2 - 1, dtype=torch.int32).pin_memory()
        B.polymul_mod_host_async(p, ha, z1 - 1, hb, z2 - 1, hc, streams[i % 3])
        jobs.append((p, a, b, ha, hb, hc))
    for s_ in streams:
        s_.synchronize()
    for p, a, b, ha, hb, hc in jobs:
        got = hc if isinstance(hc, np.ndarray) else hc.numpy().view(np.uint32)
        assert np.array_equal(got, orc.polymul_tft(p, a, b)), (p, len(a), len(b))
