"""GPU parity of every three-kernel schedule family against the oracle.

The default schedules pick one (row length, column tile) per transform
length; these tests load schedule tables that force the others, so every
column-stage kernel is exercised at every length it can serve: the TMA-fed
kernels of 32-column tiles (row lengths 2^9 .. 2^13, column depths 1 .. 10),
their thread-load fallback for operands that are not 16-byte aligned, and the
unpruned zero-padded comparator.  Each product is compared bit for bit with
the oracle; the process's schedule table is restored afterwards.
"""
import json

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


@pytest.fixture()
def schedules(tmp_path):
    """Loads {l: (sigma, C)} tables; restores the defaults afterwards."""
    from paper_1609_01010_gb300 import binding as B
    saved = {l: B.polymul_get_schedule(l) for l in range(10, 25)}
    path = tmp_path / "sched.json"

    def load(table):
        rows = [{"l": l, "sigma": s, "C": c, "us": 0.0} for l, (s, c) in sorted(table.items())]
        path.write_text(json.dumps({"device": "test", "p": 0, "schedules": rows}))
        B.polymul_load_schedules(str(path))

    yield load
    load(saved)


def valid(l, sigma, C):
    t = l - sigma
    if sigma < 9 or sigma > 13 or sigma > l or t < 1 or t > 11:
        return False
    return (2 << t) * C * 4 <= 128 * 1024 or (C == 32 and t == 10)


def to_dev(x, dev, offset=0):
    """A device copy of x starting `offset` words into its allocation."""
    import torch
    buf = torch.zeros(len(x) + offset, dtype=torch.int32, device=dev)
    buf[offset:] = torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(dev)
    return buf[offset:]


def product(p, a, b, dev, offset=0, padded=None):
    import torch
    from paper_1609_01010_gb300 import binding as B
    n = len(a) + len(b) - 1
    c = torch.full((n,), -1, dtype=torch.int32, device=dev)
    da, db = to_dev(a, dev, offset), to_dev(b, dev, offset)
    if padded:
        B.polymul_mod_padded_async(p, da, len(a) - 1, db, len(b) - 1, c, padded)
    else:
        B.polymul_mod_async(p, da, len(a) - 1, db, len(b) - 1, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32)


def case(l, rng, p):
    """Ragged operands whose product needs L = 2^l exactly."""
    n = int(rng.integers((1 << (l - 1)) + 1, (1 << l) + 1))
    z1 = int(rng.integers(1, n + 1))
    z2 = n + 1 - z1
    return rng.integers(0, p, z1, dtype=np.uint32), rng.integers(0, p, z2, dtype=np.uint32)


@pytest.mark.parametrize("l", list(range(10, 20)))
def test_tma_column_kernels_every_row_length(gpu, orc, schedules, l):
    """32-column tiles with every valid row length at L = 2^l, both primes,
    aligned operands (TMA) and operands one word past an alignment boundary
    (thread loads)."""
    rng = np.random.default_rng(1000 + l)
    sigmas = [s for s in range(9, 14) if valid(l, s, 32)]
    assert sigmas
    for sigma in sigmas:
        schedules({l: (sigma, 32)})
        for p in (W.P1, W.P2):
            a, b = case(l, rng, p)
            want = orc.polymul_tft(p, a, b)
            for off in (0, 1):
                got = product(p, a, b, gpu, offset=off)
                assert np.array_equal(got, want), (l, sigma, p, off, int(np.flatnonzero(got != want)[0]))


@pytest.mark.parametrize("l,sigma", [(20, 10), (20, 12), (21, 11), (21, 12), (22, 12), (22, 13), (23, 13)])
def test_tma_column_kernels_large(gpu, orc, schedules, l, sigma):
    rng = np.random.default_rng(2000 + l + sigma)
    schedules({l: (sigma, 32)})
    p = W.P1 if (l + sigma) % 2 else W.P2
    a, b = case(l, rng, p)
    got = product(p, a, b, gpu)
    want = orc.polymul_tft(p, a, b)
    assert np.array_equal(got, want), (l, sigma, p, int(np.flatnonzero(got != want)[0]))


def test_tma_column_kernels_padded_and_short_operands(gpu, orc, schedules):
    """The unpruned comparator (every row loaded and computed) and operands
    shorter than one row (no full row: the thread-load path), at 32-column
    tiles."""
    rng = np.random.default_rng(77)
    schedules({l: (s, 32) for l, s in [(14, 10), (15, 11), (16, 12), (17, 12)]})
    for p in (W.P1, W.P2):
        for z1, z2, Lp in [(3000, 5001, 16384), (700, 20000, 32768), (20, 40000, 65536), (65536, 65536, 131072)]:
            a = rng.integers(0, p, z1, dtype=np.uint32)
            b = rng.integers(0, p, z2, dtype=np.uint32)
            want = orc.polymul_tft(p, a, b)
            assert np.array_equal(product(p, a, b, gpu, padded=Lp), want), (p, z1, z2, Lp)
            assert np.array_equal(product(p, a, b, gpu), want), (p, z1, z2)
    from paper_1609_01010_gb300 import binding as B
    assert B.polymul_device_status(clear=True) == 0
