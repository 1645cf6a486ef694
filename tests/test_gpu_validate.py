"""Validation mode (polymul_set_validate): with it on, every entry point that
takes modular operands rejects a coefficient outside [0, p) with
POLY_EINVAL_COEF before computing anything (the output stays untouched), and
still computes the exact product of valid inputs."""
import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EINVAL_COEF = -10
SENTINEL = 0x5A5A5A5A


@pytest.fixture()
def validating():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01010_gb300 import binding as B
    B.lib()
    B.polymul_set_validate(True)
    yield torch.device("cuda:0")
    B.polymul_set_validate(False)


def dev(x, d):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(d)


def test_every_entry_point_rejects_and_leaves_output(validating, orc):
    import torch
    from paper_1609_01010_gb300 import binding as B
    L = B.lib()
    d = validating
    p = W.P1
    rng = np.random.default_rng(3)
    for za, zb in [(1, 1), (700, 300), (5000, 9000), (70000, 65536)]:
        a = rng.integers(0, p, za, dtype=np.uint32)
        b = rng.integers(0, p, zb, dtype=np.uint32)
        n = za + zb - 1
        for bad_in_b in (False, True):
            x = b.copy() if bad_in_b else a.copy()
            x[int(rng.integers(0, len(x)))] = p + int(rng.integers(0, 5))  # one word >= p
            aa, bb = (a, x) if bad_in_b else (x, b)
            da, db = dev(aa, d), dev(bb, d)
            c = torch.full((max(n, 2 * max(za, zb)),), SENTINEL, dtype=torch.int32, device=d)
            N = 1 << (max(za, zb) - 1).bit_length()
            N = max(N, 512)
            calls = {
                "polymul_mod_async": lambda: L.polymul_mod_async(p, da.data_ptr(), za - 1, db.data_ptr(), zb - 1,
                                                                 c.data_ptr(), None),
                "polymul_mod_padded_async": lambda: L.polymul_mod_padded_async(
                    p, da.data_ptr(), za - 1, db.data_ptr(), zb - 1, c.data_ptr(), 1 << (n - 1).bit_length(), None),
                "polymul_cyclic_async": lambda: L.polymul_cyclic_async(p, da.data_ptr(), za, db.data_ptr(), zb,
                                                                       c.data_ptr(), N, None),
                "polymul_negacyclic_async": lambda: L.polymul_negacyclic_async(p, da.data_ptr(), za, db.data_ptr(),
                                                                               zb, c.data_ptr(), N, None),
                "polymul_mod_radix_async": lambda: L.polymul_mod_radix_async(p, da.data_ptr(), za - 1,
                                                                             db.data_ptr(), zb - 1, c.data_ptr(),
                                                                             7, None),
            }
            for name, call in calls.items():
                assert call() == EINVAL_COEF, (name, za, zb, bad_in_b)
                torch.cuda.synchronize()
                assert (c == SENTINEL).all(), (name, za, zb)
            # host buffers
            hc = np.full(n, SENTINEL, dtype=np.uint32)
            assert L.polymul_mod_host(p, aa.ctypes.data, za - 1, bb.ctypes.data, zb - 1, hc.ctypes.data) == \
                EINVAL_COEF
            assert (hc == SENTINEL).all()
        # valid inputs still give the exact product
        c = torch.full((n,), -1, dtype=torch.int32, device=d)
        B.polymul_mod_async(p, dev(a, d), za - 1, dev(b, d), zb - 1, c)
        torch.cuda.synchronize()
        assert np.array_equal(c.cpu().numpy().view(np.uint32), orc.polymul_tft(p, a, b))


def test_batch_and_server_reject(validating, orc):
    import torch
    from paper_1609_01010_gb300 import binding as B
    d = validating
    p, a, a_off, b, b_off, c_off = W.workload4(count=16, seed=W.SEED_BASE + 41)
    c = torch.full((int(c_off[-1]),), SENTINEL, dtype=torch.int32, device=d)
    bad = b.copy()
    bad[int(b_off[7]) + 3] = p
    h = B.polymul_batch_create(p, a_off, b_off, c_off)
    try:
        for fn in ("polymul_batch_exec", "polymul_batch_exec_nograph"):
            rc = getattr(B.lib(), fn)(h, dev(a, d).data_ptr(), dev(bad, d).data_ptr(), c.data_ptr(), None)
            assert rc == EINVAL_COEF, fn
        torch.cuda.synchronize()
        assert (c == SENTINEL).all()
        B.polymul_batch_exec(h, dev(a, d), dev(b, d), c)
        torch.cuda.synchronize()
        assert B.polymul_batch_status(h) == 0
    finally:
        B.polymul_batch_destroy(h)
    assert np.array_equal(c.cpu().numpy().view(np.uint32), orc.polymul_tft_batch(p, a, a_off, b, b_off, c_off))
    srv = B.polymul_server_create(1 << 28, 2, B.SERVE_PLAIN)
    try:
        x = dev(np.array([1, 2, p], dtype=np.uint32), d)
        out = torch.full((5,), SENTINEL, dtype=torch.int32, device=d)
        with pytest.raises(B.PolymulError) as e:
            B.polymul_server_submit(srv, p, x, 2, x, 2, out)
        assert e.value.status == EINVAL_COEF
    finally:
        B.polymul_server_destroy(srv)
