"""GPU parity of the batched (persistent kernel + CUDA graph) and serving
paths: every product equals the oracle and the same product computed alone.
Exact integer results, so "the same" means bit-identical."""
import os

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


def from_dev(t):
    return t.cpu().numpy().view(np.uint32)


def alone(p, a, b, dev):
    import torch
    from paper_1609_01010_gb300 import binding as B
    dc = torch.empty(len(a) + len(b) - 1, dtype=torch.int32, device=dev)
    B.polymul_mod(p, to_dev(a, dev), len(a) - 1, to_dev(b, dev), len(b) - 1, dc)
    return from_dev(dc)


def test_batch_matches_oracle_and_plain(gpu, orc):
    """A 256-product slice of the batched workload (same degree law), through
    the graph, the graph-less persistent launch and the plain per-product path."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    p, a, a_off, b, b_off, c_off = W.workload4(count=256, seed=W.SEED_BASE + 40)
    da, db = to_dev(a, gpu), to_dev(b, gpu)
    outs = [torch.full((int(c_off[-1]),), -1, dtype=torch.int32, device=gpu) for _ in range(3)]
    h = B.polymul_batch_create(p, a_off, b_off, c_off)
    try:
        B.polymul_batch_exec(h, da, db, outs[0])
        B.polymul_batch_exec(h, da, db, outs[0])  # graph replay
        B.polymul_batch_exec_nograph(h, da, db, outs[1])
        torch.cuda.synchronize()
        assert B.polymul_batch_status(h) == 0
    finally:
        B.polymul_batch_destroy(h)
    B.polymul_mod_batched_plain(p, da, a_off, db, b_off, outs[2], c_off)
    torch.cuda.synchronize()
    got = [from_dev(o) for o in outs]
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])
    want = orc.polymul_tft_batch(p, a, a_off, b, b_off, c_off)
    assert np.array_equal(got[0], want)


def test_batch_full_workload_sampled(gpu, orc):
    """The full 4096-product workload: batch == plain everywhere, and 48
    products (the largest included) == oracle."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    p, a, a_off, b, b_off, c_off = W.workload4()
    da, db = to_dev(a, gpu), to_dev(b, gpu)
    dc = torch.empty(int(c_off[-1]), dtype=torch.int32, device=gpu)
    dc2 = torch.empty_like(dc)
    B.polymul_mod_batched(p, da, a_off, db, b_off, dc, c_off)
    B.polymul_mod_batched_plain(p, da, a_off, db, b_off, dc2, c_off)
    torch.cuda.synchronize()
    assert torch.equal(dc, dc2)
    c = from_dev(dc)
    n = np.diff(c_off)
    idx = list(np.argsort(n)[-8:]) + list(np.random.default_rng(3).choice(len(n), 40, replace=False))
    for i in idx:
        i = int(i)
        want = orc.polymul_tft(p, a[a_off[i]:a_off[i + 1]], b[b_off[i]:b_off[i + 1]])
        assert np.array_equal(c[c_off[i]:c_off[i + 1]], want), i


@pytest.mark.parametrize("kind", [1, 2])
def test_batch_bounded_wait_reports_timeout(gpu, kind):
    """Withhold one column item (kind 1) or row item (kind 2) from the work
    list: the items waiting on it give up after a short bounded wait, the
    launch ends and the status reads POLY_ETIMEOUT.  Then the restored list
    runs clean."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    p = W.P2
    sizes = [(20000, 30000), (300, 500), (9000, 9000)]
    a_off, b_off, c_off = [0], [0], [0]
    for za, zb in sizes:
        a_off.append(a_off[-1] + za)
        b_off.append(b_off[-1] + zb)
        c_off.append(c_off[-1] + za + zb - 1)
    a = W.coeffs(1, a_off[-1], p)
    b = W.coeffs(2, b_off[-1], p)
    da, db = to_dev(a, gpu), to_dev(b, gpu)
    dc = torch.zeros(c_off[-1], dtype=torch.int32, device=gpu)
    h = B.polymul_batch_create(p, a_off, b_off, c_off)
    try:
        B.polymul_batch_test_withhold(h, kind, 1 << 14)
        B.polymul_batch_exec_nograph(h, da, db, dc)
        assert B.polymul_batch_status(h) == -6  # POLY_ETIMEOUT
        B.polymul_batch_test_withhold(h, -1, 0)
        B.polymul_batch_exec_nograph(h, da, db, dc)
        assert B.polymul_batch_status(h) == 0
    finally:
        B.polymul_batch_destroy(h)
    torch.cuda.synchronize()
    c = from_dev(dc)
    for i, (za, zb) in enumerate(sizes):
        assert np.array_equal(c[c_off[i]:c_off[i + 1]],
                              alone(p, a[a_off[i]:a_off[i + 1]], b[b_off[i]:b_off[i + 1]], gpu))


@pytest.mark.parametrize("mode", [0, 1])  # batch, plain
def test_server_mix_equals_alone_and_oracle(gpu, orc, mode):
    """Requests of mixed sizes and both primes submitted back to back (so they
    are admitted while others run) give the same result as alone, in every
    dispatch mode."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    rng = np.random.default_rng(9 + mode)
    reqs = []
    for i in range(120):
        p = W.P1 if i % 2 else W.P2
        da = int(np.exp(rng.uniform(0, np.log(1 << 17))))
        db = int(np.exp(rng.uniform(0, np.log(1 << 17))))
        a = rng.integers(0, p, da + 1, dtype=np.uint32)
        b = rng.integers(0, p, db + 1, dtype=np.uint32)
        reqs.append((p, a, b, to_dev(a, gpu), to_dev(b, gpu),
                     torch.full((da + db + 1,), -1, dtype=torch.int32, device=gpu)))
    torch.cuda.synchronize()
    srv = B.polymul_server_create(1 << 30, 4, mode)
    try:
        tickets = [B.polymul_server_submit(srv, p, xa, len(a) - 1, xb, len(b) - 1, xc)
                   for p, a, b, xa, xb, xc in reqs]
        for t in tickets:
            B.polymul_server_wait(srv, t, 60000)
            assert B.polymul_server_poll(srv, t)
        stats = B.polymul_server_stats(srv)
        assert stats["count"] == len(reqs) and stats["p99_us"] > 0
        with pytest.raises(B.PolymulError) as e:
            B.polymul_server_wait(srv, 10 ** 9, 10)
        assert e.value.status == -9
    finally:
        B.polymul_server_destroy(srv)
    for p, a, b, _, _, xc in reqs:
        got = from_dev(xc)
        assert np.array_equal(got, alone(p, a, b, gpu))
    for p, a, b, _, _, xc in reqs[:30]:
        assert np.array_equal(from_dev(xc), orc.polymul_tft(p, a, b))


def test_server_budget_admission(gpu, orc):
    """A budget that holds only a few requests at a time still completes all
    of them correctly; a request larger than the budget is refused."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    p = W.P1
    rng = np.random.default_rng(4)
    budget = 6 << 20
    srv = B.polymul_server_create(budget, 2)
    try:
        big = torch.zeros(1 << 21, dtype=torch.int32, device=gpu)  # holds any operand or the output
        with pytest.raises(B.PolymulError) as e:
            B.polymul_server_submit(srv, p, big, (1 << 20) - 1, big, (1 << 20) - 1, big)
        assert e.value.status == -8  # POLY_EBUSY
        reqs = []
        for _ in range(40):
            d = int(rng.integers(20000, 60000))
            a = rng.integers(0, p, d + 1, dtype=np.uint32)
            b = rng.integers(0, p, d + 1, dtype=np.uint32)
            xc = torch.full((2 * d + 1,), -1, dtype=torch.int32, device=gpu)
            xa, xb = to_dev(a, gpu), to_dev(b, gpu)
            reqs.append((a, b, xa, xb, xc))
        torch.cuda.synchronize()
        ts = [B.polymul_server_submit(srv, p, xa, len(a) - 1, xb, len(b) - 1, xc) for a, b, xa, xb, xc in reqs]
        for t in ts:
            B.polymul_server_wait(srv, t, 60000)
    finally:
        B.polymul_server_destroy(srv)
    for a, b, _, _, xc in reqs[:10]:
        assert np.array_equal(from_dev(xc), orc.polymul_tft(p, a, b))


def test_autotune_writes_and_loads_schedules(gpu, orc, tmp_path):
    import json
    import torch
    from paper_1609_01010_gb300 import binding as B
    path = str(tmp_path / "sched.json")
    B.polymul_autotune(W.P1, 14, 17, path)
    with open(path) as f:
        table = json.load(f)
    assert [r["l"] for r in table["schedules"]] == [14, 15, 16, 17]
    for r in table["schedules"]:
        assert 9 <= r["sigma"] <= 13 and r["C"] in (8, 32, 128) and r["us"] > 0
        assert r["batch_C"] in (8, 32, 128, 256, 512, 1024, 2048) and r["batch_us"] > 0
    B.polymul_load_schedules(path)
    p, a, b = W.workload3(1 << 16)
    dc = torch.empty(2 * len(a) - 1, dtype=torch.int32, device=gpu)
    B.polymul_mod(p, to_dev(a, gpu), len(a) - 1, to_dev(b, gpu), len(b) - 1, dc)
    assert np.array_equal(from_dev(dc), orc.polymul_tft(p, a, b))
    assert os.path.getsize(path) > 0


def test_batch_tile_widths_from_the_table(gpu, orc, tmp_path):
    """Every valid column-tile width per size class (8 to 2048 columns, where
    the tile fits 64 KB), loaded from a schedule table ("batch_C"), gives the
    oracle's products; the table is restored."""
    import json
    import torch
    from paper_1609_01010_gb300 import binding as B
    saved = {l: B.polymul_get_batch_width(l) for l in range(14, 18)}
    sched = {l: B.polymul_get_schedule(l) for l in range(14, 18)}
    p, a, a_off, b, b_off, c_off = W.workload4(count=48, seed=W.SEED_BASE + 44)
    da, db = to_dev(a, gpu), to_dev(b, gpu)
    want = orc.polymul_tft_batch(p, a, a_off, b, b_off, c_off)
    path = tmp_path / "widths.json"

    def load(widths):
        rows = [{"l": l, "sigma": sched[l][0], "C": sched[l][1], "us": 0.0, "batch_C": widths[l]}
                for l in range(14, 18)]
        path.write_text(json.dumps({"device": "test", "p": p, "schedules": rows}))
        B.polymul_load_schedules(str(path))
    def fits(l, C):  # a tile of 2^(l-12) rows x C words within 64 KB
        return (C << (l - 12)) * 4 <= 64 * 1024
    try:
        for C in (8, 32, 128, 256, 512, 1024, 2048):
            widths = {l: C if fits(l, C) else 8 for l in range(14, 18)}
            load(widths)
            assert all(B.polymul_get_batch_width(l) == widths[l] for l in range(14, 18))
            dc = torch.full((int(c_off[-1]),), -1, dtype=torch.int32, device=gpu)
            B.polymul_mod_batched(p, da, a_off, db, b_off, dc, c_off)
            torch.cuda.synchronize()
            assert np.array_equal(from_dev(dc), want), C
    finally:
        load(saved)
