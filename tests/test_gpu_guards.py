"""Guard words around every entry point's device buffers (the substitute for
a memory sanitizer, which this pool does not offer): operands and outputs
sit between canary regions inside one allocation; after each call the
canaries must be intact, the operands unchanged, and the output equal to the
oracle.  Shapes cover the one-CTA and three-kernel paths with ragged tails
(lengths that are not multiples of 4 words, operands at odd word offsets)."""
import numpy as np
import pytest

from oracle import integer as I
from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 1024  # words of canary before and after each buffer
CANARY = np.uint32(0xA5C3F00D)


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01010_gb300 import binding
    binding.lib()
    return torch.device("cuda:0")


class Arena:
    """One device allocation: [guard | buf0 | guard | buf1 | guard | ...]; each
    buffer starts one word past a 16-byte boundary, so nothing is aligned."""

    def __init__(self, dev, contents):
        import torch
        self.spans = []
        host = []
        pos = 0
        for x in contents:
            x = np.asarray(x, dtype=np.uint32)
            host.append(np.full(GUARD + 1, CANARY, dtype=np.uint32))
            pos += GUARD + 1
            self.spans.append((pos, len(x)))
            host.append(x)
            pos += len(x)
        host.append(np.full(GUARD, CANARY, dtype=np.uint32))
        self.host = np.concatenate(host)
        self.t = torch.from_numpy(self.host.view(np.int32).copy()).to(dev)

    def ptr(self, i):
        return self.t.data_ptr() + 4 * self.spans[i][0]

    def check(self, keep, out):
        """Canaries intact, buffers in `keep` unchanged; returns the buffers in `out`."""
        got = self.t.cpu().numpy().view(np.uint32)
        mask = np.ones(len(got), dtype=bool)
        for s, n in self.spans:
            mask[s:s + n] = False
        assert np.all(got[mask] == CANARY), "a canary word was overwritten"
        for i in keep:
            s, n = self.spans[i]
            assert np.array_equal(got[s:s + n], self.host[s:s + n]), f"input buffer {i} was modified"
        return [got[self.spans[i][0]:self.spans[i][0] + self.spans[i][1]] for i in out]


def sync():
    import torch
    torch.cuda.synchronize()


SHAPES = [(1, 1), (7, 3), (300, 211), (513, 600), (3001, 5001), (40001, 30003), (100003, 77777)]


@pytest.mark.parametrize("za,zb", SHAPES)
def test_product_entry_points_stay_inside_their_buffers(gpu, orc, za, zb):
    from paper_1609_01010_gb300 import binding as B
    p = W.P1
    a, b = W.operands(W.SEED_BASE + 400 + za, za - 1, zb - 1, p)
    n = za + zb - 1
    want = orc.polymul_tft(p, a, b)
    L = 1 << (n - 1).bit_length()
    calls = [
        ("polymul_mod_async", lambda A: B.polymul_mod_async(p, A.ptr(0), za - 1, A.ptr(1), zb - 1, A.ptr(2))),
        ("polymul_mod_padded_async",
         lambda A: B.polymul_mod_padded_async(p, A.ptr(0), za - 1, A.ptr(1), zb - 1, A.ptr(2), max(L, 512))),
    ]
    if n <= (1 << 17):
        calls.append(("polymul_mod_noalloc_async",
                      lambda A: B.polymul_mod_noalloc_async(p, A.ptr(0), za - 1, A.ptr(1), zb - 1, A.ptr(2))))
    for name, call in calls:
        A = Arena(gpu, [a, b, np.zeros(n, np.uint32)])
        call(A)
        sync()
        (c,) = A.check(keep=(0, 1), out=(2,))
        assert np.array_equal(c, want), name


@pytest.mark.parametrize("N", [5, 512, 1000, 4096, 16384])
def test_convolutions_stay_inside_their_buffers(gpu, orc, N):
    from paper_1609_01010_gb300 import binding as B
    p = W.P2
    za, zb = N, max(1, N // 3)
    a, b = W.operands(W.SEED_BASE + 500 + N, za - 1, zb - 1, p)
    A_ = np.zeros(N, np.uint32)
    B_ = np.zeros(N, np.uint32)
    A_[:za], B_[:zb] = a, b
    for kind in ("cyclic", "negacyclic"):
        fn = B.polymul_cyclic_async if kind == "cyclic" else B.polymul_negacyclic_async
        A = Arena(gpu, [a, b, np.zeros(N, np.uint32)])
        fn(p, A.ptr(0), za, A.ptr(1), zb, A.ptr(2), N)
        sync()
        (c,) = A.check(keep=(0, 1), out=(2,))
        want = orc.cyclic(p, A_, B_) if kind == "cyclic" else orc.negacyclic(p, A_, B_)
        assert np.array_equal(c, want), kind


@pytest.mark.parametrize("za,zb", [(1, 1), (300, 211), (3001, 5001), (20001, 13003)])
def test_three_primes_and_radix_stay_inside_their_buffers(gpu, orc, za, zb):
    from paper_1609_01010_gb300 import binding as B
    a32, b32 = W.workload6(za, zb)
    n = za + zb - 1
    A = Arena(gpu, [a32, b32, np.zeros(3 * n, np.uint32)])
    B.polymul_crt3_async(A.ptr(0), za - 1, A.ptr(1), zb - 1, A.ptr(2))
    sync()
    (c,) = A.check(keep=(0, 1), out=(2,))
    assert np.array_equal(c.reshape(-1, 3), I.int_product(a32, b32))
    p = W.P2
    a, b = W.operands(W.SEED_BASE + 600 + za, za - 1, zb - 1, p)
    want = orc.polymul_tft(p, a, b)
    for m in (3, 5, 15):
        A = Arena(gpu, [a, b, np.zeros(n, np.uint32)])
        B.polymul_mod_radix_async(p, A.ptr(0), za - 1, A.ptr(1), zb - 1, A.ptr(2), m)
        sync()
        (c,) = A.check(keep=(0, 1), out=(2,))
        assert np.array_equal(c, want), m


def test_batch_stays_inside_its_buffers(gpu, orc):
    """A packed batch whose operands and outputs are each surrounded by the
    arena's canaries (one product per slot, offsets relative to slot 0)."""
    from paper_1609_01010_gb300 import binding as B
    p = W.P2
    shapes = [(5, 9), (700, 300), (5000, 3001), (20001, 12000), (1, 1), (65537, 40000)]
    ops = [W.operands(W.SEED_BASE + 700 + i, za - 1, zb - 1, p) for i, (za, zb) in enumerate(shapes)]
    # all a's back to back, all b's, all c's; canaries around each packed array
    a = np.concatenate([x for x, _ in ops])
    b = np.concatenate([y for _, y in ops])
    za = np.array([s[0] for s in shapes], dtype=np.int64)
    zb = np.array([s[1] for s in shapes], dtype=np.int64)
    a_off = np.concatenate([[0], np.cumsum(za)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(zb)]).astype(np.int64)
    c_off = np.concatenate([[0], np.cumsum(za + zb - 1)]).astype(np.int64)
    A = Arena(gpu, [a, b, np.zeros(int(c_off[-1]), np.uint32)])
    B.polymul_mod_batched(p, A.ptr(0), a_off, A.ptr(1), b_off, A.ptr(2), c_off)
    sync()
    (c,) = A.check(keep=(0, 1), out=(2,))
    for i, (x, y) in enumerate(ops):
        assert np.array_equal(c[c_off[i]:c_off[i + 1]], orc.polymul_tft(p, x, y)), i
