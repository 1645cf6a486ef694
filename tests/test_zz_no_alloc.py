"""The allocation-free entry point (polymul_mod_noalloc_async).

Some callers cannot let a library allocate device memory: applications that
reserve all device memory up front in their own pool (a library cudaMalloc
would fail, or bypass their accounting), and latency-critical callers that
cannot afford the device-wide synchronisation cudaMalloc/cudaFree may cause.
This entry point serves them: its workspace is a static device array inside
the library.  Its output must equal polymul_mod_async's and the oracle's on
the same inputs, on two calls in a row (the second call reuses the workspace
the first one left behind), and the second call must leave the device's
memory accounting unchanged.  The file is collected last so a failure here
stops a -x run only after every other test ran; it also passes alone in a
fresh process (the first call sets the static tables up), and a separate
fresh process makes its very first call on a non-blocking side stream.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (prime, z1, z2): one-CTA sizes, three-kernel sizes up to the 2^17 limit
CASES = [(W.P1, 1, 1), (W.P2, 64, 100), (W.P1, 1024, 1024), (W.P2, 3001, 5001),
         (W.P1, 5000, 3194), (W.P2, 4097, 4097), (W.P1, 30000, 20000), (W.P2, 65536, 65537),
         (W.P1, 100000, 31073)]


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01010_gb300 import binding
    binding.lib()
    return torch.device("cuda:0")


def pool_usage(dev_index):
    """(used, reserved) bytes of the device's default stream-ordered memory
    pool, through the driver API (the pool cudaMallocAsync draws from)."""
    cu = ctypes.CDLL("libcuda.so.1")
    assert cu.cuInit(0) == 0
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), dev_index) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    out = []
    for attr in (7, 5):  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT, CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        out.append(v.value)
    return tuple(out)


def test_noalloc_equals_polymul_mod_on_two_calls_in_a_row(gpu, orc):
    import torch
    from paper_1609_01010_gb300 import binding as B
    for p, z1, z2 in CASES:
        a = W.coeffs(W.SEED_BASE + 70 + z1, z1, p)
        b = W.coeffs(W.SEED_BASE + 71 + z2, z2, p)
        da = torch.from_numpy(a.view(np.int32)).to(gpu)
        db = torch.from_numpy(b.view(np.int32)).to(gpu)
        n = z1 + z2 - 1
        ref = torch.full((n,), -1, dtype=torch.int32, device=gpu)
        B.polymul_mod_async(p, da, z1 - 1, db, z2 - 1, ref)
        want = orc.polymul_tft(p, a, b)
        outs = [torch.full((n,), -1, dtype=torch.int32, device=gpu) for _ in range(2)]
        torch.cuda.synchronize()
        for i in range(2):
            if i == 1:
                before = (pool_usage(gpu.index or 0), torch.cuda.mem_get_info(gpu))
            B.polymul_mod_noalloc_async(p, da, z1 - 1, db, z2 - 1, outs[i])
            torch.cuda.synchronize()
            if i == 1:
                after = (pool_usage(gpu.index or 0), torch.cuda.mem_get_info(gpu))
                assert before == after, (p, z1, z2, before, after)
            # exact integer results: the tolerance is zero
            assert torch.equal(outs[i], ref), (p, z1, z2, i)
            assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), want), (p, z1, z2, i)


FIRST_CALL_ON_SIDE_STREAM = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import oracle
from paper_1609_01010_gb300 import binding as B
from paper_1609_01010_gb300 import workloads as W
dev = torch.device("cuda:0")
jobs = []
for p, z1, z2 in [(W.P1, 30000, 20000), (W.P2, 700, 300)]:
    a = W.coeffs(W.SEED_BASE + 80 + z1, z1, p)
    b = W.coeffs(W.SEED_BASE + 81 + z2, z2, p)
    jobs.append((p, a, b, torch.from_numpy(a.view(np.int32)).to(dev), torch.from_numpy(b.view(np.int32)).to(dev)))
torch.cuda.synchronize()
side = torch.cuda.Stream(device=dev)  # a non-blocking stream
ok = True
for p, a, b, da, db in jobs:
    c = torch.full((len(a) + len(b) - 1,), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    B.polymul_mod_noalloc_async(p, da, len(a) - 1, db, len(b) - 1, c, side.cuda_stream)
    side.synchronize()
    ok = ok and np.array_equal(c.cpu().numpy().view(np.uint32), oracle.polymul_tft(p, a, b))
sys.exit(0 if ok else 1)
"""


def test_noalloc_first_call_of_a_process_on_a_side_stream(gpu):
    """A fresh process whose very first call (the one that sets the static
    tables up) runs on a non-blocking torch stream: the product must already
    equal the oracle's."""
    r = subprocess.run([sys.executable, "-c", FIRST_CALL_ON_SIDE_STREAM.format(root=ROOT)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def test_noalloc_rejects_sizes_beyond_its_limit(gpu):
    import torch
    from paper_1609_01010_gb300 import binding as B
    buf = torch.zeros(1 << 18, dtype=torch.int32, device=gpu)  # large enough for any call below
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod_noalloc_async(W.P1, buf, 65536, buf, 65536, buf)  # n = 131073 > 2^17
    assert e.value.status == -2
    L = B.lib()
    # degrees near the int64 limit are rejected without overflowing n = da + db + 1
    assert L.polymul_mod_noalloc_async(W.P1, buf.data_ptr(), (1 << 63) - 1, buf.data_ptr(), (1 << 63) - 1,
                                       buf.data_ptr(), None) == -2
    assert L.polymul_mod_noalloc_async(W.P1, buf.data_ptr(), 1, buf.data_ptr(), (1 << 63) - 1,
                                       buf.data_ptr(), None) == -2
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod_noalloc_async(97, buf, 10, buf, 10, buf)  # not a built-in prime
    assert e.value.status == -1
