"""The allocation-free entry point (polymul_mod_noalloc_async).

Callers that cannot let a library allocate device memory (their memory is
reserved up front by their own allocator, or they cannot afford the
synchronisation cudaMalloc/cudaFree may cause) use this entry point; its
workspace is a static device array inside the library.  Its output must equal
polymul_mod_async's on the same inputs, on two calls in a row (the second
call reuses the workspace the first one left behind).  The file is collected
last so a failure here stops a -x run only after every other test ran; it also
passes alone in a fresh process (the first call sets the static tables up).
"""
import numpy as np
import pytest

from paper_1609_01010_gb300 import workloads as W

pytestmark = pytest.mark.gpu

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


def test_noalloc_equals_polymul_mod_on_two_calls_in_a_row(gpu):
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
        for _ in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device=gpu)
            B.polymul_mod_noalloc_async(p, da, z1 - 1, db, z2 - 1, out)
            torch.cuda.synchronize()
            # exact integer results: the tolerance is zero
            assert torch.equal(out, ref), (p, z1, z2)


def test_noalloc_rejects_sizes_beyond_its_limit(gpu):
    import torch
    from paper_1609_01010_gb300 import binding as B
    buf = torch.zeros(1 << 18, dtype=torch.int32, device=gpu)  # large enough for any call below
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod_noalloc_async(W.P1, buf, 65536, buf, 65536, buf)  # n = 131073 > 2^17
    assert e.value.status == -2
    with pytest.raises(B.PolymulError) as e:
        B.polymul_mod_noalloc_async(97, buf, 10, buf, 10, buf)  # not a built-in prime
    assert e.value.status == -1
