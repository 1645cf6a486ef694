"""The debug build (libpolymul_debug.so, kernels compiled with their range
and index checks): products through every kernel family equal the oracle and
leave the device status word clean, and inputs outside [0, p) -- which the
release kernels do not check -- make a range check report
POLY_EDEBUG_CHECK through the status word instead of trapping."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import oracle
from paper_1609_01010_gb300 import binding as B
from paper_1609_01010_gb300 import workloads as W
assert B.LIB_PATH.endswith("libpolymul_debug.so"), B.LIB_PATH
dev = torch.device("cuda:0")
def d(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(dev)
def h(t):
    return t.cpu().numpy().view(np.uint32)
B.lib()
B.polymul_device_status(clear=True)
rng = np.random.default_rng(9)
bad = []
def check(name, got, want):
    if not np.array_equal(got, want):
        bad.append(name)
# single products: one CTA, the three-kernel path (8- and 32-column tiles), padded, both primes
for p in (W.P1, W.P2):
    for z1, z2 in [(300, 200), (3001, 5001), (40000, 65537), (1 << 19, 300000)]:
        a = rng.integers(0, p, z1, dtype=np.uint32); b = rng.integers(0, p, z2, dtype=np.uint32)
        c = torch.empty(z1 + z2 - 1, dtype=torch.int32, device=dev)
        B.polymul_mod_async(p, d(a), z1 - 1, d(b), z2 - 1, c); torch.cuda.synchronize()
        want = oracle.polymul_tft(p, a, b)
        check(f"mod {{p}} {{z1}} {{z2}}", h(c), want)
        Lp = 1 << (z1 + z2 - 2).bit_length()
        B.polymul_mod_padded_async(p, d(a), z1 - 1, d(b), z2 - 1, c, Lp); torch.cuda.synchronize()
        check(f"padded {{p}} {{z1}} {{z2}}", h(c), want)
path = "/tmp/dbg_sched.json"
json.dump({{"device": "x", "p": 0, "schedules": [{{"l": 17, "sigma": 10, "C": 32, "us": 0}},
                                                {{"l": 20, "sigma": 11, "C": 32, "us": 0}}]}}, open(path, "w"))
B.polymul_load_schedules(path)
for z1, z2 in [(40000, 65537), (1 << 19, 300000)]:
    p = W.P1
    a = rng.integers(0, p, z1, dtype=np.uint32); b = rng.integers(0, p, z2, dtype=np.uint32)
    c = torch.empty(z1 + z2 - 1, dtype=torch.int32, device=dev)
    B.polymul_mod_async(p, d(a), z1 - 1, d(b), z2 - 1, c); torch.cuda.synchronize()
    check(f"tma {{z1}} {{z2}}", h(c), oracle.polymul_tft(p, a, b))
# batch, convolutions, general radix, allocation-free
p, a, a_off, b, b_off, c_off = W.workload4(count=64, seed=W.SEED_BASE + 43)
c = torch.empty(int(c_off[-1]), dtype=torch.int32, device=dev)
B.polymul_mod_batched(p, d(a), a_off, d(b), b_off, c, c_off); torch.cuda.synchronize()
check("batch", h(c), oracle.polymul_tft_batch(p, a, a_off, b, b_off, c_off))
p = W.P2
a = rng.integers(0, p, 4096, dtype=np.uint32); b = rng.integers(0, p, 3000, dtype=np.uint32)
c = torch.empty(4096, dtype=torch.int32, device=dev)
B.polymul_negacyclic_async(p, d(a), 4096, d(b), 3000, c, 4096); torch.cuda.synchronize()
A = np.zeros(4096, np.uint32); A[:] = a; Bv = np.zeros(4096, np.uint32); Bv[:3000] = b
check("negacyclic", h(c), oracle.negacyclic(p, A, Bv))
a = rng.integers(0, p, 300001, dtype=np.uint32); b = rng.integers(0, p, 400001, dtype=np.uint32)
c = torch.empty(700001, dtype=torch.int32, device=dev)
B.polymul_mod_radix_async(p, d(a), 300000, d(b), 400000, c, 3); torch.cuda.synchronize()
check("radix3", h(c), oracle.polymul_tft(p, a, b))
a = rng.integers(0, p, 30000, dtype=np.uint32); b = rng.integers(0, p, 20000, dtype=np.uint32)
c = torch.empty(49999, dtype=torch.int32, device=dev)
B.polymul_mod_noalloc_async(p, d(a), 29999, d(b), 19999, c); torch.cuda.synchronize()
check("noalloc", h(c), oracle.polymul_tft(p, a, b))
clean = B.polymul_device_status(clear=True)
# inputs far outside [0, p) (never validated here): the range checks report
p = W.P1
a = np.full(70000, 0xFFFFFFFF, np.uint32)
c = torch.empty(2 * 70000 - 1, dtype=torch.int32, device=dev)
B.polymul_mod_async(p, d(a), 69999, d(a), 69999, c); torch.cuda.synchronize()
tripped = B.polymul_device_status(clear=True)
print(json.dumps({{"bad": bad, "clean": clean, "tripped": tripped}}))
sys.exit(0 if (not bad and clean == 0 and tripped == -11) else 1)
"""


def test_debug_build_parity_and_range_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-m", "paper_1609_01010_gb300.build", "--debug"], cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, POLYMUL_DEBUG_LIB="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
