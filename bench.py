"""Benchmark of the TFT polynomial product mod p on GB300 (one JSON line).

Headline workload: one product mod 469762049 of two operands of 2^20
coefficients (degree 2^20 - 1), n = 2^21 - 1, L = 2^21 -- the length at which
the roofline target is quoted.  A step is one full product (plan resident;
TFT of both operands, pointwise product, ITFT) on inputs already in device
memory; 16 rotating input/output sets (268 MB, more than the 129 MB L2) keep
each step's operands out of L2.  value = n / step time (coefficients/s).

The same line also carries:
  e2e          the same product through polymul_mod_host (pinned host buffers,
               both copies inside the timed region);
  roofline     the dominant kernel (row stage) against the measured butterfly
               peak of this GPU (polymul_probe_int), its duration taken with
               CUDA events over a profiled timed pass;
  cpu_baseline the CPU oracle timed on a bounded sample on all host cores (one
               product per worker process) and on one core;
  small_configs  workload 1 (full NTT 2048) and workload 2 (degrees 3000 x 5000
               mod 2013265921, TFT length 8001, against zero-padded NTTs of 8192
               and 16384, Eq. (12)): device time per product from CUDA-graph
               replay, and the back-to-back call rate;
  step_distribution  p10/p50/p90 of the headline product over 200 runs, cold
               and warm L2;
  sweep        the large single products (d+1 in 2^16, 2^20, 2^22, 100000,
               1500000, 3000001): time, coeffs/s, compulsory-HBM fraction;
  crt3         exact integer products of 32-bit-coefficient operands (three
               primes and the CRT, Section 1) at z = 2^16, 2^20, 3000001,
               against three modular products of the same size;
  radix        general-radix products (transform length m 2^k, m = 3, 5, 15)
               against the power-of-two TFT product between 2^20 and 2^21;
  length_sweep the shape of the paper's Fig. 3: TFT product against the
               power-of-two zero-padded NTT product for n in [2^14, 2^22],
               eight lengths per octave;
  batched      4096 products (degrees log-uniform in [64, 65536]) in one
               persistent launch under a CUDA graph vs 4096 plain calls;
  serving      Poisson request stream into the continuous-batching server:
               p50/p99 latency and throughput.

--impl reference times the CPU oracle on the same workload and metric.
Multi-GPU (torchrun): each rank runs the same workload on its own GPU
(replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1609_01010_gb300 import workloads as W  # noqa: E402

METRIC = "mod-p polymul coeffs/s & HBM GB/s vs peak; batched/serve vs plain; p99 latency"
HEAD_Z = 1 << 20
L2_BYTES = 129 * 1024 * 1024
REF_BUDGET_S = 120.0


# DRAM bytes (read + write) of one k_row_fused launch at the headline size,
# from ncu (dram__bytes_read.sum + dram__bytes_write.sum, medians over 20
# launches) on the sources whose digest is recorded here; any later change to
# those sources makes the figures stale and they read null.  "bytes": with
# --cache-control none, so L2 holds what the previous kernels left there, as
# in the timed stream of products (the column stage's rows and the resident
# twiddle tables are L2 hits); "bytes_cold_l2": with ncu's default cache
# control, which flushes L2 before the launch (rows and twiddles from DRAM).
ROW_TRAFFIC = {"bytes": 270976 + 486400, "bytes_cold_l2": 50368512 + 0, "sources_sha256_16": "88150487902e5a2c"}
ROW_SOURCES = ("device.cuh", "bodies.cuh", "k_large.cuh", "modarith.cuh", "internal.h")


def row_kernel_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in ROW_SOURCES:
        with open(os.path.join(ROOT, "paper_1609_01010_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    ok = h.hexdigest()[:16] == ROW_TRAFFIC["sources_sha256_16"]
    return (ROW_TRAFFIC["bytes"], ROW_TRAFFIC["bytes_cold_l2"]) if ok else (None, None)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the measured region (clocks, throttle reasons)."""
    Q = ("clocks.sm,clocks.max.sm,utilization.gpu,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [r for r in rows if r[2] >= 30] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


# ---------------------------------------------------------------- helpers
def dev_u32(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(dev)


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def ev_time(fn, reps, stream):
    """Milliseconds per call of fn() over `reps` calls, CUDA events on `stream`."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        fn(i)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_value(units_per_rank, ms, world):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def max_over_ranks(x, world, dev):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle
def _oracle_product_worker(z):
    """One headline-size product by the oracle in a worker process (spawned)."""
    import oracle
    from paper_1609_01010_gb300 import workloads as WW
    p, a, b = WW.workload3(z)
    t0 = time.perf_counter()
    oracle.polymul_tft(p, a, b)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(sample_products: int = 2):
    """The oracle as it stands on the host cores: coefficients/s on the
    headline workload, on one core (products one after another) and on all
    cores (one product per worker process, all at once)."""
    import multiprocessing as mp
    import oracle
    p, a, b = W.workload3(HEAD_Z)
    n = len(a) + len(b) - 1
    oracle.polymul_tft(p, a[:1024], b[:1024])  # build/load
    t0 = time.perf_counter()
    for _ in range(sample_products):
        oracle.polymul_tft(p, a, b)
    dt = (time.perf_counter() - t0) / sample_products
    one = {"value": n / dt, "unit": "coeffs/s", "cores": 1, "kind": "oracle",
           "sample": f"{sample_products} full products of the headline workload (d+1 = 2^20 each, n = {n}) one "
                     f"after another on one core, recursive TFT/ITFT oracle, {dt:.2f} s per product"}
    cores = host_cores()
    # spawn: this process already holds a CUDA context, which forked workers must not inherit
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_product_worker, [1 << 10] * cores)  # start-up and library load, untimed
        t0 = time.perf_counter()
        per = pool.map(_oracle_product_worker, [HEAD_Z] * cores)
        wall = time.perf_counter() - t0
    allc = {"value": cores * n / wall, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} full headline products at once, one per worker process on {cores} host cores "
                      f"(os.sched_getaffinity), {wall:.2f} s wall, {statistics.median(per):.2f} s median per "
                      f"product"}
    out = dict(allc)
    out["single_core"] = one
    out["nproc"] = os.cpu_count()
    return out


def run_reference(args):
    """The oracle on the host cores: each step is one round of `cores` full
    headline products, one per worker process at once (the oracle itself is
    sequential); value = products' coefficients / wall time."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import multiprocessing as mp
    p, a, b = W.workload3(HEAD_Z)
    n = len(a) + len(b) - 1
    cores = host_cores()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_product_worker, [1 << 10] * cores)
        for _ in range(args.warmup):
            pool.map(_oracle_product_worker, [1 << 14] * cores)
        # Each step is one round of full products (several seconds); steps
        # stop after REF_BUDGET_S seconds so that any --steps finishes within
        # a few minutes.
        t0 = time.perf_counter()
        done = 0
        while done < args.steps and (done == 0 or time.perf_counter() - t0 < REF_BUDGET_S):
            pool.map(_oracle_product_worker, [HEAD_Z] * cores)
            done += 1
        dt = (time.perf_counter() - t0) / done
    v = cores * n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "coeffs/s", "n_gpus": args.gpus,
            "steps": done, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"tft_polymul_p{p}_z{HEAD_Z}", "p": p, "z1": HEAD_Z, "z2": HEAD_Z, "n": n,
                       "L": 1 << 21, "impl": "CPU oracle (plain C, recursive TFT/ITFT, 64-bit %)"},
            "cpu_baseline": {"value": v, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{done} of {args.steps} requested rounds timed (budget "
                                       f"{REF_BUDGET_S:.0f} s), each round {cores} full headline products at "
                                       f"once, one per worker process, after {args.warmup} warm-up rounds of "
                                       f"2^14-coefficient operands"},
            "e2e": {"value": v, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU parts
def headline(args, dev, stream, B, world):
    """Timed region: K products on rotating device buffers."""
    import torch
    p, a, b = W.workload3(HEAD_Z)
    z = HEAD_Z
    n = 2 * z - 1
    sets = 16
    A = torch.empty((sets, z), dtype=torch.int32, device=dev)
    Bm = torch.empty((sets, z), dtype=torch.int32, device=dev)
    Cm = torch.empty((sets, n), dtype=torch.int32, device=dev)
    da, db = dev_u32(a, dev), dev_u32(b, dev)
    for i in range(sets):  # same operands, distinct memory (L2-cold per step)
        A[i].copy_(da)
        Bm[i].copy_(db)
    sh = stream.cuda_stream
    ptrs = [(A[i].data_ptr(), Bm[i].data_ptr(), Cm[i].data_ptr()) for i in range(sets)]

    def step(i):
        pa, pb, pc = ptrs[i % sets]
        B.polymul_mod_async(p, pa, z - 1, pb, z - 1, pc, sh)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
        # soak so the clock sampler sees the GPU under this load
        t_end = time.perf_counter() + args.soak
        i = 0
        while time.perf_counter() < t_end:
            step(i)
            i += 1
            if i % 256 == 0:
                stream.synchronize()
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ms = ev_time(step, args.steps, stream)
        torch.cuda.synchronize()
        barrier(world)
        # correctness of the timed outputs (sampled against Definition 2)
        got = host_u32(Cm[(args.steps - 1) % sets])
    return p, z, n, ms, got, a, b, step, ptrs


def step_distribution(stream, B, p, z, ptrs, reps=200):
    """Per-product device time (CUDA events around each product) over `reps`
    products: cold L2 (the 16 rotating buffer sets, 400 MB, each product's
    operands evicted by the others) and warm L2 (one set, 25 MB, resident).
    An event between two products keeps the next product's first kernel from
    starting under the previous one's last (programmatic dependent launch), so
    these times are slightly above the back-to-back mean of the headline."""
    import torch
    sh = stream.cuda_stream
    sets = len(ptrs)
    out = {}
    for name, pick in (("cold_l2", lambda i: ptrs[i % sets]), ("warm_l2", lambda i: ptrs[0])):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        with torch.cuda.stream(stream):
            for i in range(10):
                pa, pb, pc = pick(i)
                B.polymul_mod_async(p, pa, z - 1, pb, z - 1, pc, sh)
            for i in range(reps):
                pa, pb, pc = pick(i)
                evs[i][0].record(stream)
                B.polymul_mod_async(p, pa, z - 1, pb, z - 1, pc, sh)
                evs[i][1].record(stream)
            stream.synchronize()
        us = np.array([a.elapsed_time(b) * 1e3 for a, b in evs])
        out[name] = {"p10_us": float(np.percentile(us, 10)), "p50_us": float(np.percentile(us, 50)),
                     "p90_us": float(np.percentile(us, 90)), "mean_us": float(us.mean()), "runs": reps}
    return out


def profiled_pass(args, stream, step):
    """Same K steps again with per-kernel CUDA events (row/column stages)."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    with torch.cuda.stream(stream):
        B.polymul_profile_begin()
        for i in range(args.steps):
            step(i)
        stream.synchronize()
        ms, cnt = B.polymul_profile_end()
    return ms, cnt


def e2e_pass(args, p, a, b, streams=3):
    """End to end from pinned host buffers through the public API: each step
    copies its operands in, computes and copies its product back
    (polymul_mod_host_async); steps rotate over `streams` streams with their
    own buffer sets, so one step's host-link copies run while another
    computes.  Wall-clock time from the first call to the last stream's end.
    Beside it, the synchronous polymul_mod_host latency of one product."""
    import torch
    from paper_1609_01010_gb300 import binding as B
    z = len(a)
    n = 2 * z - 1
    sets = []
    for _ in range(streams):
        ha = torch.from_numpy(a.view(np.int32)).pin_memory()
        hb = torch.from_numpy(b.view(np.int32)).pin_memory()
        hc = torch.empty(n, dtype=torch.int32).pin_memory()
        # the tensors stay referenced: freed pinned memory would be handed to the next set
        sets.append((torch.cuda.Stream(), ha.data_ptr(), hb.data_ptr(), hc, hc.data_ptr(), ha, hb))
    L = B.lib()

    def run(k):
        for i in range(k):
            st, pa, pb, _, pc = sets[i % streams][:5]
            assert L.polymul_mod_host_async(p, pa, z - 1, pb, z - 1, pc, st.cuda_stream) == 0
        for st, *_ in sets:
            st.synchronize()
    run(2 * streams)
    reps = max(3 * streams, min(args.steps, 60))
    t0 = time.perf_counter()
    run(reps)
    dt = (time.perf_counter() - t0) / reps
    ok = sampled_ok(sets[(reps - 1) % streams][3].numpy().view(np.uint32), a, b, p, [0, n // 2, n - 1])
    for _ in range(3):
        L.polymul_mod_host(p, sets[0][1], z - 1, sets[0][2], z - 1, sets[0][4])
    t0 = time.perf_counter()
    for _ in range(10):
        L.polymul_mod_host(p, sets[0][1], z - 1, sets[0][2], z - 1, sets[0][4])
    lat = (time.perf_counter() - t0) / 10
    return {"value": n / dt, "unit": "coeffs/s", "h2d_bytes_per_step": 8 * z, "d2h_bytes_per_step": 4 * n,
            "ms_per_step": dt * 1e3, "steps": reps, "streams": streams, "correct_sampled": bool(ok),
            "sync_latency_ms": lat * 1e3,
            "api": "polymul_mod_host_async on pinned host buffers (copy engines in and out, staged through a "
                   "stream-ordered device buffer), steps rotating over the streams; sync_latency_ms: one "
                   "polymul_mod_host call alone"}


def sampled_ok(c, a, b, p, ks):
    A = a.astype(np.uint64)
    Bv = b.astype(np.uint64)
    for k in ks:
        lo = max(0, k - (len(b) - 1))
        hi = min(k, len(a) - 1)
        want = int(((A[lo:hi + 1] * Bv[k - hi:k - lo + 1][::-1]) % p).sum() % p)
        if int(c[k]) != want:
            return False
    return True


def graph_device_us(call, stream, per_graph=200, replays=10):
    """Device time per call: `per_graph` calls captured into one CUDA graph
    (through the public C ABI) and replayed; no host launch cost inside."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(5):
            call()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(per_graph):
                call()
        g.replay()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(replays):
            g.replay()
        e1.record(stream)
        e1.synchronize()
    return e0.elapsed_time(e1) / (per_graph * replays) * 1e3


def small_configs(dev, stream, B):
    """Workloads 1 and 2: degree-1023 operands (full NTT 2048) and degrees
    3000 x 5000 mod 2013265921 (TFT length 8001) against the zero-padded
    NTTs of 8192 and 16384 (Eq. (12)).  Per product: the back-to-back call
    rate from one host thread (host launch cost included) and the device
    time from CUDA-graph replay."""
    import torch
    L = B.lib()
    sh = stream.cuda_stream
    out = {}
    for wname, (p, a, b) in (("workload1_ntt2048", W.workload1()), ("workload2_tft8001", W.workload2())):
        n = len(a) + len(b) - 1
        da, db = dev_u32(a, dev), dev_u32(b, dev)
        dc = torch.empty(n, dtype=torch.int32, device=dev)
        pa, pb, pc = da.data_ptr(), db.data_ptr(), dc.data_ptr()
        cases = [("tft", None)] if wname.startswith("workload1") else [("tft", None), ("padded_ntt_8192", 8192),
                                                                          ("padded_ntt_16384", 16384)]
        res = {"p": p, "n": n, "z1": len(a), "z2": len(b)}
        for name, Lp in cases:
            if Lp:
                def call(Lp=Lp):
                    assert L.polymul_mod_padded_async(p, pa, len(a) - 1, pb, len(b) - 1, pc, Lp, sh) == 0
            else:
                def call():
                    assert L.polymul_mod_async(p, pa, len(a) - 1, pb, len(b) - 1, pc, sh) == 0
            with torch.cuda.stream(stream):
                for _ in range(20):
                    call()
                rate_us = ev_time(lambda i: call(), 500, stream) * 1e3
            res[name] = {"device_us": graph_device_us(call, stream), "call_rate_us": rate_us}
        want = sampled_ok(host_u32(dc), a, b, p, [0, n // 2, n - 1])
        res["correct_sampled"] = bool(want)
        if "padded_ntt_16384" in res:
            res["device_speedup_vs_padded_16384"] = res["padded_ntt_16384"]["device_us"] / res["tft"]["device_us"]
            res["device_speedup_vs_padded_8192"] = res["padded_ntt_8192"]["device_us"] / res["tft"]["device_us"]
        out[wname] = res
    out["note"] = ("device_us: CUDA graph of 200 calls through the C ABI, replayed (device time per product); "
                   "call_rate_us: 500 back-to-back calls from one host thread, CUDA events (bounded by the host "
                   "launch cost at these sizes)")
    return out


def length_sweep(dev, stream, B, lo=14, hi=22, per_octave=8, reps=20):
    """The shape of the paper's Fig. 3 (Section 5): TFT product time against
    the power-of-two zero-padded NTT product (Eq. 12, padded to the next
    power of two >= n) over lengths n in [2^lo, 2^hi] in fine steps; the NTT
    is a staircase, the TFT follows n.  Equal operand lengths, n = 2z - 1."""
    import torch
    p = W.P1
    zmax = (1 << hi) // 2 + 1
    a = dev_u32(W.coeffs(W.SEED_BASE + 60, zmax, p), dev)
    b = dev_u32(W.coeffs(W.SEED_BASE + 61, zmax, p), dev)
    c = torch.empty(2 * zmax, dtype=torch.int32, device=dev)
    sh = stream.cuda_stream
    rows = []
    with torch.cuda.stream(stream):
        for e in range(lo * per_octave, hi * per_octave + 1):
            n = int(round(2.0 ** (e / per_octave)))
            z = (n + 1) // 2
            n = 2 * z - 1
            Lp = 1 << (n - 1).bit_length()
            res = {"n": n, "L": Lp}
            for name, pad in (("tft_us", None), ("padded_us", Lp)):
                def f(i, pad=pad):
                    if pad:
                        B.polymul_mod_padded_async(p, a, z - 1, b, z - 1, c, pad, sh)
                    else:
                        B.polymul_mod_async(p, a, z - 1, b, z - 1, c, sh)
                for i in range(3):
                    f(i)
                res[name] = ev_time(f, reps, stream) * 1e3
            res["speedup"] = res["padded_us"] / res["tft_us"]
            rows.append(res)
    return {"p": p, "points": rows,
            "note": "inputs L2-resident (one buffer set); padded = every butterfly of the power-of-two NTT"}


def sweep(dev, stream, B, peaks, reps=20):
    import torch
    rows = []
    hbm = peaks.get("hbm_gbs", 6800.0)
    for z in W.LARGE_SIZES:
        p, a, b = W.workload3(z)
        n = 2 * z - 1
        sets = max(2, min(16, int(2 * L2_BYTES / (16 * z)) + 1))
        A = [dev_u32(a, dev) for _ in range(sets)]
        Bv = [dev_u32(b, dev) for _ in range(sets)]
        C = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(sets)]
        sh = stream.cuda_stream

        def f(i):
            j = i % sets
            B.polymul_mod_async(p, A[j], z - 1, Bv[j], z - 1, C[j], sh)
        with torch.cuda.stream(stream):
            for i in range(3):
                f(i)
            ms = ev_time(f, reps, stream)
        byt = 4 * (2 * z + n)
        L = 1 << (n - 1).bit_length()
        rows.append({"z": z, "n": n, "L": L, "n_over_L": round(n / L, 3), "us": ms * 1e3,
                     "coeffs_per_s": n / (ms * 1e-3), "hbm_compulsory_gbs": byt / (ms * 1e-3) / 1e9,
                     "hbm_compulsory_frac": byt / (ms * 1e-3) / 1e9 / hbm})
        del A, Bv, C
        torch.cuda.empty_cache()
    return rows


def exact_coeff(a, b, k):
    """c_k = sum a_i b_{k-i} over the integers (uint64 halves summed apart)."""
    lo = max(0, k - (len(b) - 1))
    hi = min(k, len(a) - 1)
    pr = a[lo:hi + 1].astype(np.uint64) * b[k - hi:k - lo + 1][::-1].astype(np.uint64)
    return (int(np.sum(pr >> np.uint64(32), dtype=np.uint64)) << 32) + int(np.sum(pr & np.uint64(0xFFFFFFFF),
                                                                                   dtype=np.uint64))


def crt3(dev, stream, B, mod_us, reps=20):
    """Exact integer products (three primes + CRT) of two operands of z
    uniform 32-bit words, against three modular products of the same size."""
    import torch
    rows = []
    for z in (1 << 16, 1 << 20, 3000001):
        a, b = W.workload6(z)
        n = 2 * z - 1
        sets = max(2, min(8, int(2 * L2_BYTES / (28 * z)) + 1))
        A = [dev_u32(a, dev) for _ in range(sets)]
        Bv = [dev_u32(b, dev) for _ in range(sets)]
        C = [torch.empty((n, 3), dtype=torch.int32, device=dev) for _ in range(sets)]
        sh = stream.cuda_stream

        def f(i):
            j = i % sets
            B.polymul_crt3_async(A[j], z - 1, Bv[j], z - 1, C[j], sh)
        with torch.cuda.stream(stream):
            for i in range(3):
                f(i)
            ms = ev_time(f, reps, stream)
        got = C[(reps - 1) % sets].cpu().numpy().view(np.uint32)
        ks = [0, n // 2, n - 1] + [int(k) for k in np.random.default_rng(z).integers(0, n, 13)]
        ok = all(int(got[k, 0]) + (int(got[k, 1]) << 32) + (int(got[k, 2]) << 64) == exact_coeff(a, b, k)
                 for k in ks)
        byt = 4 * 2 * z + 12 * n
        row = {"z": z, "n": n, "us": ms * 1e3, "coeffs_per_s": n / (ms * 1e-3),
               "hbm_compulsory_gbs": byt / (ms * 1e-3) / 1e9, "correct_sampled": ok}
        if z in mod_us:
            row["vs_three_mod_products"] = 3 * mod_us[z] / (ms * 1e3)
        rows.append(row)
        del A, Bv, C
        torch.cuda.empty_cache()
    return rows


def radix_sweep(dev, stream, B, reps=20):
    """General-radix products (transform length m 2^k, odd m) against the
    power-of-two TFT product (m = 1) mod 2013265921 (p - 1 = 15 2^27) at
    lengths between 2^20 and 2^21."""
    import torch
    p = W.P2
    rows = []
    for frac in (1.05, 1.3, 1.6, 1.9):
        n = int(frac * (1 << 20)) | 1
        z = (n + 1) // 2
        a, b = W.operands(W.SEED_BASE + 8, z - 1, z - 1, p)
        sets = 4
        A = [dev_u32(a, dev) for _ in range(sets)]
        Bv = [dev_u32(b, dev) for _ in range(sets)]
        C = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(sets)]
        sh = stream.cuda_stream
        row = {"n": n}
        ref = None
        for m in (1, 3, 5, 15):
            def f(i, m=m):
                j = i % sets
                B.polymul_mod_radix_async(p, A[j], z - 1, Bv[j], z - 1, C[j], m, sh)
            with torch.cuda.stream(stream):
                for i in range(3):
                    f(i)
                ms = ev_time(f, reps, stream)
            out = C[(reps - 1) % sets].cpu().numpy()
            if ref is None:
                ref = out
            row[f"m{m}_us"] = ms * 1e3
            row[f"m{m}_identical_to_m1"] = bool(np.array_equal(out, ref))
        rows.append(row)
        del A, Bv, C
        torch.cuda.empty_cache()
    return rows


def batched(dev, stream, B, reps=5):
    import torch
    p, a, a_off, b, b_off, c_off = W.workload4()
    count = len(a_off) - 1
    da, db = dev_u32(a, dev), dev_u32(b, dev)
    dc = torch.empty(int(c_off[-1]), dtype=torch.int32, device=dev)
    dc2 = torch.empty_like(dc)
    sh = stream.cuda_stream
    t0 = time.perf_counter()
    h = B.polymul_batch_create(p, a_off, b_off, c_off)
    t_plan = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        B.polymul_batch_exec(h, da, db, dc, sh)  # captures and instantiates the graph
        stream.synchronize()
        assert B.polymul_batch_status(h) == 0
        ms_graph = ev_time(lambda i: B.polymul_batch_exec(h, da, db, dc, sh), reps, stream)
        ms_nograph = ev_time(lambda i: B.polymul_batch_exec_nograph(h, da, db, dc, sh), reps, stream)
        B.polymul_mod_batched_plain(p, da, a_off, db, b_off, dc2, c_off, sh)
        stream.synchronize()
        ms_plain = ev_time(lambda i: B.polymul_mod_batched_plain(p, da, a_off, db, b_off, dc2, c_off, sh), reps,
                           stream)
        stream.synchronize()
    st = B.polymul_batch_status(h)
    same = bool(torch.equal(dc, dc2))
    B.polymul_batch_destroy(h)
    n_total = int(c_off[-1])
    byt = 4 * (len(a) + len(b) + n_total)
    return {"workload": "4096 products mod 2013265921, degrees log-uniform in [64, 65536]",
            "products": count, "coeffs_out": n_total, "graph_ms": ms_graph, "nograph_ms": ms_nograph,
            "plain_ms": ms_plain, "speedup_vs_plain": ms_plain / ms_graph,
            "coeffs_per_s": n_total / (ms_graph * 1e-3), "hbm_compulsory_gbs": byt / (ms_graph * 1e-3) / 1e9,
            "plan_create_ms": t_plan * 1e3, "status": st, "identical_to_plain": same,
            "plain": "one polymul_mod_async per product (its own 1 or 3 kernel launches)"}


def serve_run(dev, B, mode, t_arr, prime, da_, db_, pools, budget, check_every=997):
    """One request stream through a server in `mode`; latency = submit -> GPU completion."""
    import torch
    pool_words = 1 << 21
    arena_words = 1 << 28  # 1 GiB output ring (outputs of unchecked requests may be overwritten)
    arena = torch.empty(arena_words, dtype=torch.int32, device=dev)
    rng = np.random.default_rng(5)
    srv = B.polymul_server_create(budget, 4, mode)
    checks = []
    head = 0
    # every request's addresses are computed before the clock starts, so the
    # submit loop costs one library call per request
    reqs = []
    for i in range(len(t_arr)):
        q = int(prime[i])
        za, zb = int(da_[i]) + 1, int(db_[i]) + 1
        n = za + zb - 1
        offa, offb = int(rng.integers(0, pool_words)), int(rng.integers(0, pool_words))
        if i % check_every == 0:
            pc = torch.empty(n, dtype=torch.int32, device=dev)
            checks.append((q, offa, za, offb, zb, pc))
            c_ptr = pc.data_ptr()
        else:
            if head + n > arena_words:
                head = 0
            c_ptr = arena.data_ptr() + 4 * head
            head += n
        reqs.append((float(t_arr[i]), q, pools[q].data_ptr() + 4 * offa, za - 1, pools[q].data_ptr() + 4 * offb,
                     zb - 1, c_ptr))
    submit = B.polymul_server_submit
    tickets = []
    t0 = time.perf_counter()
    for ta, q, pa, da, pb, db, pc in reqs:
        while time.perf_counter() - t0 < ta:
            pass
        tickets.append(submit(srv, q, pa, da, pb, db, pc))
    t_sub = time.perf_counter() - t0
    for t in tickets:
        B.polymul_server_wait(srv, t, 120000)
    t_all = time.perf_counter() - t0
    stats = B.polymul_server_stats(srv)
    # per size class: small requests (L <= 2^17, the ones the serving form
    # batches and runs on its high-priority lane) and large ones
    lat = np.array([B.polymul_server_latency(srv, t) for t in tickets])
    n_req = da_[:len(tickets)].astype(np.int64) + db_[:len(tickets)].astype(np.int64) + 1
    small = np.ceil(np.log2(n_req)) <= 17
    classes = {}
    for name, mask in (("small_L_le_2^17", small), ("large", ~small)):
        v = lat[mask]
        if len(v):
            classes[name] = {"requests": int(len(v)), "p50_us": float(np.percentile(v, 50)),
                             "p99_us": float(np.percentile(v, 99)), "max_us": float(v.max())}
    stats["classes"] = classes
    B.polymul_server_destroy(srv)
    del arena
    return stats, t_sub, t_all, checks


def serving(dev, B, seconds, rate=20000.0, budget=8 << 30, burst=20000):
    """Workload 5 through the server (one batched launch per admitted group,
    POLY_SERVE_BATCH), beside the same stream served one plain product per
    request (POLY_SERVE_PLAIN); then a saturation burst (all requests
    submitted at once) for each mode."""
    import oracle
    t_arr, prime, da_, db_ = W.request_stream(rate=rate, seconds=seconds)
    pool_words = 1 << 21
    pools = {q: dev_u32(W.coeffs(W.SEED_BASE + 50 + i, pool_words + (1 << 20) + 2, q), dev)
             for i, q in enumerate((W.P1, W.P2))}
    pool_host = {q: host_u32(pools[q]) for q in pools}
    n_total = int((da_ + db_ + 1).sum())
    out = {"workload": f"Poisson {rate:.0f} req/s for {seconds} s, p in {{469762049, 2013265921}}, "
                       "degrees log-uniform in [256, 2^20], 8 GB admission budget, 4 streams",
           "requests": len(t_arr)}
    ok = True
    nchk = 0
    # warm-up (untimed): a burst of 2000 requests through each mode loads
    # every kernel variant the stream meets
    w = min(2000, len(t_arr))
    for mode in (B.SERVE_BATCH, B.SERVE_PLAIN):
        serve_run(dev, B, mode, np.zeros(w), prime[:w], da_[:w], db_[:w], pools, budget, check_every=10 ** 9)
    for name, mode in (("batch", B.SERVE_BATCH), ("plain", B.SERVE_PLAIN)):
        stats, t_sub, t_all, checks = serve_run(dev, B, mode, t_arr, prime, da_, db_, pools, budget)
        out[name] = {"p50_us": stats["p50_us"], "p90_us": stats["p90_us"], "p99_us": stats["p99_us"],
                     "max_us": stats["max_us"], "mean_us": stats["mean_us"], "submit_s": t_sub, "drain_s": t_all,
                     "throughput_req_per_s": len(t_arr) / t_all, "coeffs_per_s": n_total / t_all,
                     "classes": stats["classes"]}
        for q, offa, za, offb, zb, pc in checks[:3]:
            want = oracle.polymul_tft(q, pool_host[q][offa:offa + za], pool_host[q][offb:offb + zb])
            ok = ok and bool(np.array_equal(host_u32(pc), want))
            nchk += 1
    # three times the configured rate for a few seconds (between the light
    # configured load and saturation)
    t3, prime3, da3, db3 = W.request_stream(rate=3 * rate, seconds=min(5.0, seconds), seed=W.SEED_BASE + 15)
    load3 = {}
    for name, mode in (("batch", B.SERVE_BATCH), ("plain", B.SERVE_PLAIN)):
        stats, t_sub, t_all, _ = serve_run(dev, B, mode, t3, prime3, da3, db3, pools, budget, check_every=10 ** 9)
        load3[name] = {"p50_us": stats["p50_us"], "p99_us": stats["p99_us"], "max_us": stats["max_us"],
                       "throughput_req_per_s": len(t3) / t_all, "classes": stats["classes"]}
    out["load_3x"] = dict(rate_req_per_s=3 * rate, seconds=min(5.0, seconds), requests=len(t3), **load3)
    out["load_3x"]["p99_vs_plain"] = load3["plain"]["p99_us"] / load3["batch"]["p99_us"]
    # saturation: the first `burst` requests of the stream submitted back to back
    m = min(burst, len(t_arr))
    zeros = np.zeros(m)
    sat = {}
    for name, mode in (("batch", B.SERVE_BATCH), ("plain", B.SERVE_PLAIN)):
        stats, t_sub, t_all, _ = serve_run(dev, B, mode, zeros, prime[:m], da_[:m], db_[:m], pools, budget,
                                           check_every=10 ** 9)
        sat[name] = {"req_per_s": m / t_all, "coeffs_per_s": int((da_[:m] + db_[:m] + 1).sum()) / t_all,
                     "p50_us": stats["p50_us"], "p99_us": stats["p99_us"]}
    out["saturation"] = dict(requests=m, **sat)
    out["p50_us"] = out["batch"]["p50_us"]
    out["p99_us"] = out["batch"]["p99_us"]
    out["p50_vs_plain"] = out["plain"]["p50_us"] / out["batch"]["p50_us"]
    out["p99_vs_plain"] = out["plain"]["p99_us"] / out["batch"]["p99_us"]
    out["saturation_vs_plain"] = sat["batch"]["req_per_s"] / sat["plain"]["req_per_s"]
    out["checked_against_oracle"] = nchk
    out["checks_ok"] = ok
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--soak", type=float, default=1.5, help="seconds of untimed load before the timed region")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--schedule", action="append", default=[], metavar="L:SIGMA:C",
                    help="use rows of 2^SIGMA words and column tiles of C words for transform length 2^L "
                         "(repeatable; default: the library's tuned table)")
    ap.add_argument("--skip", default="",
                    help="comma list of parts to skip: e2e,cpu,padded,sweep,crt3,fig3,radix,batched,serving")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1609_01010_gb300 import binding as B
    B.lib()
    skip = set(x for x in args.skip.split(",") if x)
    if args.schedule:
        import tempfile
        rows = []
        for spec in args.schedule:
            l_, sg_, c_ = (int(x) for x in spec.split(":"))
            rows.append({"l": l_, "sigma": sg_, "C": c_, "us": 0.0})
        with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as f:
            json.dump({"device": "bench --schedule", "p": 0, "schedules": rows}, f)
        B.polymul_load_schedules(f.name)
        os.unlink(f.name)
    peaks, peak_src = load_peaks()
    stream = torch.cuda.Stream(device=dev)

    int_peaks = {}
    for kind, name in B.PROBE_KINDS.items():
        ops, pms = B.polymul_probe_int(kind, 1 << 15)
        int_peaks[name] = {"per_s": ops, "ms": pms}
    with ClockSampler(local) as clk:
        p, z, n, ms, got, a, b, step, ptrs = headline(args, dev, stream, B, world)
        prof_ms, prof_cnt = profiled_pass(args, stream, step)
        dist = step_distribution(stream, B, p, z, ptrs)
    ms = max_over_ranks(ms, world, dev)
    ks = [0, 1, n // 3, n // 2, n - 1] + list(np.random.default_rng(1).integers(0, n, 27))
    correct = sampled_ok(got, a, b, p, [int(k) for k in ks])

    value = job_value(n, ms, world)
    # roofline of the dominant kernel: the row stage (k_row_fused)
    sch_sigma, _ = B.polymul_get_schedule(21)
    S = 1 << sch_sigma
    k_rows = -(-n // S)
    bfly_per_launch = 3 * (S // 2) * sch_sigma * k_rows
    ops_per_bfly = 7  # lazy regime (p < 2^30): 3 IMAD + 4 integer ALU per butterfly
    pw_ops = 11       # pointwise: 4 IMAD (REDC) + 3 IMAD (Shoup) + 4 ALU
    ops_per_launch = bfly_per_launch * ops_per_bfly + k_rows * S * pw_ops
    row_ms = prof_ms[2] / max(1, prof_cnt[2])
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    issue_tops = sm_count * 4 * 32 * sm_mhz * 1e6 / 1e12
    # measured peak: the butterfly probe (the kernels' own butterfly, register
    # only, full occupancy) in butterflies/s, times the 7 ops a butterfly counts
    peak_tops = int_peaks["forward butterfly"]["per_s"] * ops_per_bfly / 1e12
    achieved = ops_per_launch / (row_ms * 1e-3) / 1e12 if row_ms > 0 else None
    total_prof = sum(prof_ms[1:4])
    roofline = {"bound": "alu", "kernel": "k_row_fused (row stage: forward x2, pointwise, inverse)",
                "achieved": achieved, "peak": peak_tops, "unit": "Tintop/s",
                "frac": (achieved / peak_tops) if achieved else None,
                "traffic": row_kernel_traffic()[0],
                "traffic_cold_l2": row_kernel_traffic()[1],
                "traffic_note": "ncu DRAM bytes per launch: traffic with L2 as the stream of products leaves it "
                                "(--cache-control none), traffic_cold_l2 after ncu's L2 flush; the row data are "
                                "16.8 MB read + 8.4 MB written per launch",
                "peak_source": "measured on this GPU by polymul_probe_int kind 0 (the lazy forward butterfly of "
                               "the transform kernels, 16 independent register chains per thread, full occupancy): "
                               f"{int_peaks['forward butterfly']['per_s'] / 1e12:.3f} T butterflies/s x 7 ops",
                "issue_ceiling": {"value": issue_tops, "unit": "Tintop/s",
                                  "derivation": f"{sm_count} SMs x 4 SMSP x 32 lanes x {sm_mhz:.0f} MHz (one "
                                                "warp-instruction issue per SMSP per clock)"},
                "int_peaks": int_peaks,
                "algorithmic_ops_per_launch": ops_per_launch,
                "row_stage_us_per_launch": row_ms * 1e3,
                "kernel_share_of_step": {"col_tft": prof_ms[1] / total_prof if total_prof else None,
                                         "rows": prof_ms[2] / total_prof if total_prof else None,
                                         "col_itft": prof_ms[3] / total_prof if total_prof else None},
                "kernel_us_per_step": {"col_tft": prof_ms[1] / max(1, prof_cnt[1]) * 1e3,
                                       "rows": row_ms * 1e3,
                                       "col_itft": prof_ms[3] / max(1, prof_cnt[3]) * 1e3}}
    # The whole product against the same peak: the column stages' butterflies
    # (TFT: t - 1 levels of both operands, the top one a copy since the upper
    # half of each operand is zero; ITFT: t levels of the product) plus the
    # row stage's operations, over the step time.
    t_col = 21 - sch_sigma
    col_bfly = 2 * (1 << 20) * (t_col - 1) + (1 << 20) * t_col
    prod_ops = col_bfly * ops_per_bfly + ops_per_launch
    roofline["product"] = {"algorithmic_ops": prod_ops, "achieved": prod_ops / (ms * 1e-3) / 1e12,
                           "frac": prod_ops / (ms * 1e-3) / 1e12 / peak_tops,
                           "note": "all three kernels' butterflies (7 ops) and pointwise products (11 ops) "
                                   "per step time, against the same measured peak"}
    hbm = peaks.get("hbm_gbs", 6800.0)
    comp_bytes = 4 * (2 * z + n)
    line = {"metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"tft_polymul_p{p}_z{z}", "p": p, "z1": z, "z2": z, "n": n, "L": 1 << 21,
                       "l2": "16 rotating input/output sets (268 MB > 129 MB L2)", "replicas": world,
                       "parallelism": "replicas" if world > 1 else "single"},
            "correct_sampled": correct,
            "hbm_compulsory": {"bytes_per_step": comp_bytes, "gbs": comp_bytes / (ms * 1e-3) / 1e9,
                               "peak_gbs": hbm, "frac": comp_bytes / (ms * 1e-3) / 1e9 / hbm,
                               "peak_source": peak_src},
            "roofline": roofline, "gpu_launches": 3 * args.steps, "step_distribution": dist,
            "clocks": clk.summary()}
    if rank == 0:
        if "e2e" not in skip:
            line["e2e"] = e2e_pass(args, p, a, b)
        if "padded" not in skip:
            line["small_configs"] = small_configs(dev, stream, B)
        if "sweep" not in skip:
            line["sweep"] = sweep(dev, stream, B, peaks)
        if "crt3" not in skip:
            mod_us = {r["z"]: r["us"] for r in line.get("sweep", [])}
            line["crt3"] = crt3(dev, stream, B, mod_us)
        if "fig3" not in skip:
            line["length_sweep"] = length_sweep(dev, stream, B)
        if "radix" not in skip:
            line["radix"] = radix_sweep(dev, stream, B)
        if "batched" not in skip:
            line["batched"] = batched(dev, stream, B)
        if "serving" not in skip and args.serve_seconds > 0:
            line["serving"] = serving(dev, B, args.serve_seconds)
        if "cpu" not in skip:
            line["cpu_baseline"] = cpu_oracle_rate()
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
