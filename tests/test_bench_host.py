"""Host-side logic of bench.py's multi-GPU form (replicas) on CPU: two gloo
ranks agree on the max-over-ranks step time and the whole-job value, and the
reference arm prints only on rank 0.  No GPU is touched."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [0.25, 0.40][rank]
        ms = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        bench.barrier(world)
        q.put((rank, ms, bench.job_value(1000, ms, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_and_sum():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0.40, 0.40]
    # value = units of all ranks / the slowest rank's time
    assert out[0][2] == pytest.approx(2 * 1000 / 0.40e-3)


def test_reference_arm_other_ranks_exit_quietly(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_job_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(2097151, 0.05, 1) == pytest.approx(2097151 / 0.05e-3)
    line = json.dumps({"value": bench.job_value(10, 1.0, 4)})
    assert json.loads(line)["value"] == pytest.approx(40 / 1e-3)
