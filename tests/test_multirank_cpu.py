"""The multi-GPU path on the CPU: world size 2 over gloo (no GPU).

The sweep shards into independent replicas (no exchange step): under torchrun each
rank runs its own copy and the benchmark reports every rank's units over the
slowest rank's time, printed by rank 0 alone; the reference arm runs on rank 0 only
and the other ranks exit without work.  These tests run the benchmark's own
reduction over two gloo ranks and the reference arm with a rank-1 environment.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [1200.0, 1850.0][rank]  # rank 1 is the slow replica
        t = bench.max_over_ranks(ms, world, torch.device("cpu"))
        rate = bench.job_rate(world, 50000 * 3, t / 1000.0)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 1850.0  # every rank sees the slowest time
        assert abs(rate - 2 * 50000 * 3 / 1.85) < 1e-6  # both ranks' units over it


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_rate(1, 100, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only():
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1", "--steps", "1",
            "--warmup", "0", "--gpus", "2"]
    env1 = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r1 = subprocess.run(base, env=env1, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    env0 = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r0 = subprocess.run(base, env=env0, capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0
    lines = [x for x in r0.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
