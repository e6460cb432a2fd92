"""The multi-rank plumbing of bench.py (replicas: barrier, max and sum over ranks, rank-0-only
output) with two gloo ranks on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init("gloo")
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 10.0 + rank)
    sm = bench.sum_over_ranks(dist, 1.0 + rank)
    info = bench.dist_info()
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((rank, mx, sm, info))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, mx, sm, info in res:
        assert mx == 11.0 and sm == 3.0
        assert info == (rank, 2, rank)


def test_single_rank_without_torchrun():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    old = os.environ.copy()
    os.environ.clear()
    os.environ.update(env)
    try:
        assert bench.dist_init("gloo") is None
        assert bench.max_over_ranks(None, 3.5) == 3.5
        assert bench.dist_info() == (0, 1, 0)
    finally:
        os.environ.clear()
        os.environ.update(old)


def test_reference_arm_line_on_cpu():
    """--impl reference runs the FP64 oracle on a tiny workload and prints the contract line."""
    pytest.importorskip("numpy")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "0", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "px/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
