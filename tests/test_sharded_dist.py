"""The data-parallel refinement over keyframes (paper_2503_17491_gb300.sharded) with two gloo
ranks on CPU: the keyframe split covers every keyframe once, and after a few steps both replicas
hold the same parameters as one process refining over all keyframes.  The per-rank work is a
CPU stand-in (the quadratic loss sum_v 0.5 |p - c_v|^2 per keyframe v and plain Adam), since the
kernels need a GPU; the exchange and the update order are what is under test."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _View:
    def __init__(self, rows, cols, k):
        self.rows, self.cols, self.k = rows, cols, k


class _CpuOps:
    def __init__(self, n, views, targets):
        self.views = views
        self.m = None

    def grads(self, params):
        g = [torch.zeros_like(p) for p in params]
        loss = torch.zeros(1, dtype=torch.float64)
        for v in self.views:
            for j, p in enumerate(params):
                c = float(v.k + 1) * (j + 1)
                g[j] += (p - c)
                loss += 0.5 * ((p - c) ** 2).sum()
        return g, loss

    def adam(self, params, grads):
        if self.m is None:
            self.m = [torch.zeros_like(p) for p in params]
            self.v = [torch.zeros_like(p) for p in params]
            self.t = 0
        self.t += 1
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m.mul_(0.9).add_(0.1 * g)
            v.mul_(0.999).add_(0.001 * g * g)
            p.sub_(0.05 * (m / (1 - 0.9 ** self.t)) / ((v / (1 - 0.999 ** self.t)).sqrt() + 1e-12))


def _views():
    sizes = [(64, 1024), (128, 1024), (32, 1800), (64, 1024), (128, 1024), (32, 1800), (16, 64)]
    return [_View(r, c, k) for k, (r, c) in enumerate(sizes)]


def _run(steps):
    from paper_2503_17491_gb300 import sharded
    params = [torch.linspace(-1, 1, 12, dtype=torch.float64).reshape(3, 4).clone(),
              torch.zeros(3, 4, dtype=torch.float64), torch.ones(3, 2, dtype=torch.float64)]
    r = sharded.ShardedRefiner(params, _views(), [None] * 7,
                               ops_factory=lambda n, vs, ts: _CpuOps(n, vs, ts))
    losses = [float(r.step()) for _ in range(steps)]
    return [p.clone() for p in params], losses, r.split


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo")
    params, losses, split = _run(4)
    # the float32 exchange against the float64 sum of the same float32 values
    g = torch.from_numpy(np.random.default_rng(rank).normal(size=4096) *
                         10.0 ** np.random.default_rng(7 + rank).uniform(-6, 3, 4096)
                         ).to(torch.float32)
    mine = g.clone()
    dist.all_reduce(g, op=dist.ReduceOp.SUM)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    dist.destroy_process_group()
    q.put((rank, [p.numpy() for p in params], losses, split,
           (g.numpy(), [x.numpy() for x in parts])))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_exact_and_balanced():
    sys.path.insert(0, ROOT)
    from paper_2503_17491_gb300 import sharded
    sizes = [v.rows * v.cols for v in _views()]
    for world in (1, 2, 3, 8):
        split = sharded.partition_views(sizes, world)
        flat = sorted(i for part in split for i in part)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in part) for part in split]
        if world <= len(sizes):
            assert max(loads) - min(loads) <= max(sizes)


def test_two_gloo_ranks_match_one_process():
    """Both replicas end with identical parameters, equal to one process over all keyframes
    within the float32 exchange's rounding (the per-rank partial sums are rounded to float32
    before they are added); the float32 all-reduce is within (N - 1) 2^-24 sum_r |g_r| of the
    float64 sum of its inputs."""
    sys.path.insert(0, ROOT)
    ref_params, ref_losses, _ = _run(4)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    # read the results before joining: a child does not exit while its queued data is unread
    res = sorted((q.get(timeout=120) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    (_, pa, la, sa, xa), (_, pb, lb, sb, xb) = res
    assert sa == sb and sorted(sa[0] + sa[1]) == list(range(7)) and sa[0] and sa[1]
    for a, b, r in zip(pa, pb, ref_params):
        assert (a == b).all()                                  # replicas stay identical
        torch.testing.assert_close(torch.from_numpy(a), r, rtol=1e-5, atol=1e-6)
    assert la == lb
    assert la == pytest.approx(ref_losses, rel=1e-6)
    red, parts = xa
    assert (xb[0] == red).all()
    exact = sum(x.astype(np.float64) for x in parts)
    bound = (len(parts) - 1) * 2.0 ** -24 * sum(np.abs(x.astype(np.float64)) for x in parts)
    assert (np.abs(red.astype(np.float64) - exact) <= bound).all()
