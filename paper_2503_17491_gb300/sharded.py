"""Data-parallel refinement over keyframes: every rank holds a replica of the map, renders and
differentiates its own share of the keyframes, and one all-reduce (sum) of the per-primitive
parameter gradients and the loss precedes an identical Adam step on every replica.

The exchange is the only collective of the path: the forward needs none, since each keyframe is
rendered whole by one rank.  Keyframes are shared out longest-first by pixel count (each to the
rank with the fewest pixels so far), so the split is deterministic and balanced.

The exchange is one float32 all-reduce of n x 10 gradient values plus the loss (the gradients'
own precision; 20 MB at 500,000 primitives).  `ShardedRefiner` takes its per-rank work from an `ops` object (`grads(params) -> (grads, loss)`,
`adam(params, grads)`); `GpuOps` runs the library's render, loss, backward and Adam calls on this
rank's keyframes.  The scale term of the loss is not supported here (it lives in the fused step).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import api


def partition_views(sizes, world: int) -> list[list[int]]:
    """Indices of the keyframes each rank renders: longest first, each to the least-loaded rank
    (ties to the lower rank); within a rank, in registration order."""
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(x) for x in out]


class GpuOps:
    """One rank's share: render, loss, backward over its keyframes; Adam on the whole map."""

    def __init__(self, n, views, targets, cfg=None, loss_cfg=None, adam_cfg=None,
                 max_pairs=None, device="cuda"):
        self.loss_cfg = loss_cfg or api.LossConfig()
        if self.loss_cfg.lambda_s != 0.0:
            raise ValueError("the scale term needs the fused refinement step")
        self.adam_cfg = adam_cfg or api.AdamConfig()
        self.n = n
        self.state = api.adam_state(n, device)
        self.ctx = None
        if views:
            P = sum(v.rows * v.cols for v in views)
            self.ctx = api.SplatContext(n, len(views), P, max_pairs, cfg)
            self.ctx.set_views(views)
            self.t_depth = torch.cat([t[0].reshape(-1) for t in targets]).contiguous()
            self.t_normal = torch.cat([t[1].reshape(3, -1) for t in targets], 1).contiguous()

    def grads(self, params):
        if self.ctx is None:
            return [torch.zeros_like(p) for p in params], torch.zeros(1, dtype=torch.float64,
                                                                      device=params[0].device)
        d, nrm, a = self.ctx.render(*params)
        L, gD, gN, gO = self.ctx.view_loss(d, nrm, a, self.t_depth, self.t_normal, self.loss_cfg)
        return list(self.ctx.backward(*params, gD, gN, gO)), L

    def adam(self, params, grads):
        api.adam_step(params, grads, self.state, self.adam_cfg)


class ShardedRefiner:
    """One refinement iteration of a shared map over keyframes split across the ranks of the
    default process group (a single process when none is initialised)."""

    def __init__(self, params, views, targets, ops_factory=None, group=None, **kw):
        self.params = params
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.split = partition_views([v.rows * v.cols for v in views], self.world)
        mine = self.split[self.rank]
        factory = ops_factory or (lambda n, vs, ts: GpuOps(n, vs, ts, **kw))
        self.ops = factory(params[0].shape[0], [views[i] for i in mine],
                           [targets[i] for i in mine])

    def step(self) -> torch.Tensor:
        """One iteration; returns the loss summed over all ranks' keyframes as a one-element
        float32 tensor on the parameters' device (no host synchronisation).  The gradients and
        the loss travel in one float32 buffer: with N ranks each element of the sum is rounded
        at most N - 1 times, |error| <= (N - 1) 2^-24 sum_r |g_r|."""
        grads, loss = self.ops.grads(self.params)
        flat = torch.cat([g.reshape(-1).to(torch.float32) for g in grads] +
                         [loss.reshape(-1).to(torch.float32)])
        if self.world > 1:
            dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=self.group)
        out, k = [], 0
        for g in grads:
            out.append(flat[k:k + g.numel()].view(g.shape).to(g.dtype))
            k += g.numel()
        self.ops.adam(self.params, out)
        return flat[k:k + 1]
