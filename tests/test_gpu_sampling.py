"""Keyframe sampling on the device (splat_set_view_sampling) against the oracle's draws, and its
effect on the render and the refinement loss.  Marked gpu."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import make_ctx, to_dev

pytestmark = pytest.mark.gpu

SEED = 0x1234_5678_9ABC_DEF0


@pytest.fixture(scope="module")
def scene():
    return scenes.workload(3, n=20_000)


def test_drawn_views_match_the_oracle(scene):
    """Twelve consecutive renders draw, view for view, what the oracle draws for calls 0..11."""
    views = scene.views[:8]
    ctx = make_ctx(scene.n, views)
    ctx.set_view_sampling(3, 0.4, SEED)
    dev = to_dev(scene)
    for s in range(12):
        ctx.render(*dev)
        got = ctx.active_views()
        ref = oracle.sample_active_views(len(views), 3, 0.4, SEED, s)
        np.testing.assert_array_equal(got, ref, err_msg=f"call {s}")
    ctx.set_view_sampling(0)
    ctx.render(*dev)
    assert ctx.active_views().all()


def test_sampled_render_keeps_the_drawn_views(scene):
    """Drawn views render bit-identically to a render of every view; the others are empty."""
    views = scene.views[:6]
    dev = to_dev(scene)
    full = make_ctx(scene.n, views)
    d0, n0, a0 = (t.cpu().numpy() for t in full.render(*dev))
    ctx = make_ctx(scene.n, views)
    ctx.set_view_sampling(2, 0.4, SEED + 1)
    seen = np.zeros(len(views), bool)
    for _ in range(4):
        d, n, a = (t.cpu().numpy() for t in ctx.render(*dev))
        act = ctx.active_views()
        seen |= act
        for k, v in enumerate(views):
            sl = slice(ctx.offsets[k], ctx.offsets[k] + v.n_pixels)
            if act[k]:
                np.testing.assert_array_equal(d[sl], d0[sl])
                np.testing.assert_array_equal(a[sl], a0[sl])
                np.testing.assert_array_equal(n[:, sl], n0[:, sl])
            else:
                assert not a[sl].any() and not d[sl].any()
    assert seen.sum() >= 2


def test_refinement_loss_counts_the_drawn_views_only(scene):
    """With sampling, splat_refine_step's loss is the loss of the drawn views' pixels alone."""
    views = scene.views[:5]
    dev = [t.clone() for t in to_dev(scene)]
    targets = [scenes.render_targets(scene, v) for v in views]
    t_depth = torch.from_numpy(np.concatenate([t[0].ravel() for t in targets])).cuda()
    t_normal = torch.from_numpy(np.concatenate([t[1].reshape(3, -1) for t in targets], 1)).cuda()
    full = make_ctx(scene.n, views)
    d0, n0, a0 = full.render(*[t.clone() for t in dev])
    ctx = make_ctx(scene.n, views)
    ctx.set_view_sampling(2, 0.4, SEED + 2)
    state = api.adam_state(scene.n, dev[0].device)
    loss_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.refine_step(dev, state, t_depth, t_normal.contiguous(), api.LossConfig(), api.AdamConfig(),
                    loss_out)
    act = ctx.active_views()
    assert 1 <= act.sum() < len(views)
    mask = torch.zeros_like(t_depth)
    for k, v in enumerate(views):
        if act[k]:
            mask[ctx.offsets[k]:ctx.offsets[k] + v.n_pixels] = 1
    L, *_ = api.loss(d0, n0, a0, (t_depth * mask).contiguous(), t_normal.contiguous())
    ref = float(L.item())
    got = float(loss_out.item())
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
