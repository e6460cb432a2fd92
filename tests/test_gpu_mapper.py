"""The local-model loop of Sec. 3.3 assembled from the library's calls (api.Mapper): keyframes
of a ray-cast street are added one by one, the map grows from each (valid mask first, then the
densification masks) and is refined with keyframe sampling.  Checks that the pieces compose: the
map grows by the drawn slots, refinement lowers the loss, and the rendered ranges approach the
scans.  Marked gpu."""
import numpy as np
import pytest
import torch

from paper_2503_17491_gb300 import api, scenes

pytestmark = pytest.mark.gpu


def _range_stats(mapper, k, target):
    d, n, a = mapper.render()
    torch.cuda.synchronize()
    v = mapper.ctx.views[k]
    o, P = mapper.ctx.offsets[k], v.rows * v.cols
    D, O = d[o:o + P].cpu().numpy(), a[o:o + P].cpu().numpy()
    Dt = target.ravel()
    valid = Dt > 0
    cov = valid & (O > 0.5)
    err = np.abs(D[cov] / O[cov] - Dt[cov])
    return float(cov.sum() / valid.sum()), float(np.median(err)) if err.size else np.inf


def test_mapper_grows_and_refines_a_street():
    s = scenes.workload(3, n=1000)
    views = s.views[:4]
    targets = [scenes.render_targets(s, v) for v in views]
    P = sum(v.rows * v.cols for v in views)
    n_new = 15_000
    mapper = api.Mapper(capacity=n_new * len(views), max_views=len(views), max_pixels=P,
                        n_new=n_new,
                        loss_cfg=api.LossConfig(lambda_n=0.1, lambda_o=0.1, normal_mode=1,
                                                lambda_s=0.01, tau_s=0.5),
                        densify_cfg=api.DensifyConfig(scale_k=2.0, opacity=0.6, seed=3),
                        draws=2, seed=5)
    report = []
    for k, (v, (dt, nt)) in enumerate(zip(views, targets)):
        mapper.add_keyframe(v, torch.from_numpy(dt).cuda(), torch.from_numpy(nt).cuda())
        assert mapper.n == (k + 1) * n_new
        cov0, err0 = _range_stats(mapper, k, dt)
        losses = mapper.refine(40)
        cov1, err1 = _range_stats(mapper, k, dt)
        report.append((k, cov0, err0, cov1, err1, losses[0], losses[-1]))
        assert mapper.ctx.status() == 0
        assert np.isfinite(losses).all()
        assert losses[-1] < losses[0]
        assert cov1 >= cov0 - 0.02 and err1 < err0
    print(report)
    # after all keyframes, every scan is mostly covered and its rendered ranges are close
    for k, (dt, _) in enumerate(targets):
        cov, err = _range_stats(mapper, k, dt)
        print("keyframe", k, "coverage", cov, "median range error", err)
        assert cov > 0.95 and err < 0.15


def test_mapper_keeps_a_window_of_recent_keyframes():
    """With max_keyframes, only the most recent keyframes stay registered: the map keeps growing
    with every keyframe while refinement runs over the window, and the window's scans end up
    covered by the map."""
    s = scenes.workload(3, n=1000)
    views = s.views[:6]
    targets = [scenes.render_targets(s, v) for v in views]
    window = 3
    P = max(sum(v.rows * v.cols for v in views[k:k + window]) for k in range(len(views)))
    n_new = 10_000
    mapper = api.Mapper(capacity=n_new * len(views), max_views=window, max_pixels=P,
                        n_new=n_new, max_keyframes=window,
                        loss_cfg=api.LossConfig(lambda_n=0.1, lambda_o=0.1, normal_mode=1,
                                                lambda_s=0.01, tau_s=0.5),
                        densify_cfg=api.DensifyConfig(scale_k=2.0, opacity=0.6, seed=3),
                        draws=2, seed=5)
    for k, (v, (dt, nt)) in enumerate(zip(views, targets)):
        mapper.add_keyframe(v, torch.from_numpy(dt).cuda(), torch.from_numpy(nt).cuda())
        assert mapper.n == (k + 1) * n_new
        assert len(mapper.views) == min(k + 1, window)
        assert mapper.views[-1] is v
        newest = len(mapper.views) - 1
        cov0, err0 = _range_stats(mapper, newest, dt)
        # each iteration's loss covers the keyframes drawn for it, so the losses of different
        # iterations are not compared; the newest keyframe's rendered ranges must improve
        losses = mapper.refine(30)
        cov1, err1 = _range_stats(mapper, newest, dt)
        assert mapper.ctx.status() == 0
        assert np.isfinite(losses).all()
        assert cov1 >= cov0 - 0.02 and err1 < err0
    for j, (dt, _) in enumerate(targets[-window:]):
        cov, err = _range_stats(mapper, j, dt)
        print("window keyframe", j, "coverage", cov, "median range error", err)
        assert cov > 0.9 and err < 0.2
