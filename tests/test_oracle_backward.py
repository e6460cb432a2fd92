"""Pins of the FP64 oracle's analytic gradient (Supp. D.2 plus the chain rule through the
quaternion, log-scale and opacity logit): central finite differences of the FP64 forward.

A component is skipped (redrawn) when the +-h renders differ in any contributor count, because
the image is then not differentiable there (a cutoff was crossed).
"""
import math

import numpy as np
import pytest

from paper_2503_17491_gb300 import scenes


def _loss(oracle_mod, params, flip, order, v, gD, gN, gO):
    out = oracle_mod.render(params, flip, order, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
    L = float((gD * out["D"]).sum() + (gN * out["N"]).sum() + (gO * out["O"]).sum())
    return L, out["n_contrib"]


def _fd_check(oracle_mod, scene, seed, min_checked=20):
    v = scene.views[0]
    proj = oracle_mod.project_contract(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws,
                                       v.rows, v.cols, v.elev_min, v.elev_max)
    flip, order = proj["flip"], oracle_mod.sort_order(proj["kappa"])
    base = [a.copy() for a in oracle_mod.split_params(scene.pos_logit, scene.quat,
                                                       scene.log_scale)]
    rng = np.random.default_rng(seed)
    gD = rng.normal(size=(v.rows, v.cols))
    gN = rng.normal(size=(3, v.rows, v.cols))
    gO = rng.normal(size=(v.rows, v.cols))
    an = oracle_mod.render_backward(base, flip, order, v.T_ws, v.rows, v.cols, v.elev_min,
                                    v.elev_max, gD, gN, gO)
    groups = [("g_pos", 0, 3), ("g_logit", 1, 1), ("g_quat", 2, 4), ("g_log_scale", 3, 2)]
    L0, nc0 = _loss(oracle_mod, base, flip, order, v, gD, gN, gO)
    checked = skipped = 0
    worst = 0.0
    for name, gi, width in groups:
        scale = np.abs(an[name]).max() + 1e-30
        for i in range(scene.n):
            for k in range(width):
                p = [a.copy() for a in base]
                arr = p[gi]
                idx = (i, k) if arr.ndim == 2 else (i,)
                x = arr[idx]
                h = 1e-6 * max(1.0, abs(x))
                arr[idx] = x + h
                Lp, ncp = _loss(oracle_mod, p, flip, order, v, gD, gN, gO)
                arr[idx] = x - h
                Lm, ncm = _loss(oracle_mod, p, flip, order, v, gD, gN, gO)
                if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                    skipped += 1
                    continue
                fd = (Lp - Lm) / (2 * h)
                a = an[name][idx]
                err = abs(fd - a) / max(abs(a), 1e-3 * scale)
                worst = max(worst, err)
                assert err < 2e-6, (name, i, k, fd, a)
                checked += 1
    assert checked >= min_checked, (checked, skipped)
    return worst, checked, skipped


@pytest.mark.parametrize("n,seed", [(1, 0), (3, 1), (8, 2), (20, 3)])
def test_fd_gradient_tiny_scenes(oracle_mod, n, seed):
    scene = scenes.tiny_scene(n, seed, rows=12, cols=48, fov_deg=20)
    v = scene.views[0]
    # keep clear of the alpha_max clamp (a kink) in this test: opacity <= 0.9
    scene.pos_logit[:, 3] = np.minimum(scene.pos_logit[:, 3], math.log(0.9 / 0.1))
    out = oracle_mod.full_view(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws, v.rows,
                               v.cols, v.elev_min, v.elev_max, mode="brute")
    assert out["O"].max() > 0.2, "scene should be visible"
    _fd_check(oracle_mod, scene, seed, min_checked=5 * n)


def test_fd_gradient_posed_overlapping(oracle_mod):
    """Overlapping splats, a general pose (rotation + translation), and the dL/dO channel."""
    scene = scenes.tiny_scene(12, 7, rows=10, cols=40, fov_deg=25, dist=(3.0, 4.0),
                              log_scale=(-1.2, -0.6))
    scene.pos_logit[:, 3] = np.minimum(scene.pos_logit[:, 3], math.log(0.9 / 0.1))
    scene.views[0].T_ws = scenes.random_pose(np.random.default_rng(9), 0.3, 10.0)
    v = scene.views[0]
    out = oracle_mod.full_view(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws, v.rows,
                               v.cols, v.elev_min, v.elev_max, mode="brute")
    assert (out["n_contrib"] >= 2).sum() > 5, "want overlapping contributors"
    _fd_check(oracle_mod, scene, 11, min_checked=60)


def test_clamped_alpha_has_no_opacity_gradient(oracle_mod):
    """Where alpha is clamped to alpha_max, alpha does not depend on o: with upstream gradients
    only on clamped pixels, dL/dlogit = 0 while the range still moves with the position."""
    from test_oracle_forward import one_splat
    pl, q, ls = one_splat(5.0, 0.99999, 3.0, 3.0)
    v = scenes.View(np.eye(4), 9, 360, scenes.deg(-2), scenes.deg(2))
    params = oracle_mod.split_params(pl, q, ls)
    proj = oracle_mod.project_contract(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
    out = oracle_mod.render(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                            v.elev_max)
    clamped = (out["O"] == 0.99).astype(np.float64)
    assert clamped.sum() > 5 and (out["O"] > 0).sum() > clamped.sum()
    g = oracle_mod.render_backward(params, proj["flip"], None, v.T_ws, v.rows, v.cols,
                                   v.elev_min, v.elev_max, clamped, np.zeros((3, 9, 360)),
                                   clamped)
    assert g["g_logit"][0] == 0.0
    assert np.abs(g["g_pos"]).max() > 0


def test_gradient_zero_outside_coverage(oracle_mod):
    """Upstream gradients on pixels the splat does not reach give a zero parameter gradient."""
    from test_oracle_forward import one_splat
    pl, q, ls = one_splat(5.0, 0.7, 0.2, 0.2)
    v = scenes.View(np.eye(4), 17, 128, scenes.deg(-10), scenes.deg(10))
    params = oracle_mod.split_params(pl, q, ls)
    out = oracle_mod.render(params, np.ones(1, np.int8), None, v.T_ws, v.rows, v.cols,
                            v.elev_min, v.elev_max)
    mask = (out["O"] == 0).astype(np.float64)
    g = oracle_mod.render_backward(params, np.ones(1, np.int8), None, v.T_ws, v.rows, v.cols,
                                   v.elev_min, v.elev_max, mask, np.stack([mask] * 3), mask)
    for k in ("g_pos", "g_logit", "g_quat", "g_log_scale"):
        assert np.abs(g[k]).max() == 0.0
