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


def _se3_hat(xi):
    rho, om = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0.0, -om[2], om[1]], [om[2], 0.0, -om[0]], [-om[1], om[0], 0.0]]
    X[:3, 3] = rho
    return X


@pytest.mark.parametrize("seed", [21, 22])
def test_fd_pose_gradient(oracle_mod, seed):
    """dL/dxi for the left perturbation T^c_w <- exp(xi^) T^c_w, xi = (rho, omega) in the sensor
    frame, against central differences of the FP64 forward rendered at the perturbed pose (the
    matrix exponential from scipy; same list order and normal signs)."""
    linalg = pytest.importorskip("scipy.linalg")
    scene = scenes.tiny_scene(14, seed, rows=10, cols=40, fov_deg=25, dist=(3.0, 6.0),
                              log_scale=(-1.2, -0.6))
    scene.pos_logit[:, 3] = np.minimum(scene.pos_logit[:, 3], math.log(0.9 / 0.1))
    scene.views[0].T_ws = scenes.random_pose(np.random.default_rng(seed), 0.3, 10.0)
    v = scene.views[0]
    proj = oracle_mod.project_contract(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws,
                                       v.rows, v.cols, v.elev_min, v.elev_max)
    flip, order = proj["flip"], oracle_mod.sort_order(proj["kappa"])
    params = oracle_mod.split_params(scene.pos_logit, scene.quat, scene.log_scale)
    rng = np.random.default_rng(seed + 100)
    gD = rng.normal(size=(v.rows, v.cols))
    gN = rng.normal(size=(3, v.rows, v.cols))
    gO = rng.normal(size=(v.rows, v.cols))
    an = oracle_mod.render_backward(params, flip, order, v.T_ws, v.rows, v.cols, v.elev_min,
                                    v.elev_max, gD, gN, gO)["g_pose"]
    T_cw = np.linalg.inv(v.T_ws)

    def loss_at(xi):
        T_ws = np.linalg.inv(linalg.expm(_se3_hat(xi)) @ T_cw)
        out = oracle_mod.render(params, flip, order, T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
        return float((gD * out["D"]).sum() + (gN * out["N"]).sum() + (gO * out["O"]).sum()), \
            out["n_contrib"]

    _, nc0 = loss_at(np.zeros(6))
    assert nc0.sum() > 20, "scene should be visible"
    scale = np.abs(an).max()
    checked = 0
    for k in range(6):
        h = 1e-6
        xi = np.zeros(6)
        xi[k] = h
        Lp, ncp = loss_at(xi)
        Lm, ncm = loss_at(-xi)
        if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
            continue
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - an[k]) <= 2e-6 * max(abs(an[k]), 1e-3 * scale), (k, fd, an[k])
        checked += 1
    assert checked >= 5


def test_pose_gradient_translation_part_is_centre_sum(oracle_mod):
    """A pure translation of the sensor moves every centre by rho and no axis or normal: dL/drho
    is the sum of the centres' sensor-frame gradients; the rotation part is not zero."""
    scene = scenes.tiny_scene(6, 3, rows=10, cols=40, fov_deg=25, dist=(3.0, 6.0))
    v = scene.views[0]
    proj = oracle_mod.project_contract(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws,
                                       v.rows, v.cols, v.elev_min, v.elev_max)
    params = oracle_mod.split_params(scene.pos_logit, scene.quat, scene.log_scale)
    rng = np.random.default_rng(5)
    g = oracle_mod.render_backward(params, proj["flip"], oracle_mod.sort_order(proj["kappa"]),
                                   v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max,
                                   rng.normal(size=(10, 40)), rng.normal(size=(3, 10, 40)),
                                   rng.normal(size=(10, 40)))
    np.testing.assert_allclose(g["g_pose"][:3], g["g_b"][:, 6:9].sum(0), rtol=1e-12, atol=1e-12)
    assert np.abs(g["g_pose"][3:]).max() > 0
