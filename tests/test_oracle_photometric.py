"""Pins of the oracle's photometric registration residual (Sec. 3.3.3, Eq. L_photo) and its
Gauss-Newton normal equations."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_17491_gb300 import scenes


def se3_exp(xi):
    """exp of xi = (rho, omega) as a 4 x 4 matrix (Rodrigues plus the left Jacobian)."""
    rho, w = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(w)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-12:
        R, V = np.eye(3) + W, np.eye(3) + 0.5 * W
    else:
        R = np.eye(3) + math.sin(th) / th * W + (1 - math.cos(th)) / th ** 2 * W @ W
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * W + (th - math.sin(th)) / th ** 3 * W @ W
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, V @ rho
    return T


def _street(rows=32, cols=512):
    s = scenes.workload(3, n=1000)
    v = s.views[0]
    vm = scenes.View(v.T_ws, rows, cols, v.elev_min, v.elev_max)
    motion = se3_exp([0.6, -0.2, 0.05, 0.0, 0.01, 0.03])     # query sensor relative to the render
    vq = scenes.View(v.T_ws @ motion, rows, cols, v.elev_min, v.elev_max)
    D = scenes.render_targets(s, vm, noise=0.0)[0].ravel().astype(np.float64)
    Dq = scenes.render_targets(s, vq, noise=0.0)[0].ravel().astype(np.float64)
    O = (D > 0).astype(np.float64)
    T_true = np.linalg.inv(vq.T_ws) @ vm.T_ws                 # render frame -> query frame
    return vm, D, O, Dq, T_true


def test_identity_pose_on_its_own_image_gives_zero_residual():
    vm, D, O, Dq, T_true = _street()
    out = oracle.photometric_normal_eqs(D, O, D, np.eye(4), vm.rows, vm.cols, vm.elev_min,
                                        vm.elev_max, 0.5, 0.2)
    assert out["count"] > 0.5 * D.size
    assert np.abs(out["r"][out["used"]]).max() < 1e-9
    assert out["cost"] < 1e-15 and np.abs(out["g"]).max() < 1e-6


def test_jacobian_by_finite_differences_of_the_pose():
    vm, D, O, Dq, T_true = _street(rows=16, cols=256)
    T = T_true @ se3_exp([0.05, 0.02, -0.01, 0.004, -0.002, 0.003])
    base = oracle.photometric_normal_eqs(D, O, Dq, T, vm.rows, vm.cols, vm.elev_min, vm.elev_max,
                                         0.5, 1e9)
    h = 1e-6
    fd = np.zeros((D.size, 6))
    both = base["used"].copy()
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        a = oracle.photometric_normal_eqs(D, O, Dq, T @ se3_exp(e), vm.rows, vm.cols, vm.elev_min,
                                          vm.elev_max, 0.5, 1e9)
        b = oracle.photometric_normal_eqs(D, O, Dq, T @ se3_exp(-e), vm.rows, vm.cols,
                                          vm.elev_min, vm.elev_max, 0.5, 1e9)
        both &= a["used"] & b["used"]
        fd[:, k] = (a["r"] - b["r"]) / (2 * h)
    J = base["J"][both]
    err = np.abs(fd[both] - J).max(1) / (1.0 + np.abs(J).max(1))
    # a sample that crosses a bilinear cell edge between +h and -h has a one-sided slope
    assert np.mean(err < 1e-4) > 0.995, np.sort(err)[-10:]
    assert both.sum() > 1000


def test_huber_weights_and_cost():
    """One pixel, hand values: |r| beyond delta gets w = delta / |r| and the linear cost."""
    rows, cols = 4, 16
    D = np.zeros(rows * cols)
    O = np.zeros(rows * cols)
    D[1 * cols + 3], O[1 * cols + 3] = 10.0, 1.0
    Dq = np.full(rows * cols, 10.5)
    out = oracle.photometric_normal_eqs(D, O, Dq, np.eye(4), rows, cols, -0.2, 0.2, 0.5, 0.2)
    assert out["count"] == 1
    r = out["r"][1 * cols + 3]
    assert r == pytest.approx(-0.5, abs=1e-12)
    assert out["w"][1 * cols + 3] == pytest.approx(0.4)
    assert out["cost"] == pytest.approx(0.2 * (0.5 - 0.1))
    J = out["J"][1 * cols + 3]
    np.testing.assert_allclose(out["g"], 0.4 * J * r, rtol=1e-12)
    # flat query image: the sample has no slope, so J is the range's own derivative:
    # d|p'|/d rho = p / |p| (rotation part zero: p x p = 0)
    np.testing.assert_allclose(J[3:], 0.0, atol=1e-12)
    v = oracle.pixel_rays(rows, cols, -0.2, 0.2).reshape(-1, 3)[1 * cols + 3]
    np.testing.assert_allclose(J[:3], v, atol=1e-12)


def test_gauss_newton_recovers_a_known_pose():
    """From a 0.15 m / 1 degree offset, Gauss-Newton steps on the normal equations bring the
    pose back towards the true one (ray-cast street, exact ranges)."""
    vm, D, O, Dq, T_true = _street()
    T = T_true @ se3_exp([0.12, -0.08, 0.03, 0.0, 0.0, math.radians(1.0)])

    def err(T):
        E = np.linalg.inv(T_true) @ T
        ang = math.acos(max(-1.0, min(1.0, (np.trace(E[:3, :3]) - 1) / 2)))
        return np.linalg.norm(E[:3, 3]), ang

    e0 = err(T)
    for _ in range(8):
        out = oracle.photometric_normal_eqs(D, O, Dq, T, vm.rows, vm.cols, vm.elev_min,
                                            vm.elev_max, 0.5, 0.3)
        dx = -np.linalg.solve(out["H"] + 1e-9 * np.eye(6), out["g"])
        T = T @ se3_exp(dx)
    e1 = err(T)
    assert e1[0] < 0.2 * e0[0] and e1[1] < 0.2 * e0[1], (e0, e1)


def test_ambiguity_band_flags_cell_edges_and_steep_slopes():
    """The band flags exactly the used pixels whose u' lies within band_px of a cell edge (u'
    from the motion's closed form: a turn of 0.3 columns about z and a 0.2 m lift), plus, on a
    query image ramping across columns by s metres per column, every pixel when s band_px
    exceeds band_r and no extra pixel when it does not."""
    rows, cols, emin, emax = 24, 256, -0.3, 0.3
    dg, dth = 2 * math.pi / cols, (emax - emin) / (rows - 1)
    phi = 0.3 * dg
    T = se3_exp([0.0, 0.0, 0.2, 0.0, 0.0, phi])
    T[:3, 3] = [0.0, 0.0, 0.2]                 # a pure lift after the turn about z
    D = np.full(rows * cols, 10.0)
    O = np.ones(rows * cols)
    # u' of every pixel: p = 10 v(u), p' = Rz(phi) p + (0, 0, 0.2)
    r, c = np.divmod(np.arange(rows * cols), cols)
    gam = math.pi - (c + 0.5) * dg
    th = emax - r * dth
    x, y, z = 10 * np.cos(th) * np.cos(gam + phi), 10 * np.cos(th) * np.sin(gam + phi), 10 * np.sin(th) + 0.2
    cq = (math.pi - np.arctan2(y, x)) / dg - 0.5
    rq = (emax - np.arctan2(z, np.hypot(x, y))) / dth
    fr, fc = rq - np.floor(rq), cq - np.floor(cq)
    bp = 0.25
    near = (np.minimum(fr, 1 - fr) <= bp) | (np.minimum(fc, 1 - fc) <= bp)
    for s, steep in ((0.01, False), (1.0, True)):
        Dq = 10.0 + s * np.tile(np.arange(cols, dtype=float), rows)
        out = oracle.photometric_normal_eqs(D, O, Dq, T, rows, cols, emin, emax, 0.5, 1.0,
                                            band_px=bp, band_r=0.005)
        used = out["used"]
        assert used.sum() > 0.8 * rows * cols
        seam = (c == 0) | (c == cols - 1)      # the ramp wraps from 255 s back to 0 there
        m = ~seam & (np.floor(rq) >= 0) & (np.floor(rq) + 1 < rows)
        if steep:
            assert out["band"][m].all()
        else:
            np.testing.assert_array_equal(out["band"][m], near[m])
            assert 0 < near[m].sum() < m.sum()
