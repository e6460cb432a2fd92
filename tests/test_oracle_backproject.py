"""Pins of the oracle's back-projection of a rendered range image (Sec. 3.3: the rasterised
range image is back-projected to a point cloud at its pose)."""
import math

import numpy as np

from paper_2503_17491_gb300 import scenes
from test_oracle_forward import one_splat


def _render(oracle_mod, pl, q, ls, v):
    out = oracle_mod.full_view(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max,
                               mode="brute")
    return out["D"].astype(np.float32), out["O"].astype(np.float32)


def test_head_on_splat_round_trip(oracle_mod):
    """A splat facing the sensor on the ray of the centre pixel: D/O there is its range, so the
    back-projected point is the splat centre."""
    v = scenes.View(np.eye(4), 9, 361, scenes.deg(-4), scenes.deg(4))   # pixel (4, 180) is +x
    pl, q, ls = one_splat(7.25, 0.8, 0.4, 0.4)
    D, O = _render(oracle_mod, pl, q, ls, v)
    P = oracle_mod.backproject(D, O, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max, 0.05)
    k = 4 * v.cols + 180
    np.testing.assert_allclose(P[:, k], [7.25, 0.0, 0.0], atol=2e-6)


def test_wall_points_lie_on_the_wall(oracle_mod):
    """One large splat in the plane x = 5 facing the sensor: every pixel it covers back-projects
    onto that plane (single contributor: D/O is the hit range exactly), and uncovered pixels
    are invalid (NaN)."""
    v = scenes.View(np.eye(4), 16, 256, scenes.deg(-10), scenes.deg(10))
    pl, q, ls = one_splat(5.0, 0.9, 2.0, 2.0)
    D, O = _render(oracle_mod, pl, q, ls, v)
    P = oracle_mod.backproject(D, O, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max, 0.05)
    valid = O.ravel() >= 0.05
    assert valid.sum() > 200 and (~valid).sum() > 200
    np.testing.assert_allclose(P[0, valid], 5.0, atol=5e-6)
    assert np.isnan(P[:, ~valid]).all()


def test_pose_moves_the_cloud_rigidly(oracle_mod):
    """The cloud at a pose T_ws is T_ws applied to the cloud at the identity, and the pairwise
    distances of the points do not change."""
    v = scenes.View(np.eye(4), 16, 256, scenes.deg(-10), scenes.deg(10))
    pl, q, ls = one_splat(5.0, 0.9, 2.0, 2.0)
    D, O = _render(oracle_mod, pl, q, ls, v)
    T = scenes.random_pose(np.random.default_rng(3), 2.0, 40.0)
    P0 = oracle_mod.backproject(D, O, np.eye(4), v.rows, v.cols, v.elev_min, v.elev_max, 0.05)
    P1 = oracle_mod.backproject(D, O, T, v.rows, v.cols, v.elev_min, v.elev_max, 0.05)
    ok = ~np.isnan(P0[0])
    np.testing.assert_allclose(P1[:, ok], T[:3, :3] @ P0[:, ok] + T[:3, 3:4], atol=1e-9)
    a, b = P0[:, ok][:, :50], P1[:, ok][:, :50]
    da = np.linalg.norm(a[:, :, None] - a[:, None, :], axis=0)
    db = np.linalg.norm(b[:, :, None] - b[:, None, :], axis=0)
    np.testing.assert_allclose(da, db, atol=1e-9)
    assert math.isclose(np.linalg.det(T[:3, :3]), 1.0, rel_tol=1e-12)
