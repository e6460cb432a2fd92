"""GPU parity of the photometric residual and its Gauss-Newton normal equations
(splat_photometric) against the FP64 oracle.  Marked gpu."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import make_ctx, to_dev
from test_oracle_photometric import se3_exp

pytestmark = pytest.mark.gpu


def _t34(T):
    return torch.from_numpy(np.asarray(T, np.float32)[:3, :4].copy()).cuda()


def _setup(n=30_000, rows=64, cols=1024):
    s = scenes.workload(3, n=n)
    v = s.views[0]
    vm = scenes.View(v.T_ws, rows, cols, v.elev_min, v.elev_max)
    motion = se3_exp([0.6, -0.2, 0.05, 0.0, 0.01, 0.03])
    vq = scenes.View(v.T_ws @ motion, rows, cols, v.elev_min, v.elev_max)
    Dq = scenes.render_targets(s, vq, noise=0.0)[0].ravel().astype(np.float32)
    T_true = np.linalg.inv(vq.T_ws) @ vm.T_ws
    return s, vm, Dq, T_true


# Ambiguity band of the photometric residual (oracle.photometric_normal_eqs): pixels whose u' lies
# within PHOTO_BAND_PX of a cell edge (the binary32 floor of u' may pick the neighbouring bilinear
# cell), or where the query image's slopes move the sample by more than PHOTO_BAND_R when u' moves
# by PHOTO_BAND_PX.  PHOTO_BAND_PX is about the binary32 error of u' (c' near 1024 columns carries
# a rounding of 6e-5 px, the arctangent about as much again); measured on GB300 on both scenes
# below, no pixel differed from the oracle by more than 6.1e-4 m in r or 2.7e-4 in J even with no
# band at all.
PHOTO_BAND_PX, PHOTO_BAND_R = 1e-4, 1e-3


@pytest.mark.parametrize("n,rows", [(30_000, 64), (100_000, 128)])
def test_photometric_parity_on_a_rendered_view(n, rows):
    """The render of the map at the model pose against a ray-cast query scan: per-pixel
    residuals, weights and Jacobians within 1e-3 of the oracle's outside the ambiguity band (at
    most 1 % of the used pixels), the same set of used pixels everywhere, and the reduced normal
    equations of the unflagged pixels within 1e-3."""
    s, vm, Dq, T_true = _setup(n=n, rows=rows)
    ctx = make_ctx(s.n, [vm])
    d, nn, a = ctx.render(*to_dev(s))
    T = (T_true @ se3_exp([0.05, -0.03, 0.01, 0.002, 0.0, 0.004])).astype(np.float32)
    out, px = ctx.photometric(0, d, a, torch.from_numpy(Dq).cuda(), _t34(T), o_min=0.5,
                              huber_delta=0.3, per_pixel=True)
    torch.cuda.synchronize()
    D, O = d.cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64)
    T64 = np.eye(4)
    T64[:3] = T[:3].astype(np.float64)
    ref = oracle.photometric_normal_eqs(D, O, Dq.astype(np.float64), T64, vm.rows, vm.cols,
                                        vm.elev_min, vm.elev_max, 0.5, 0.3,
                                        band_px=PHOTO_BAND_PX, band_r=PHOTO_BAND_R)
    px = px.cpu().numpy().astype(np.float64)
    used = px[1] > 0
    assert ref["count"] > 5000
    ok = ~ref["band"]
    assert (ref["band"] & ref["used"]).sum() <= 0.01 * ref["count"]
    np.testing.assert_array_equal(used[ok], ref["used"][ok])
    both = used & ref["used"] & ok
    assert np.abs(px[0][both] - ref["r"][both]).max() <= 1e-3
    assert np.abs(px[1][both] - ref["w"][both]).max() <= 1e-3
    J = px[2:].T[both]
    Jr = ref["J"][both]
    assert (np.abs(J - Jr) <= 1e-3 * np.maximum(np.abs(Jr).max(1, keepdims=True), 1.0)).all()
    # the reduction equals the sum of the kernel's own per-pixel terms
    H, g, cost, count = api.unpack_normal_eqs(out)
    w = px[1]
    Hs = (px[2:] * w) @ px[2:].T
    gs = (px[2:] * w) @ px[0]
    assert count == int(used.sum())
    np.testing.assert_allclose(H, Hs, rtol=1e-4, atol=1e-4 * np.abs(Hs).max())
    np.testing.assert_allclose(g, gs, rtol=1e-4, atol=1e-4 * np.abs(gs).max())
    # the normal equations of the unflagged pixels against the oracle's
    wu = np.where(both, w, 0.0)
    Hu = (px[2:] * wu) @ px[2:].T
    gu = (px[2:] * wu) @ px[0]
    Jo, wo, ro = ref["J"], np.where(both, ref["w"], 0.0), ref["r"]
    Ho = (Jo.T * wo) @ Jo
    go = (Jo.T * wo) @ ro
    assert np.linalg.norm(Hu - Ho) <= 1e-3 * np.linalg.norm(Ho)
    assert np.linalg.norm(gu - go) <= 1e-3 * np.linalg.norm(go)
    # the Huber cost over all used pixels
    assert cost == pytest.approx(ref["cost"], rel=1e-3)


def test_gauss_newton_on_the_gpu_recovers_a_known_pose():
    """Ray-cast model and query scans (exact ranges): Gauss-Newton steps with the GPU's normal
    equations, the pose update on the host, bring a 0.15 m / 1 degree offset down five-fold (the
    oracle's own iteration on these images needs ten steps for that)."""
    s, vm, Dq, T_true = _setup(n=1000)
    D = scenes.render_targets(s, vm, noise=0.0)[0].ravel().astype(np.float32)
    O = (D > 0).astype(np.float32)
    ctx = make_ctx(s.n, [vm])
    Dt, Ot, Qt = (torch.from_numpy(x).cuda() for x in (D, O, Dq))
    T = T_true @ se3_exp([0.12, -0.08, 0.03, 0.0, 0.0, math.radians(1.0)])

    def err(T):
        E = np.linalg.inv(T_true) @ T
        return np.linalg.norm(E[:3, 3]), math.acos(max(-1.0, min(1.0, (np.trace(E[:3, :3]) - 1) / 2)))

    e0 = err(T)
    for _ in range(11):
        H, g, cost, count = api.unpack_normal_eqs(ctx.photometric(0, Dt, Ot, Qt, _t34(T), 0.5, 0.3))
        T = T @ se3_exp(-np.linalg.solve(H + 1e-9 * np.eye(6), g))
    e1 = err(T)
    assert e1[0] < 0.2 * e0[0] and e1[1] < 0.2 * e0[1], (e0, e1)


def test_photometric_arguments():
    s, vm, Dq, T_true = _setup(n=500, rows=16, cols=64)
    ctx = make_ctx(s.n, [vm])
    d, n, a = ctx.render(*to_dev(s))
    Q = torch.from_numpy(Dq).cuda()
    with pytest.raises(api._lib.SplatError):
        ctx.photometric(1, d, a, Q, _t34(np.eye(4)))
    with pytest.raises(api._lib.SplatError):
        ctx.photometric(0, d, a, Q, _t34(np.eye(4)), o_min=0.0)
    out = ctx.photometric(0, d, a, torch.zeros_like(Q), _t34(np.eye(4)))
    H, g, cost, count = api.unpack_normal_eqs(out)
    assert count == 0 and not H.any() and not g.any()
