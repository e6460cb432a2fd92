"""GPU parity of the self-regularised normal term (Eq. loss_normal with the normals of the
rendered range map) through splat_view_loss and splat_refine_step.  Marked gpu."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import make_ctx, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _scene_and_targets(n=20_000, which=(0, 2, 5)):
    s = scenes.workload(3, n=n)
    views = [s.views[k] for k in which]
    targets = [scenes.render_targets(s, v) for v in views]
    t_depth = np.concatenate([t[0].ravel() for t in targets]).astype(np.float32)
    t_normal = np.concatenate([t[1].reshape(3, -1) for t in targets], 1).astype(np.float32)
    return s, views, t_depth, t_normal


def _oracle_view_loss(ctx, views, D, N, O, Dt, lam_n, lam_o, o_eps):
    """Oracle: the L1 and opacity terms per pixel plus the range-map normal term per view."""
    L, gD, gN, gO = oracle.loss(D, N, O, Dt, np.zeros_like(N), 0.0, lam_o, o_eps)
    for k, v in enumerate(views):
        sl = slice(ctx.offsets[k], ctx.offsets[k] + v.n_pixels)
        val, gd, gn = oracle.range_normal_loss(D[sl], N[:, sl], Dt[sl], v.rows, v.cols,
                                               v.elev_min, v.elev_max, lam_n)
        L += val
        gD[sl] += gd.ravel()
        gN[:, sl] = gn.reshape(3, -1)
    return L, gD, gN, gO


def _close_fraction(a, b, rel, floor):
    return np.mean(np.abs(a - b) <= rel * np.maximum(np.abs(b), floor))


def test_view_loss_range_map_normals_parity():
    """Rendered images of three uneven views: the loss and its gradients against the FP64 oracle
    on the same binary32 images.  The term's sign decision (which side faces the sensor) is taken
    in binary32 on the GPU and in binary64 by the oracle, so a few grazing stencils may differ."""
    s, views, t_depth, t_normal = _scene_and_targets()
    ctx = make_ctx(s.n, views)
    pl, q, ls = to_dev(s)
    d, n, a = ctx.render(pl, q, ls)
    cfg = api.LossConfig(lambda_n=0.7, lambda_o=0.1, o_eps=1e-6, normal_mode=1)
    L, gD, gN, gO = ctx.view_loss(d, n, a, torch.from_numpy(t_depth).cuda(), None, cfg)
    torch.cuda.synchronize()
    D, N, O = d.cpu().numpy(), n.cpu().numpy(), a.cpu().numpy()
    Lr, gDr, gNr, gOr = _oracle_view_loss(ctx, views, D.astype(np.float64), N.astype(np.float64),
                                          O.astype(np.float64), t_depth.astype(np.float64), 0.7,
                                          0.1, 1e-6)
    stencils = int((np.abs(gNr).sum(0) > 0).sum())
    assert stencils > 0.3 * ctx.n_pixels
    assert float(L) == pytest.approx(Lr, rel=5e-4)
    np.testing.assert_allclose(gO.cpu().numpy(), gOr, rtol=1e-5, atol=1e-7)
    fN = _close_fraction(gN.cpu().numpy(), gNr, 1e-3, 0.7)
    fD = _close_fraction(gD.cpu().numpy(), gDr, 2e-3, 1.0)
    assert fN >= 0.9995 and fD >= 0.9995, (fN, fD)
    assert np.isfinite(gD.cpu().numpy()).all()


def test_view_loss_target_mode_matches_splat_loss():
    """normal_mode 0 through splat_view_loss is the context-free splat_loss."""
    s, views, t_depth, t_normal = _scene_and_targets(n=5_000, which=(1,))
    ctx = make_ctx(s.n, views)
    d, n, a = ctx.render(*to_dev(s))
    Dt, Nt = torch.from_numpy(t_depth).cuda(), torch.from_numpy(t_normal).cuda()
    cfg = api.LossConfig(lambda_n=0.4, lambda_o=0.2)
    A = ctx.view_loss(d, n, a, Dt, Nt, cfg)
    B = api.loss(d, n, a, Dt, Nt, cfg)
    for x, y in zip(A[1:], B[1:]):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
    assert float(A[0]) == pytest.approx(float(B[0]), rel=1e-6)


def test_bad_normal_modes_are_rejected():
    s, views, t_depth, t_normal = _scene_and_targets(n=1_000, which=(1,))
    ctx = make_ctx(s.n, views)
    d, n, a = ctx.render(*to_dev(s))
    Dt = torch.from_numpy(t_depth).cuda()
    with pytest.raises(api._lib.SplatError):   # target mode needs target normals
        ctx.view_loss(d, n, a, Dt, None, api.LossConfig())
    with pytest.raises(api._lib.SplatError):
        ctx.view_loss(d, n, a, Dt, None, api.LossConfig(normal_mode=2))
    with pytest.raises(api._lib.SplatError):   # the context-free loss has no view geometry
        api.loss(d, n, a, Dt, torch.zeros_like(n), api.LossConfig(normal_mode=1))


def test_refine_step_range_map_normals():
    """splat_refine_step in the range-map normal mode: its loss is that of splat_view_loss on the
    same render, and a few steps reduce it."""
    s, views, t_depth, _ = _scene_and_targets(n=20_000, which=(0, 1, 2))
    Dt = torch.from_numpy(t_depth).cuda()
    cfg = api.LossConfig(lambda_n=0.2, normal_mode=1)
    ctx = make_ctx(s.n, views)
    params = [t.clone() for t in to_dev(s)]
    d, n, a = ctx.render(*params)
    L0 = float(ctx.view_loss(d, n, a, Dt, None, cfg)[0])
    state = api.adam_state(s.n)
    loss_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ls = []
    for _ in range(6):
        ctx.refine_step(params, state, Dt, None, cfg, api.AdamConfig(), loss_out)
        ls.append(float(loss_out.item()))
    assert ls[0] == pytest.approx(L0, rel=1e-5)
    assert ls[-1] < ls[0]


@pytest.mark.parametrize("p", [-1.0, 0.5])
def test_range_weight_parity(p):
    """rho_d = Dt^p on the L1 range term, context-free splat_loss against the oracle."""
    rng = np.random.default_rng(12)
    P = 6000
    D = rng.uniform(0, 60, P).astype(np.float32)
    N = rng.normal(size=(3, P)).astype(np.float32)
    O = rng.uniform(0, 1, P).astype(np.float32)
    Dt = np.where(rng.uniform(size=P) < 0.2, 0, rng.uniform(0.5, 60, P)).astype(np.float32)
    Nt = rng.normal(size=(3, P)).astype(np.float32)
    cfg = api.LossConfig(lambda_n=0.3, lambda_o=0.05, rho_exp=p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    L, gD, gN, gO = api.loss(t(D), t(N), t(O), t(Dt), t(Nt), cfg)
    Lr, gDr, gNr, gOr = oracle.loss(D, N, O, Dt, Nt, 0.3, 0.05, 1e-6, rho_exp=p)
    assert float(L) == pytest.approx(Lr, rel=1e-5)
    np.testing.assert_allclose(gD.cpu().numpy(), gDr, rtol=2e-6, atol=1e-7)
