"""GPU gradient, loss, Adam and refinement-step parity through the C ABI.  Marked gpu."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import (BAND, BAND_CAP, compare_grads, gpu_grads_as_oracle, make_ctx, oracle_view, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _band_mask(band):
    """1 outside the ambiguity band, 0 inside; the band may take out at most BAND_CAP of the
    pixels."""
    inside = int((band != 0).sum())
    assert inside <= BAND_CAP * band.size, (inside, band.size)
    return (band == 0).astype(np.float64)


def _upstream(v, band, seed):
    """Random upstream gradients, zero on ambiguity-band pixels."""
    rng = np.random.default_rng(seed)
    gD = rng.normal(size=(v.rows, v.cols))
    gN = rng.normal(size=(3, v.rows, v.cols))
    gO = rng.normal(size=(v.rows, v.cols))
    m = _band_mask(band)
    return gD * m, gN * m, gO * m


def _coherent_upstream(v, band, seed):
    """Upstream gradients of one sign in range and opacity (dL/dD ~ 1, dL/dO ~ 0.5, small normal
    terms), zero on ambiguity-band pixels.  A pose gradient is a sum over all pixels; with
    random-sign upstream gradients it cancels down to ~1/sqrt(pixels) of its terms' magnitude,
    and its relative error grows by the same factor, so pose sums are compared on inputs that
    do not cancel."""
    rng = np.random.default_rng(seed)
    gD = 1.0 + 0.2 * rng.normal(size=(v.rows, v.cols))
    gN = 0.05 * rng.normal(size=(3, v.rows, v.cols))
    gO = 0.5 + 0.1 * rng.normal(size=(v.rows, v.cols))
    m = _band_mask(band)
    return gD * m, gN * m, gO * m


def _grad_parity(s, tile=(16, 16), seed=0, label=""):
    v = s.views[0]
    ref, params, flip, cul = oracle_view(s, v, tile)
    gD, gN, gO = _upstream(v, ref["band"], seed)
    g_ref = oracle.render_backward(params, flip, None, v.T_ws, v.rows, v.cols, v.elev_min,
                                   v.elev_max, gD, gN, gO, culled=cul)
    ctx = make_ctx(s.n, s.views, tile)
    ctx.set_pose_gradient(True)
    pl, q, ls = to_dev(s)
    ctx.render(pl, q, ls)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
    g = ctx.backward(pl, q, ls, f(gD.ravel()), f(gN.reshape(3, -1)), f(gO.ravel()))
    torch.cuda.synchronize()
    got = gpu_grads_as_oracle(*g)
    _pose_parity(ctx.pose_gradients()[0].double().cpu().numpy(), g_ref["g_pose"], label)
    return compare_grads(got, {k: g_ref[k] for k in got}, label), ctx


def _pose_parity(got, ref, label=""):
    """Pose gradient (dL/drho, dL/domega): each 3-vector within the gradient tolerance of the
    oracle's, relative to its own norm."""
    for part, sl in (("rho", slice(0, 3)), ("omega", slice(3, 6))):
        nb = np.linalg.norm(ref[sl])
        assert nb > 0, (label, part)
        rel = np.linalg.norm(got[sl] - ref[sl]) / nb
        assert rel <= 1e-3, (label, part, got[sl], ref[sl], rel)


@pytest.mark.parametrize("tile", [(16, 16), (4, 64)])
def test_grad_parity_workload0(tile):
    _grad_parity(scenes.workload(0), tile, 1, "workload0")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grad_parity_tiny_posed(seed):
    s = scenes.tiny_scene(60, seed, rows=24, cols=128, fov_deg=25, dist=(1.0, 20.0),
                          log_scale=(-2.5, -0.6))
    s.views[0].T_ws = scenes.random_pose(np.random.default_rng(seed + 3), 1.0, 15.0)
    _grad_parity(s, (16, 16), seed, "tiny")


def test_grad_parity_workload1():
    res, ctx = _grad_parity(scenes.workload(1), (16, 16), 4, "workload1")
    st = ctx.stats()
    assert st["bwd_evals"] > 0 and st["fwd_evals"] >= st["bwd_evals"] // 2


def test_grad_against_fp64_finite_differences():
    """GPU gradient against central finite differences of the FP64 oracle (tiny scene)."""
    s = scenes.tiny_scene(6, 11, rows=12, cols=48, fov_deg=20, dist=(2.0, 5.0),
                          log_scale=(-1.6, -0.8))
    s.pos_logit[:, 3] = np.minimum(s.pos_logit[:, 3], math.log(0.9 / 0.1))
    v = s.views[0]
    ref, params, flip, cul = oracle_view(s, v)
    gD, gN, gO = _upstream(v, ref["band"], 5)
    order = oracle.sort_order(oracle.project_contract(s.pos_logit, s.quat, s.log_scale, v.T_ws,
                                                      v.rows, v.cols, v.elev_min,
                                                      v.elev_max)["kappa"])

    def L(p):
        o = oracle.render(p, flip, order, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
        return (gD * o["D"]).sum() + (gN * o["N"]).sum() + (gO * o["O"]).sum(), o["n_contrib"]

    ctx = make_ctx(s.n, s.views)
    pl, q, ls = to_dev(s)
    ctx.render(pl, q, ls)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
    got = gpu_grads_as_oracle(*ctx.backward(pl, q, ls, f(gD.ravel()), f(gN.reshape(3, -1)),
                                            f(gO.ravel())))
    base = [a.copy() for a in params]
    _, nc0 = L(base)
    names = [("g_pos", 0, 3), ("g_logit", 1, 1), ("g_quat", 2, 4), ("g_log_scale", 3, 2)]
    checked = 0
    for name, gi, width in names:
        scale = np.abs(got[name]).max()
        for i in range(s.n):
            for k in range(width):
                p = [a.copy() for a in base]
                idx = (i, k) if p[gi].ndim == 2 else (i,)
                x = p[gi][idx]
                h = 1e-6 * max(1.0, abs(x))
                p[gi][idx] = x + h
                Lp, ncp = L(p)
                p[gi][idx] = x - h
                Lm, ncm = L(p)
                if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                    continue
                fd = (Lp - Lm) / (2 * h)
                assert abs(got[name][idx] - fd) <= 1e-3 * max(abs(fd), scale), (name, i, k)
                checked += 1
    assert checked >= 40


def test_multiview_grads_sum_and_autograd():
    """Gradients of a batched render equal the sum of the single-view gradients; the autograd
    Function returns the same tensors as the direct backward call."""
    s = scenes.workload(3, n=20_000)
    views = [s.views[0], s.views[2], s.views[4]]
    pl, q, ls = to_dev(s)
    ctx = make_ctx(s.n, views)
    rng = np.random.default_rng(3)
    P = sum(v.n_pixels for v in views)
    gD = torch.from_numpy(rng.normal(size=P).astype(np.float32)).cuda()
    gN = torch.from_numpy(rng.normal(size=(3, P)).astype(np.float32)).cuda()
    gO = torch.from_numpy(rng.normal(size=P).astype(np.float32)).cuda()
    ctx.render(pl, q, ls)
    gb = ctx.backward(pl, q, ls, gD, gN, gO)
    acc = tuple(torch.zeros_like(t) for t in (pl, q, ls))
    for k, v in enumerate(views):
        c1 = make_ctx(s.n, [v])
        c1.render(pl, q, ls)
        o = ctx.offsets[k]
        c1.backward(pl, q, ls, gD[o:o + v.n_pixels].contiguous(),
                    gN[:, o:o + v.n_pixels].contiguous(), gO[o:o + v.n_pixels].contiguous(),
                    out=acc, accumulate=True)
    for a, b in zip(gb, acc):
        d = (a - b).norm() / b.norm()
        assert float(d) < 1e-5, float(d)
    # autograd
    plr, qr, lsr = (t.clone().requires_grad_(True) for t in (pl, q, ls))
    d, nrm, al = api.render(plr, qr, lsr, ctx)
    ((d * gD).sum() + (nrm * gN).sum() + (al * gO).sum()).backward()
    for a, b in zip((plr.grad, qr.grad, lsr.grad), gb):
        assert float((a - b).norm() / b.norm()) < 1e-5


def test_loss_parity():
    rng = np.random.default_rng(0)
    P = 5000
    D = rng.uniform(0, 50, P).astype(np.float32)
    N = rng.normal(size=(3, P)).astype(np.float32)
    O = rng.uniform(0, 1, P).astype(np.float32)
    Dt = np.where(rng.uniform(size=P) < 0.2, 0, rng.uniform(1, 50, P)).astype(np.float32)
    Nt = rng.normal(size=(3, P)).astype(np.float32)
    Nt /= np.linalg.norm(Nt, axis=0)
    cfg = api.LossConfig(lambda_n=0.5, lambda_o=0.1, o_eps=1e-6)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    L, gD, gN, gO = api.loss(t(D), t(N), t(O), t(Dt), t(Nt), cfg)
    Lr, gDr, gNr, gOr = oracle.loss(D, N, O, Dt, Nt, 0.5, 0.1, 1e-6)
    assert float(L) == pytest.approx(Lr, rel=1e-5)
    np.testing.assert_array_equal(gD.cpu().numpy(), gDr)
    np.testing.assert_allclose(gN.cpu().numpy(), gNr, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(gO.cpu().numpy(), gOr, rtol=1e-5)


def test_adam_parity():
    rng = np.random.default_rng(1)
    n = 3000
    params = [rng.normal(size=(n, w)).astype(np.float32) for w in (4, 4, 2)]
    cfg = api.AdamConfig(lr_pos=1e-3, lr_opacity=2e-2, lr_rot=3e-3, lr_scale=5e-3, eps=1e-8)
    P = [torch.from_numpy(p.copy()).cuda() for p in params]
    state = api.adam_state(n)
    ref = [p.astype(np.float64).copy() for p in params]
    ms = [np.zeros(p.size) for p in params]
    vs = [np.zeros(p.size) for p in params]
    lrs = [np.array([1e-3, 1e-3, 1e-3, 2e-2]), np.full(4, 3e-3), np.full(2, 5e-3)]
    for step in range(1, 4):
        grads = [rng.normal(size=p.shape).astype(np.float32) for p in params]
        api.adam_step(P, [torch.from_numpy(g).cuda() for g in grads], state, cfg)
        for j in range(3):
            w = params[j].shape[1]
            for c in range(w):   # one lr per column group
                sl = np.s_[:, c]
                pr = np.ascontiguousarray(ref[j][sl])
                m = np.ascontiguousarray(ms[j].reshape(-1, w)[sl])
                vv = np.ascontiguousarray(vs[j].reshape(-1, w)[sl])
                oracle.adam(pr, grads[j][sl], m, vv, float(lrs[j][c]), 0.9, 0.999, 1e-8, step)
                ref[j][sl] = pr
                ms[j].reshape(-1, w)[sl] = m
                vs[j].reshape(-1, w)[sl] = vv
    assert int(state[-1]) == 3
    for j in range(3):
        np.testing.assert_allclose(P[j].cpu().numpy(), ref[j], rtol=0, atol=2e-6)


def test_refine_graph_replay_equals_eager():
    """The fused refinement step replayed from a CUDA graph matches the same steps run eagerly."""
    s = scenes.workload(3, n=20_000)
    views = s.views[:3]
    targets = [scenes.render_targets(s, v) for v in views]
    tt = [(torch.from_numpy(d).cuda(), torch.from_numpy(n).cuda()) for d, n in targets]
    runs = []
    for use_graph in (False, True):
        params = [t.clone() for t in to_dev(s)]
        r = api.Refiner(params, views, tt, mode="batched")
        if use_graph:
            r.capture(warmup=0)
            for _ in range(3):
                r.step()
        else:
            for _ in range(3):
                r.step()
        torch.cuda.synchronize()
        runs.append(([p.cpu().numpy() for p in params], float(r.loss_out), int(r.state[-1])))
    (pa, la, sa), (pb, lb, sb) = runs
    assert sa == sb == 3
    assert lb == pytest.approx(la, rel=1e-4)
    for a, b in zip(pa, pb):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-4)


def test_refine_step_reduces_loss_and_matches_plain():
    """Batched (fused, one pass over all keyframes) and plain (one launch sequence per keyframe)
    refinement give the same first-step loss and reduce it over a few steps."""
    s = scenes.workload(3, n=30_000)
    views = s.views[:4]
    targets = [scenes.render_targets(s, v) for v in views]
    tt = [(torch.from_numpy(d).cuda(), torch.from_numpy(n).cuda()) for d, n in targets]
    losses = {}
    for mode in ("plain", "batched"):
        params = [t.clone() for t in to_dev(s)]
        r = api.Refiner(params, views, tt, mode=mode)
        ls = []
        for _ in range(5):
            ls.append(float(r.step()))
        losses[mode] = ls
    assert losses["batched"][0] == pytest.approx(losses["plain"][0], rel=1e-5)
    assert losses["batched"][-1] < losses["batched"][0]
    assert losses["plain"][-1] == pytest.approx(losses["batched"][-1], rel=2e-3)


def test_pose_gradient_batched_views():
    """Several views of uneven shapes in one backward: each view's pose gradient against the
    oracle's for that view alone."""
    s = scenes.workload(3, n=20_000)
    views = [s.views[0], s.views[2], s.views[5]]
    ctx = make_ctx(s.n, views)
    ctx.set_pose_gradient(True)
    pl, q, ls = to_dev(s)
    ctx.render(pl, q, ls)
    P = ctx.n_pixels
    gD = np.zeros(P)
    gN = np.zeros((3, P))
    gO = np.zeros(P)
    refs = []
    for k, v in enumerate(views):
        ref, params, flip, cul = oracle_view(s, v)
        d, n, o = _coherent_upstream(v, ref["band"], 40 + k)
        sl = slice(ctx.offsets[k], ctx.offsets[k] + v.n_pixels)
        gD[sl], gN[:, sl], gO[sl] = d.ravel(), n.reshape(3, -1), o.ravel()
        refs.append(oracle.render_backward(params, flip, None, v.T_ws, v.rows, v.cols,
                                           v.elev_min, v.elev_max, d, n, o,
                                           culled=cul)["g_pose"])
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
    ctx.backward(pl, q, ls, f(gD), f(gN), f(gO))
    got = ctx.pose_gradients().double().cpu().numpy()
    for k in range(len(views)):
        _pose_parity(got[k], refs[k], f"view {k}")
    # off again: the next backward forms no pose terms and the copy is refused
    ctx.set_pose_gradient(False)
    ctx.backward(pl, q, ls, f(gD), f(gN), f(gO))
    with pytest.raises(api._lib.SplatError):
        ctx.pose_gradients()


def test_record_pool_overflow_sets_capacity_status():
    """Faint, wide splats make every 4x8 block record every primitive; with the pair capacity
    just above the pairs used and the tile capacity at the tiles used, the contributor-record
    pool runs out: the capacity status bit is set, nothing faults, and the backward still
    returns finite values.  The same scene with a generous capacity records everything."""
    rng = np.random.default_rng(12)
    n = 300
    g = rng.uniform(-1.2, 1.2, n)
    r = rng.uniform(3.0, 6.0, n)
    p = np.stack([r * np.cos(g), r * np.sin(g), rng.uniform(-0.3, 0.3, n)], 1)
    pl, q, ls = scenes.gaussians_on(p, -p, rng, log_scale=(0.4, 0.5))
    pl[:, 3] = math.log(0.02 / 0.98)
    view = scenes.View(np.eye(4), 32, 128, scenes.deg(-20), scenes.deg(20))
    s = scenes.Scene("faint", pl, q, ls, [view])
    pl_d, q_d, ls_d = to_dev(s)
    big = make_ctx(s.n, s.views)
    big.render(pl_d, q_d, ls_d)
    assert big.status() == 0
    st = big.stats()
    cfg = api.RenderConfig(tile_h=16, tile_w=16)
    ctx = api.SplatContext(s.n, 1, view.n_pixels, st["n_pairs"] + 8, cfg, max_tiles=st["n_tiles"])
    ctx.set_views(s.views)
    d, nrm, a = ctx.render(pl_d, q_d, ls_d)
    torch.cuda.synchronize()
    assert ctx.stats()["n_pairs"] == st["n_pairs"]          # the lists themselves fit
    assert ctx.status() & api._lib.SPLAT_STATUS_CAPACITY     # the records did not
    P = view.n_pixels
    g_out = ctx.backward(pl_d, q_d, ls_d, torch.ones(P, device="cuda"),
                         torch.zeros(3, P, device="cuda"), torch.zeros(P, device="cuda"))
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in g_out)


def test_refine_step_scale_term():
    """splat_refine_step with the scale term: the loss grows by the oracle's L_s, and Adam's
    first moment of the log-scales by (1 - beta1) times the oracle's L_s gradient (one step from
    zero moments, same render gradients)."""
    s = scenes.workload(3, n=20_000)
    views = s.views[:3]
    targets = [scenes.render_targets(s, v) for v in views]
    t_depth = torch.from_numpy(np.concatenate([t[0].ravel() for t in targets])).cuda()
    t_normal = torch.from_numpy(np.concatenate([t[1].reshape(3, -1) for t in targets],
                                               1)).contiguous().cuda()
    adam_cfg = api.AdamConfig()
    out = {}
    for lam in (0.0, 0.3):
        params = [t.clone() for t in to_dev(s)]
        state = api.adam_state(s.n)
        loss_out = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx = make_ctx(s.n, views)
        ctx.refine_step(params, state, t_depth, t_normal, api.LossConfig(lambda_s=lam, tau_s=0.15),
                        adam_cfg, loss_out)
        out[lam] = (float(loss_out.item()), state[2].double().cpu().numpy())
    v_s, g_s = oracle.scale_regularizer(s.log_scale, 0.3, 0.15)
    assert v_s > 0 and (g_s != 0).sum() > 1000
    assert out[0.3][0] - out[0.0][0] == pytest.approx(v_s, rel=1e-5)
    dm = (out[0.3][1] - out[0.0][1]) / (1.0 - adam_cfg.beta1)
    g_render = np.abs(out[0.0][1]) / (1.0 - adam_cfg.beta1)
    # the render gradients are summed with float atomics: the two runs differ by their rounding
    tol = 1e-4 * g_render + 1e-6
    assert (np.abs(dm - g_s) <= tol).all(), np.abs(dm - g_s).max()
