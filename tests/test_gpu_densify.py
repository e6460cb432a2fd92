"""GPU parity of map growth (splat_densify): the drawn pixels bit-exact against the oracle's
integer draw, the new primitives within binary32 tolerance.  Marked gpu."""
import math

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


def _setup(n=20_000, which=(0, 2, 5)):
    s = scenes.workload(3, n=n)
    views = [s.views[k] for k in which]
    t_depth = np.concatenate([scenes.render_targets(s, v)[0].ravel() for v in views])
    return s, views, t_depth.astype(np.float32)


def _grown(s, n_new):
    pl, q, ls = to_dev(s)
    cap = s.n + n_new
    out = []
    for t, w in ((pl, 4), (q, 4), (ls, 2)):
        big = torch.full((cap, w), 7.0, device="cuda")
        big[:s.n] = t
        out.append(big)
    return out


def _compare(params, n_old, ref, label):
    pl, q, ls = (t[n_old:].cpu().numpy().astype(np.float64) for t in params)
    rpl, rq, rls, pix = ref
    filled = pix >= 0
    gpu_filled = pl[:, 3] != oracle.DENSIFY_EMPTY_LOGIT
    np.testing.assert_array_equal(gpu_filled, filled, err_msg=label)
    tol = 1e-4 + 2e-6 * np.abs(rpl[:, :3]).max(1, keepdims=True)
    assert (np.abs(pl[:, :3] - rpl[:, :3]) <= tol).all(), (label, np.abs(pl[:, :3] - rpl[:, :3]).max())
    np.testing.assert_allclose(pl[:, 3], rpl[:, 3], atol=1e-6)
    np.testing.assert_allclose(q, rq, atol=2e-6)
    np.testing.assert_allclose(ls, rls, atol=2e-6)
    return int(filled.sum())


def _oracle_views(views):
    return [(v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max) for v in views]


def test_initialisation_draws_match_the_oracle():
    """Valid-mask growth over three posed views of uneven shapes, two calls in a row (the second
    uses the next counter of the random stream)."""
    s, views, t_depth = _setup()
    n_new = 6000
    ctx = make_ctx(s.n, views)
    cfg = api.DensifyConfig(w0=0.05, w_cap=2.0, scale_k=2.0, opacity=0.4, seed=77)
    Dt = torch.from_numpy(t_depth).cuda()
    for call in range(2):
        params = _grown(s, n_new)
        ctx.densify(params, s.n, n_new, Dt, cfg=cfg)
        torch.cuda.synchronize()
        ref = oracle.densify(_oracle_views(views), t_depth, None, None, n_new, refine=False,
                             w0=0.05, w_cap=2.0, scale_k=2.0, opacity=0.4, seed=77, call=call)
        filled = _compare(params, s.n, ref, f"call {call}")
        assert filled > 0.9 * n_new
        orig = to_dev(s)
        for a, b in zip(params, orig):
            torch.testing.assert_close(a[:s.n], b, rtol=0, atol=0)


def test_refinement_masks_match_the_oracle():
    """Densification during refinement: M_n and M_e on the rendered images of the current map."""
    s, views, t_depth = _setup(n=8_000)
    ctx = make_ctx(s.n, views)
    d, n, a = ctx.render(*to_dev(s))
    torch.cuda.synchronize()
    n_new = 3000
    params = _grown(s, n_new)
    cfg = api.DensifyConfig(refine=True, lambda_do=0.6, lambda_de=0.2, w0=0.1, w_cap=4.0,
                            scale_k=1.0, opacity=0.5, seed=5)
    ctx.densify(params, s.n, n_new, torch.from_numpy(t_depth).cuda(), d, a, cfg)
    torch.cuda.synchronize()
    D, O = d.cpu().numpy(), a.cpu().numpy()
    ref = oracle.densify(_oracle_views(views), t_depth, D, O, n_new, refine=True, lambda_do=0.6,
                         lambda_de=0.2, w0=0.1, w_cap=4.0, scale_k=1.0, opacity=0.5, seed=5,
                         call=0)
    assert _compare(params, s.n, ref, "refine") > 100


def test_grown_map_renders_and_empty_slots_are_inert():
    """Nothing masked writes every slot empty; empty slots take no pairs and set no status."""
    s, views, t_depth = _setup(n=5_000, which=(1,))
    ctx = make_ctx(s.n + 500, views)
    params = _grown(s, 500)
    ctx.densify(params, s.n, 500, torch.zeros_like(torch.from_numpy(t_depth)).cuda())
    torch.cuda.synchronize()
    assert (params[0][s.n:, 3] == -30.0).all()
    d0, n0, a0 = make_ctx(s.n, views).render(*to_dev(s))
    d1, n1, a1 = ctx.render(*params)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    torch.testing.assert_close(d1, d0, rtol=0, atol=0)
    torch.testing.assert_close(a1, a0, rtol=0, atol=0)
    # a real draw: the new primitives cover the valid pixels they were drawn from
    ctx.densify(params, s.n, 500, torch.from_numpy(t_depth).cuda(),
                cfg=api.DensifyConfig(scale_k=3.0, opacity=0.9))
    only_new = [t[s.n:].contiguous() for t in params]
    c2 = make_ctx(500, views)
    d2, n2, a2 = c2.render(*only_new)
    torch.cuda.synchronize()
    assert c2.status() == 0 and float(a2.max()) > 0.5


def test_invalid_densify_arguments():
    s, views, t_depth = _setup(n=1_000, which=(1,))
    ctx = make_ctx(s.n, views)
    params = _grown(s, 10)
    Dt = torch.from_numpy(t_depth).cuda()
    with pytest.raises(api._lib.SplatError):   # no room
        ctx.densify(params, s.n, 11, Dt)
    with pytest.raises(api._lib.SplatError):   # refinement needs the rendered images
        ctx.densify(params, s.n, 10, Dt, cfg=api.DensifyConfig(refine=True))
    with pytest.raises(api._lib.SplatError):
        ctx.densify(params, s.n, 10, Dt, cfg=api.DensifyConfig(w_cap=20.0))
    with pytest.raises(api._lib.SplatError):
        ctx.densify(params, s.n, 10, Dt, cfg=api.DensifyConfig(opacity=1.0))
