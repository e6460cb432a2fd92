"""The documented size limits on the GPU: the most views one call takes (64), the widest and the
tallest image (32,767 columns or rows), and one view past the limit rejected.  Lists bit-exact
against the oracle, sampled pixels composited by the oracle.  Marked gpu."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import check_lists, compare_images, make_ctx, oracle_view, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_sixty_four_views_in_one_call():
    """64 uneven views (the most a context takes) of one map: lists bit-exact, and the batched
    images of a few views bit-identical to rendering those views alone."""
    s = scenes.workload(3, n=3_000)
    rng = np.random.default_rng(64)
    views = []
    for k in range(64):
        rows = int(rng.choice([16, 24, 32, 40]))
        cols = int(rng.choice([128, 256, 300, 512]))
        T = s.views[k % len(s.views)].T_ws.copy()
        T[:3, 3] += rng.normal(0, 0.5, 3)
        views.append(scenes.View(T, rows, cols, scenes.deg(-15), scenes.deg(12)))
    ctx = make_ctx(s.n, views)
    pl, q, ls = to_dev(s)
    d, n, a = ctx.render(pl, q, ls)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert check_lists(ctx, s, views) > 0
    for k in (0, 31, 63):
        c1 = make_ctx(s.n, [views[k]])
        d1, n1, a1 = c1.render(pl, q, ls)
        o, P = ctx.offsets[k], views[k].rows * views[k].cols
        np.testing.assert_array_equal(d[o:o + P].cpu().numpy(), d1.cpu().numpy())
        np.testing.assert_array_equal(a[o:o + P].cpu().numpy(), a1.cpu().numpy())
    with pytest.raises(api._lib.SplatError):
        api.SplatContext(s.n, 65, 1000)


@pytest.mark.parametrize("rows,cols", [(40, 32767), (32767, 8)])
def test_widest_and_tallest_image(rows, cols):
    """An image at the column limit (an azimuth step of 0.011 degrees) and one at the row limit
    (an elevation step of 0.001 degrees): lists bit-exact, sampled pixels within tolerance."""
    s = scenes.tiny_scene(60, 9, rows=rows, cols=cols, fov_deg=30, dist=(2.0, 20.0),
                          log_scale=(-3.5, -2.0))
    v = s.views[0]
    ctx = make_ctx(s.n, [v])
    d, n, a = ctx.render(*to_dev(s))
    torch.cuda.synchronize()
    assert ctx.status() == 0
    check_lists(ctx, s, [v])
    dn, nn, an = d.cpu().numpy(), n.cpu().numpy(), a.cpu().numpy()
    covered = np.nonzero(an > 0)[0]
    assert covered.size > 100
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(covered, 1500), rng.integers(0, v.n_pixels, 500)])
    px = np.stack([idx // v.cols, idx % v.cols], 1)
    ref, *_ = oracle_view(s, v, pixels=px)
    compare_images(dn[idx], nn[:, idx], an[idx], ref, f"{rows}x{cols}")
