"""GPU back-projection of rendered range images (splat_backproject) against the oracle's, on the
same rendered images.  Marked gpu."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import scenes
from gpu_common import make_ctx, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


@pytest.mark.parametrize("o_min", [0.5, 0.05])
def test_backproject_batched_views(o_min):
    """Several posed views in one call: the valid pixels are the same (the decision O >= o_min
    is taken on the same binary32 values), and every point agrees with the FP64 oracle within
    the binary32 ray and pose rounding (~1e-7 of the range and of the pose translation)."""
    s = scenes.workload(3, n=20_000)
    views = [s.views[0], s.views[4], s.views[9]]
    ctx = make_ctx(s.n, views)
    d, n, a = ctx.render(*to_dev(s))
    pts = ctx.backproject(d, a, o_min).cpu().numpy().astype(np.float64)
    D, O = d.cpu().numpy(), a.cpu().numpy()
    for k, v in enumerate(views):
        sl = slice(ctx.offsets[k], ctx.offsets[k] + v.n_pixels)
        ref = oracle.backproject(D[sl], O[sl], v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max,
                                 o_min)
        got = pts[:, sl]
        vr, vg = ~np.isnan(ref[0]), ~np.isnan(got[0])
        np.testing.assert_array_equal(vr, vg)
        assert vr.sum() > 0.05 * v.n_pixels
        rng = np.where(vr, D[sl] / np.where(vr, O[sl], 1), 0)
        tol = 2e-6 * (rng[vr] + np.abs(v.T_ws[:3, 3]).sum()) + 1e-5
        err = np.abs(got[:, vr] - ref[:, vr]).max(0)
        assert (err <= tol).all(), (err.max(), tol[err.argmax()])
