"""splat_render_noalloc: the forward render for callers that cannot allocate device memory.

The entry point keeps all of its workspace in one array of the library, so it must give the same
images as the context-based splat_render, call after call (the array keeps the previous call's
contents), and refuse sizes beyond its stated limits.  This file is collected last so that a run
that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_17491_gb300 import _lib, scenes
from gpu_common import D_TOL, O_TOL, COS_TOL, make_ctx, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(lib, pl, q, ls, v, cfg=None):
    P = v.rows * v.cols
    out = (torch.full((P,), float("nan"), device="cuda"),
           torch.full((3, P), float("nan"), device="cuda"),
           torch.full((P,), float("nan"), device="cuda"))
    g = _lib.splat_gaussians(pl.data_ptr(), q.data_ptr(), ls.data_ptr(), pl.shape[0])
    T = np.ascontiguousarray(v.T_ws, np.float64)
    intr = _lib.splat_lidar_intrinsics(v.rows, v.cols, v.elev_min, v.elev_max)
    code = lib.splat_render_noalloc(ctypes.byref(g), T.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.byref(intr), cfg, out[0].data_ptr(),
                                    out[1].data_ptr(), out[2].data_ptr(),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, out


def _close(a, b):
    d0, n0, o0 = (x.cpu().numpy() for x in a)
    d1, n1, o1 = (x.cpu().numpy() for x in b)
    assert np.isfinite(d1).all() and np.isfinite(n1).all() and np.isfinite(o1).all()
    assert np.abs(d1 - d0).max() <= D_TOL
    assert np.abs(o1 - o0).max() <= O_TOL
    nr, ng = np.linalg.norm(n0, axis=0), np.linalg.norm(n1, axis=0)
    m = nr > 1e-6
    cos = np.sum(n0 * n1, 0)[m] / (nr[m] * ng[m])
    assert (1 - cos).max(initial=0) <= COS_TOL


def test_noalloc_render_matches_context_render_twice():
    lib = _lib.load()
    s = scenes.tiny_scene(3000, 21, rows=48, cols=512, fov_deg=20, dist=(0.8, 40.0),
                          log_scale=(-3.0, -0.8))
    s.views[0].T_ws = scenes.random_pose(np.random.default_rng(5), 1.0, 10.0)
    v = s.views[0]
    pl, q, ls = to_dev(s)
    ctx = make_ctx(s.n, [v])
    ref = ctx.render(pl, q, ls)
    torch.cuda.synchronize()
    assert float(ref[2].max()) > 0.5
    for _ in range(2):
        code, out = _noalloc(lib, pl, q, ls, v)
        assert code == 0, lib.splat_error_string(code)
        _close(ref, out)
    # a second, different view in between keeps working on the shared array
    v2 = scenes.View(np.eye(4), 32, 1024, scenes.deg(-15), scenes.deg(15))
    ctx2 = make_ctx(s.n, [v2])
    ref2 = ctx2.render(pl, q, ls)
    code, out2 = _noalloc(lib, pl, q, ls, v2)
    assert code == 0
    _close(ref2, out2)
    code, out = _noalloc(lib, pl, q, ls, v)
    assert code == 0
    _close(ref, out)


def test_noalloc_rejects_sizes_beyond_its_limits():
    lib = _lib.load()
    s = scenes.tiny_scene(16385, 1)
    pl, q, ls = to_dev(s)
    code, _ = _noalloc(lib, pl, q, ls, s.views[0])
    assert code == _lib.SPLAT_OK + 1   # SPLAT_ERR_INVALID_ARG
    s2 = scenes.tiny_scene(10, 1)
    pl, q, ls = to_dev(s2)
    big = scenes.View(np.eye(4), 257, 64, scenes.deg(-10), scenes.deg(10))
    assert _noalloc(lib, pl, q, ls, big)[0] == 1
    wide = scenes.View(np.eye(4), 64, 2048, scenes.deg(-10), scenes.deg(10))
    assert _noalloc(lib, pl, q, ls, wide)[0] == 1
