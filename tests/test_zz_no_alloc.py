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


def test_noalloc_empty_map_renders_the_background():
    """n = 0: the call succeeds and every output pixel is the empty composite (D = N = O = 0)."""
    lib = _lib.load()
    v = scenes.View(np.eye(4), 32, 256, scenes.deg(-10), scenes.deg(10))
    z4 = torch.zeros(0, 4, device="cuda")
    code, out = _noalloc(lib, z4, z4.clone(), torch.zeros(0, 2, device="cuda"), v)
    assert code == 0, lib.splat_error_string(code)
    for t in out:
        assert float(t.abs().max()) == 0.0


def test_noalloc_pair_overflow_returns_capacity():
    """Large splats close around the sensor bin about 526,000 (tile, primitive) pairs, more than
    the array's 262,144: the device-side count stops at the limit and the call returns
    SPLAT_ERR_CAPACITY; the next call within the limits renders correctly again."""
    import math
    lib = _lib.load()
    rng = np.random.default_rng(31)
    n = 6000
    g = rng.uniform(-math.pi, math.pi, n)
    r = rng.uniform(2.0, 4.0, n)
    p = np.stack([r * np.cos(g), r * np.sin(g), rng.uniform(-0.3, 0.3, n)], 1)
    pl, q, ls = scenes.gaussians_on(p, -p, rng, log_scale=(0.3, 0.5))
    pl[:, 3] = math.log(0.6 / 0.4)
    v = scenes.View(np.eye(4), 64, 1024, scenes.deg(-20), scenes.deg(20))
    big = scenes.Scene("wide", pl, q, ls, [v])
    code, _ = _noalloc(lib, *to_dev(big), v)
    assert code == 3, lib.splat_error_string(code)   # SPLAT_ERR_CAPACITY
    s = scenes.tiny_scene(500, 4, rows=32, cols=256)
    pl2, q2, ls2 = to_dev(s)
    ref = make_ctx(s.n, s.views).render(pl2, q2, ls2)
    code, out = _noalloc(lib, pl2, q2, ls2, s.views[0])
    assert code == 0
    _close(ref, out)


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np
import torch
from paper_2503_17491_gb300 import _lib, scenes
import test_zz_no_alloc as t
lib = _lib.load()
s = scenes.tiny_scene(2000, 9, rows=32, cols=512, fov_deg=20, dist=(0.8, 40.0))
v = s.views[0]
pl, q, ls = t.to_dev(s)
outs = []
for _ in range(2):
    code, out = t._noalloc(lib, pl, q, ls, v)
    assert code == 0, lib.splat_error_string(code)
    outs.append(out)
ref = t.make_ctx(s.n, [v]).render(pl, q, ls)
torch.cuda.synchronize()
for out in outs:
    t._close(ref, out)
print("fresh process ok")
"""


def test_noalloc_first_call_of_a_fresh_process_with_lazy_loading():
    """In a new process with CUDA's lazy module loading, the allocation-free render is the first
    call into the library (no context exists yet): its set-up call loads what it uses and finds
    the array, and two calls in a row match the context render made afterwards."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    code = _FRESH.format(root=os.path.dirname(here), tests=here)
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh process ok" in r.stdout
