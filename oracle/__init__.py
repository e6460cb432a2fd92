"""FP64 CPU oracle of the spherical 2D-Gaussian rasterizer (Splat-LOAM, arXiv 2503.17491).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``.  The product path never imports it.

This module is a ctypes wrapper around ``splat_oracle.c`` (plain C, FP64 render and gradient,
plus its own implementation of the binary32 binning contract).  It shares no code with the CUDA
library.  Every function takes and returns numpy arrays.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  render / render_backward : pinned (closed form, invariants, finite differences, brute force)
  project_contract / bin   : pinned (brute-force coverage, wrap/pole/behind cases, series bounds)
  loss / adam              : pinned (hand-computed values, textbook Adam recurrence)
  render_backward g_pose   : pinned (finite differences of the pose through exp(xi^))
  backproject              : pinned (round trip through a rendered head-on splat, a wall at a
                             known distance, pose composition)
  sample_active_views      : pinned (frequencies of the truncated geometric law; Philox words
                             by uniformity and avalanche, no published output vectors used)
  scale_regularizer        : pinned (hand values, finite differences)
  range_normal_loss        : pinned (a planar range map gives the plane's normal; finite
                             differences in D and N)
  densify                  : pinned (systematic-sampling counts against brute-force enumeration
                             of the sample points, evenly spaced picks on flat weights, masks by
                             their definitions, a step edge's weight, selection frequencies over
                             many draws; new primitives by round trip through the projection)
  photometric_normal_eqs   : pinned (zero residual at the true pose, Jacobian by finite
                             differences of the pose, Huber weights by hand, Gauss-Newton
                             recovering a known pose offset on a synthetic scene)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splat_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile splat_oracle.c into _build/liboracle.so (gcc, no contraction of a*b+c)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_F = ctypes.c_float


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_version.restype = _I
            lib.or_pose_inverse.argtypes = [_P, _P, _P]
            lib.or_contract_atan2f.argtypes = [_F, _F]
            lib.or_contract_atan2f.restype = _F
            lib.or_contract_expf.argtypes = [_F]
            lib.or_contract_expf.restype = _F
            lib.or_project_contract.argtypes = [_I64, _P, _P, _P, _P, _I, _I, _F, _F, _I, _I,
                                                _F, _F, _I, _P, _P, _P, _P, _P, _P]
            lib.or_contract_logf.argtypes = [_F]
            lib.or_contract_logf.restype = _F
            lib.or_contract_reach_radius.argtypes = [_F, _F]
            lib.or_contract_reach_radius.restype = _F
            lib.or_bin.argtypes = [_I64, _P, _P, _P, _I, _I, _I, _I, _I64, _P, _P, _I64]
            lib.or_bin.restype = _I64
            lib.or_tile_ranges.argtypes = [_I64, _P, _I64, _I64, _P, _P]
            lib.or_sort_order.argtypes = [_I64, _P, _P]
            lib.or_render.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _I, _I,
                                      _D, _D, _I, _I, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P,
                                      _I]
            lib.or_render_backward.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P,
                                               _I, _I, _D, _D, _I, _I, _P, _P, _I64, _P, _P, _P,
                                               _P, _P, _P, _P, _P, _P, _P, _I]
            lib.or_pose_gradient.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]
            lib.or_pose_gradient.restype = None
            lib.or_reach_pairs.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _I, _D, _D, _P, _P, _P,
                                           _I64]
            lib.or_reach_pairs.restype = _I64
            lib.or_loss.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P]
            lib.or_loss.restype = _D
            lib.or_adam.argtypes = [_I64, _P, _P, _P, _P, _D, _D, _D, _D, _I]
            _lib = lib
    return _lib


def _ptr(a):
    """Raw address of an array.  The caller keeps the array referenced until the C call returns:
    a converted copy is bound to a local first, never passed inline as a temporary."""
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# Default per-pixel cutoffs (3DGS conventions; the paper gives none): alpha_min, alpha_max,
# t_min, sigma_cut.
DEFAULT_CFG = (1.0 / 255.0, 0.99, 1e-4, 3.0)

# Ambiguity band of the parity checks (render(..., band=)): a pixel is flagged when one of its
# composite decisions lies this close to its threshold -- box edge (relative to sigma),
# alpha_min (absolute), stop on t_min (relative), in-front sign (relative to the range),
# alpha_max clamp (absolute) -- a few times the binary32 error of each decision quantity.
AMBIGUITY_BAND = (1e-5, 1e-6, 5e-5, 5e-7, 1e-6)


def pose_inverse(T_ws):
    R = np.zeros(9)
    t = np.zeros(3)
    T = _c(T_ws, np.float64)
    _load().or_pose_inverse(_ptr(T), _ptr(R), _ptr(t))
    return R.reshape(3, 3), t


def contract_atan2f(y, x) -> float:
    return float(_load().or_contract_atan2f(float(np.float32(y)), float(np.float32(x))))


def contract_expf(x) -> float:
    return float(_load().or_contract_expf(float(np.float32(x))))


def contract_logf(x) -> float:
    return float(_load().or_contract_logf(float(np.float32(x))))


def contract_reach_radius(o, alpha_min=1.0 / 255.0) -> float:
    """The binary32 contract's radius of the contributing region (splat units), with its margin."""
    return _load().or_contract_reach_radius(float(o), float(alpha_min))


def project_contract(pos_logit, quat, log_scale, T_ws, rows, cols, elev_min, elev_max,
                     tile_h=16, tile_w=16, sigma_cut=3.0, flip_normals=1, alpha_min=1.0 / 255.0):
    """Binary32 contract for one view: kappa, flip (+1/-1), pixel rect (r0, r1, c0, nc),
    tile rect (tr0, tr1, tc0, ntc), tile count, valid flag."""
    pl = _c(pos_logit, np.float32)
    q = _c(quat, np.float32)
    ls = _c(log_scale, np.float32)
    n = pl.shape[0]
    kappa = np.zeros(n, np.float32)
    flip = np.zeros(n, np.int8)
    pix = np.zeros((n, 4), np.int32)
    til = np.zeros((n, 4), np.int32)
    cnt = np.zeros(n, np.int32)
    valid = np.zeros(n, np.uint8)
    T = _c(T_ws, np.float64)
    _load().or_project_contract(n, _ptr(pl), _ptr(q), _ptr(ls), _ptr(T),
                                rows, cols, float(np.float32(elev_min)),
                                float(np.float32(elev_max)), tile_h, tile_w,
                                float(np.float32(sigma_cut)), float(np.float32(alpha_min)),
                                int(flip_normals),
                                _ptr(kappa), _ptr(flip), _ptr(pix), _ptr(til), _ptr(cnt),
                                _ptr(valid))
    return dict(kappa=kappa, flip=flip, pix_rect=pix, tile_rect=til, count=cnt, valid=valid)


def bin_pairs(proj, rows, cols, tile_h=16, tile_w=16, tile_offset=0):
    """Sorted (key, id) of every (tile, primitive) pair; key = (tile_offset + tile) << 32 |
    bits(kappa)."""
    cnt = proj["count"]
    m = int(cnt.astype(np.int64).sum())
    keys = np.zeros(max(m, 1), np.uint64)
    ids = np.zeros(max(m, 1), np.uint32)
    got = _load().or_bin(len(cnt), _ptr(proj["kappa"]), _ptr(proj["tile_rect"]), _ptr(cnt),
                         rows, cols, tile_h, tile_w, tile_offset, _ptr(keys), _ptr(ids), m)
    assert got == m
    return keys[:m], ids[:m]


def tile_ranges(keys, n_tiles, tile_offset=0):
    keys = _c(keys, np.uint64)
    start = np.zeros(n_tiles, np.int64)
    end = np.zeros(n_tiles, np.int64)
    _load().or_tile_ranges(len(keys), _ptr(keys), tile_offset, n_tiles, _ptr(start), _ptr(end))
    return start, end


def sort_order(kappa):
    kappa = _c(kappa, np.float32)
    order = np.zeros(len(kappa), np.int32)
    _load().or_sort_order(len(kappa), _ptr(kappa), _ptr(order))
    return order


def split_params(pos_logit, quat, log_scale):
    """FP32 parameter arrays -> exact FP64 copies (pos, logit, quat, log_scale)."""
    pl = np.asarray(pos_logit, np.float64)
    return (_c(pl[:, :3], np.float64), _c(pl[:, 3], np.float64), _c(quat, np.float64),
            _c(log_scale, np.float64))


class Culled:
    """Per-tile lists of one view (culled mode): start, end per tile, primitive ids."""

    def __init__(self, keys, ids, rows, cols, tile_h, tile_w):
        n_tiles = -(-rows // tile_h) * -(-cols // tile_w)
        self.start, self.end = tile_ranges(keys, n_tiles)
        self.ids = _c(ids, np.int32)
        self.tile_h, self.tile_w = tile_h, tile_w


def render(params, flip, order, T_ws, rows, cols, elev_min, elev_max, cfg=DEFAULT_CFG,
           band=None, culled: Culled | None = None, tile_h=16, tile_w=16, n_threads=0,
           pixels=None):
    """FP64 forward of one view.  params = (pos, logit, quat, log_scale) FP64 arrays;
    flip = int8 +-1 per primitive; order = brute-mode composite order (ignored if culled).
    pixels: optional (k,2) int array of (row, col) to render instead of the whole image.
    Returns dict D (H,W), N (3,H,W), O, T (final transmittance), n_contrib, band flags
    (shapes (k,), (3,k), ... when pixels is given)."""
    pos, logit, quat, ls = [_c(a, np.float64) for a in params]
    n = pos.shape[0]
    px = None if pixels is None else _c(pixels, np.int32).reshape(-1, 2)
    hw = rows * cols if px is None else len(px)
    D = np.zeros(hw)
    N = np.zeros(3 * hw)
    O = np.zeros(hw)
    T = np.zeros(hw)
    nc = np.zeros(hw, np.int32)
    bf = np.zeros(hw, np.uint8)
    order = _c(order if order is not None else np.arange(n), np.int32)
    cfg_a = np.asarray(cfg, np.float64)
    band_a = None if band is None else np.asarray(band, np.float64)
    if culled is not None:
        ts, te, ti, th, tw = culled.start, culled.end, culled.ids, culled.tile_h, culled.tile_w
    else:
        ts = te = ti = None
        th, tw = tile_h, tile_w
    flip_a = _c(flip, np.int8)
    Tw = _c(T_ws, np.float64)
    _load().or_render(n, _ptr(pos), _ptr(logit), _ptr(quat), _ptr(ls),
                      _ptr(flip_a), _ptr(order), len(order), _ptr(ts), _ptr(te),
                      _ptr(ti), _ptr(Tw), rows, cols,
                      float(elev_min), float(elev_max), th, tw, _ptr(cfg_a), _ptr(band_a),
                      _ptr(px), 0 if px is None else len(px),
                      _ptr(D), _ptr(N), _ptr(O), _ptr(T), _ptr(nc), _ptr(bf), n_threads)
    shp = (rows, cols) if px is None else (len(px),)
    return dict(D=D.reshape(shp), N=N.reshape((3,) + shp), O=O.reshape(shp), T=T.reshape(shp),
                n_contrib=nc.reshape(shp), band=bf.reshape(shp))


def render_backward(params, flip, order, T_ws, rows, cols, elev_min, elev_max, gD, gN, gO,
                    cfg=DEFAULT_CFG, culled: Culled | None = None, tile_h=16, tile_w=16,
                    n_threads=0, pixels=None):
    """FP64 analytic gradient of L = sum gD*D + gN.N + gO*O (over the given pixels, or all).
    Returns dict with g_pos (n,3), g_logit (n,), g_quat (n,4), g_log_scale (n,2),
    g_b (n,9) = (b_a, b_b, b_c) in the sensor frame, g_n (n,3), g_o (n,), and g_pose (6,) =
    (dL/drho, dL/domega) for the left perturbation T^c_w <- exp(xi^) T^c_w, xi = (rho, omega)."""
    px = None if pixels is None else _c(pixels, np.int32).reshape(-1, 2)
    pos, logit, quat, ls = [_c(a, np.float64) for a in params]
    n = pos.shape[0]
    out = dict(g_pos=np.zeros((n, 3)), g_logit=np.zeros(n), g_quat=np.zeros((n, 4)),
               g_log_scale=np.zeros((n, 2)), g_b=np.zeros((n, 9)), g_n=np.zeros((n, 3)),
               g_o=np.zeros(n))
    order = _c(order if order is not None else np.arange(n), np.int32)
    if culled is not None:
        ts, te, ti, th, tw = culled.start, culled.end, culled.ids, culled.tile_h, culled.tile_w
    else:
        ts = te = ti = None
        th, tw = tile_h, tile_w
    flip_a = _c(flip, np.int8)
    Tw = _c(T_ws, np.float64)
    cfg_a = _c(cfg, np.float64)
    gD_a = _c(gD, np.float64).ravel()
    gN_a = _c(gN, np.float64).ravel()
    gO_a = _c(gO, np.float64).ravel()
    _load().or_render_backward(
        n, _ptr(pos), _ptr(logit), _ptr(quat), _ptr(ls), _ptr(flip_a), _ptr(order),
        len(order), _ptr(ts), _ptr(te), _ptr(ti), _ptr(Tw), rows, cols,
        float(elev_min), float(elev_max), th, tw, _ptr(cfg_a),
        _ptr(px), 0 if px is None else len(px), _ptr(gD_a), _ptr(gN_a),
        _ptr(gO_a), _ptr(out["g_pos"]), _ptr(out["g_logit"]),
        _ptr(out["g_quat"]), _ptr(out["g_log_scale"]), _ptr(out["g_b"]), _ptr(out["g_n"]),
        _ptr(out["g_o"]), n_threads)
    out["g_pose"] = np.zeros(6)
    _load().or_pose_gradient(n, _ptr(pos), _ptr(logit), _ptr(quat), _ptr(ls), _ptr(flip_a),
                             _ptr(Tw), _ptr(out["g_b"]), _ptr(out["g_n"]), _ptr(out["g_pose"]))
    return out


def reach_pairs(params, T_ws, rows, cols, elev_min, elev_max, cfg=DEFAULT_CFG,
                cap=50_000_000):
    """Brute force: every (pixel index, primitive) whose ray reaches the primitive, without
    compositing (box test, hit in front, alpha >= alpha_min)."""
    pos, logit, quat, ls = [_c(a, np.float64) for a in params]
    n = pos.shape[0]
    pix = np.zeros(cap, np.int64)
    prim = np.zeros(cap, np.int32)
    Tw = _c(T_ws, np.float64)
    cfg_a = _c(cfg, np.float64)
    k = _load().or_reach_pairs(n, _ptr(pos), _ptr(logit), _ptr(quat), _ptr(ls), _ptr(Tw), rows,
                               cols, float(elev_min), float(elev_max), _ptr(cfg_a), _ptr(pix),
                               _ptr(prim), cap)
    assert k <= cap
    return pix[:k], prim[:k]


def loss(D, N, O, Dt, Nt, lambda_n=1.0, lambda_o=0.0, o_eps=1e-6, rho_exp=0.0):
    """(L, gD, gN, gO) over flattened pixels; N, Nt are (3, npx) planar.  The L1 range term is
    weighted by rho_d = Dt^rho_exp (rho_exp = 0: rho_d = 1)."""
    D = _c(D, np.float64).ravel()
    N = _c(N, np.float64).ravel()
    O = _c(O, np.float64).ravel()
    Dt = _c(Dt, np.float64).ravel()
    Nt = _c(Nt, np.float64).ravel()
    npx = D.size
    gD = np.zeros(npx)
    gN = np.zeros(3 * npx)
    gO = np.zeros(npx)
    L = _load().or_loss(npx, _ptr(D), _ptr(N), _ptr(O), _ptr(Dt), _ptr(Nt), lambda_n, lambda_o,
                        o_eps, float(rho_exp), _ptr(gD), _ptr(gN), _ptr(gO))
    return L, gD, gN.reshape(3, npx), gO


def adam(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-15, step=1):
    """In-place FP64 Adam on 1-D float64 arrays."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    _load().or_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), lr, b1, b2, eps, int(step))


def full_view(pos_logit, quat, log_scale, T_ws, rows, cols, elev_min, elev_max, *,
              cfg=DEFAULT_CFG, band=None, tile_h=16, tile_w=16, mode="culled", flip_normals=1,
              n_threads=0):
    """Convenience: contract + binning + FP64 render of one view from FP32 inputs."""
    proj = project_contract(pos_logit, quat, log_scale, T_ws, rows, cols, elev_min, elev_max,
                            tile_h, tile_w, cfg[3], flip_normals, cfg[0])
    params = split_params(pos_logit, quat, log_scale)
    emin, emax = float(np.float32(elev_min)), float(np.float32(elev_max))
    if mode == "culled":
        keys, ids = bin_pairs(proj, rows, cols, tile_h, tile_w)
        cul = Culled(keys, ids, rows, cols, tile_h, tile_w)
        out = render(params, proj["flip"], None, T_ws, rows, cols, emin, emax, cfg, band,
                     culled=cul, n_threads=n_threads)
        out["keys"], out["ids"], out["culled"] = keys, ids, cul
    else:
        order = sort_order(proj["kappa"])
        out = render(params, proj["flip"], order, T_ws, rows, cols, emin, emax, cfg, band,
                     tile_h=tile_h, tile_w=tile_w, n_threads=n_threads)
        out["order"] = order
    out["proj"], out["params"] = proj, params
    return out


def pixel_rays(rows, cols, elev_min, elev_max):
    """Unit ray of every pixel (rows, cols, 3), sensor frame, FP64: column c at azimuth
    pi - 2 pi (c + 1/2) / W, row r at elevation elev_max - r (elev_max - elev_min) / (H - 1)
    (elev_max for H = 1) -- the pixel centres of the spherical projection (Sec. 3.1)."""
    g = math.pi - 2.0 * math.pi * (np.arange(cols) + 0.5) / cols
    if rows > 1:
        th = elev_max - np.arange(rows) * (elev_max - elev_min) / (rows - 1)
    else:
        th = np.array([elev_max])
    ct, st = np.cos(th)[:, None], np.sin(th)[:, None]
    return np.stack([ct * np.cos(g)[None, :], ct * np.sin(g)[None, :],
                     np.broadcast_to(st, (rows, cols))], 2)


def backproject(D, O, T_ws, rows, cols, elev_min, elev_max, o_min):
    """Back-projection of a rendered range image to a world-frame point cloud (Sec. 3.3: the
    rasterised range image is back-projected at its pose, p = T_ws phi^-1(u, d)).  D is the
    unnormalised blended range, so the range of a pixel is d = D / O where O >= o_min (both in
    binary32, as rendered); other pixels give NaN.  Returns (3, rows * cols) FP64."""
    D = np.asarray(D, np.float32).reshape(rows, cols)
    O = np.asarray(O, np.float32).reshape(rows, cols)
    valid = O >= np.float32(o_min)
    d = np.where(valid, D.astype(np.float64) / np.where(valid, O, 1).astype(np.float64), np.nan)
    ps = pixel_rays(rows, cols, elev_min, elev_max) * d[..., None]
    T = np.asarray(T_ws, np.float64)
    pw = ps.reshape(-1, 3) @ T[:3, :3].T + T[:3, 3]
    return pw.T.copy()


# ---- keyframe sampling (Sec. 3.3, local model refinement) --------------------------------------

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_U32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
    as 1, 2, 3", SC 2011), written from its definition: a round maps (c0, c1, c2, c3) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)) and the key is bumped by the
    Weyl constants (W0, W1) between rounds.  Python integers, so no width tricks are involved."""
    c0, c1, c2, c3 = (int(x) & _U32 for x in ctr)
    k0, k1 = (int(x) & _U32 for x in key)
    for r in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & _U32, p1 & _U32, ((p0 >> 32) ^ c3 ^ k1) & _U32, \
            p0 & _U32
        if r < 9:
            k0 = (k0 + _PHILOX_W0) & _U32
            k1 = (k1 + _PHILOX_W1) & _U32
    return c0, c1, c2, c3


def view_sampling_thresholds(n_views, p_newest):
    """Integer thresholds of the truncated geometric distribution over keyframe age a
    (a = 0 the newest): P(a) = p (1 - p)^a / Z over a < n_views, so P(newest) = p / Z >= p.
    t_a = floor(C_a 2^32) for the cumulative C_a, a < n_views - 1; FP64 with the products and
    sums taken in age order."""
    q = 1.0 - p_newest
    P = []
    w = p_newest
    for _ in range(n_views):
        P.append(w)
        w = w * q
    Z = 0.0
    for x in P:
        Z = Z + x
    thr = []
    c = 0.0
    for a in range(n_views - 1):
        c = c + P[a]
        thr.append(min(int(math.floor((c / Z) * 4294967296.0)), _U32))
    return thr


def sample_active_views(n_views, draws, p_newest, seed, step):
    """Views drawn for refinement step `step`: draw j in [0, draws) takes the first word x of
    Philox((j, step, 0, 0), (seed lo, seed hi)), its age is the number of thresholds <= x, and
    the view is n_views - 1 - age (the last registered view is the newest).  Returns the active
    flags (a view drawn at least once)."""
    thr = view_sampling_thresholds(n_views, p_newest)
    act = np.zeros(n_views, bool)
    for j in range(draws):
        x = philox4x32_10((j, step, 0, 0), (seed & _U32, (seed >> 32) & _U32))[0]
        age = sum(1 for t in thr if x >= t)
        act[n_views - 1 - age] = True
    return act


def scale_regularizer(log_scale, lambda_s, tau_s):
    """Scale term of the mapping loss (Eq. L_s, its sign read as a penalty on growth beyond
    tau_s): lambda_s sum_i max(0, max(s_a, s_b)_i - tau_s), s = exp(log s), and its gradient with
    respect to log s (s of the larger axis, the first one on a tie).  FP64."""
    ls = np.asarray(log_scale, np.float64).reshape(-1, 2)
    s = np.exp(ls)
    first = s[:, 0] >= s[:, 1]
    sm = np.where(first, s[:, 0], s[:, 1])
    on = sm > tau_s
    value = lambda_s * float(np.sum(np.where(on, sm - tau_s, 0.0)))
    g = np.zeros_like(ls)
    g[:, 0] = np.where(on & first, lambda_s * s[:, 0], 0.0)
    g[:, 1] = np.where(on & ~first, lambda_s * s[:, 1], 0.0)
    return value, g


def range_normal_loss(D, N, Dt, rows, cols, elev_min, elev_max, lambda_n=1.0):
    """Self-regularised normal term of the mapping loss (Eq. loss_normal): the rendered normal N is
    compared with the normal of the rendered range map, N(D) (Sec. 3.3, after 2DGS).  Reading:
    for pixel u = (r, c) with r + 1 < H, x = (r, c + 1 mod W) and y = (r + 1, c) (the azimuth
    wraps), P(w) = D(w) v(w) with v the pixel-centre ray, m = (P(x) - P(u)) x (P(y) - P(u)),
    n_D = -sign(m . v(u)) m / |m| (facing the sensor); the term lambda_n (1 - N(u) . n_D) counts
    where the targets of u, x and y are valid (Dt > 0), their rendered ranges are positive (a
    zero range puts P at the sensor, where m . v(u) vanishes and the side is undefined) and
    m != 0.  D and N are used as rendered
    (unnormalised blends).  Returns (value, dL/dD (H, W), dL/dN (3, H, W)), FP64; the sign
    is held fixed in the gradient."""
    D = np.asarray(D, np.float64).reshape(rows, cols)
    N = np.asarray(N, np.float64).reshape(3, rows, cols)
    Dt = np.asarray(Dt, np.float64).reshape(rows, cols)
    V = pixel_rays(rows, cols, elev_min, elev_max)
    P = V * D[..., None]
    gD = np.zeros((rows, cols))
    gP = np.zeros((rows, cols, 3))
    gN = np.zeros((3, rows, cols))
    value = 0.0
    for r in range(rows - 1):
        for c in range(cols):
            cx = (c + 1) % cols
            if not (Dt[r, c] > 0 and Dt[r, cx] > 0 and Dt[r + 1, c] > 0):
                continue
            if not (D[r, c] > 0 and D[r, cx] > 0 and D[r + 1, c] > 0):
                continue
            dx = P[r, cx] - P[r, c]
            dy = P[r + 1, c] - P[r, c]
            m = np.cross(dx, dy)
            mn = np.linalg.norm(m)
            if mn == 0.0:
                continue
            s = -1.0 if np.dot(m, V[r, c]) > 0 else 1.0
            nd = s * m / mn
            n = N[:, r, c]
            value += lambda_n * (1.0 - np.dot(n, nd))
            gN[:, r, c] += -lambda_n * nd
            g = -lambda_n * n                                  # dL/dn_D
            gm = s * (g - (m / mn) * np.dot(m / mn, g)) / mn     # dL/dm
            gdx = np.cross(dy, gm)
            gdy = np.cross(gm, dx)
            gP[r, cx] += gdx
            gP[r + 1, c] += gdy
            gP[r, c] -= gdx + gdy
    gD = np.einsum("hwk,hwk->hw", gP, V)
    return value, gD, gN


# ---- map growth: densification masks and range-gradient-weighted sampling (Sec. 3.3.1-3.3.2) ----

DENSIFY_QUANT = 256.0        # weights are counted in 1/256 m
DENSIFY_EMPTY_LOGIT = -30.0  # opacity logit of a slot no pixel took (below alpha_min)


def densify_weights(Dt, D, O, rows, cols, refine, lambda_do, lambda_de, w0, w_cap):
    """Integer sampling weights q(u) of one view (rows x cols), binary32 arithmetic.
    Mask: M_v = Dt > 0 (Sec. 3.3.1); in refinement also M_n or M_e (Sec. 3.3.2), M_n = O <=
    lambda_do, M_e = |D - Dt| >= lambda_de.  Weight from the range gradients of the target:
    g_x = Dt(r, c + 1 mod W) - Dt(r, c), g_y = Dt(r + 1, c) - Dt(r, c) (0 where a neighbour is
    missing or invalid), w = min((w0 + |g_x|) + |g_y|, w_cap), q = floor(256 w) on the mask, else 0."""
    f = np.float32
    Dt = np.asarray(Dt, f).reshape(rows, cols)
    valid = Dt > 0
    m = valid.copy()
    if refine:
        D = np.asarray(D, f).reshape(rows, cols)
        O = np.asarray(O, f).reshape(rows, cols)
        m &= (O <= f(lambda_do)) | (np.abs(D - Dt) >= f(lambda_de))
    right = np.roll(Dt, -1, 1)
    gx = np.where(valid & np.roll(valid, -1, 1), right - Dt, f(0))
    gy = np.zeros_like(Dt)
    gy[:-1] = np.where(valid[:-1] & valid[1:], Dt[1:] - Dt[:-1], f(0))
    w = np.minimum((f(w0) + np.abs(gx)) + np.abs(gy), f(w_cap))
    q = np.floor(w * f(DENSIFY_QUANT)).astype(np.uint64)
    return np.where(m, q, 0).astype(np.uint64).ravel()


def densify_offset(Q, seed, call):
    """The systematic-sampling offset o in [0, Q): x = first word of Philox((0, call, 2, 0),
    (seed lo, seed hi)), o = floor(x Q / 2^32)."""
    x = philox4x32_10((0, call, 2, 0), (seed & _U32, (seed >> 32) & _U32))[0]
    return (x * int(Q)) >> 32


def systematic_counts(q, n_d, o):
    """Systematic (low-variance) weighted sampling of n_d points: with Q = sum q and the
    exclusive prefix C, sample j sits at s_j = floor((j Q + o) / n_d) and pixel i takes the
    samples with C_i <= s_j < C_i + q_i.  Returns (count per pixel, first sample index per pixel)
    from the closed form #{j : s_j < X} = clamp(ceil((X n_d - o) / Q), 0, n_d).  Python integers."""
    q = [int(x) for x in q]
    Q = sum(q)
    cnt = []
    first = []
    C = 0

    def below(X):
        t = X * n_d - o
        return 0 if t <= 0 else min(n_d, -(-t // Q))

    for qi in q:
        a, b = below(C), below(C + qi)
        first.append(a)
        cnt.append(b - a)
        C += qi
    return np.array(cnt, np.int64), np.array(first, np.int64)


def init_primitive(d, v_s, T_ws, dgamma, dtheta, scale_k, opacity):
    """A new primitive from a sampled pixel (Sec. 3.3.1): centre T_ws (d v), normal towards the
    sensor, t_n = -R_ws v, as the rotation of shortest arc from e_z (quaternion (w, x, y, z) =
    (1 + n_z, -n_y, n_x, 0) normalised; (0, 1, 0, 0) when 1 + n_z < 1e-6), isotropic scale
    scale_k d sqrt(dgamma dtheta), the given opacity.  Returns (pos_logit[4], quat[4],
    log_scale[2]), FP64."""
    T = np.asarray(T_ws, np.float64)
    v = np.asarray(v_s, np.float64)
    mu = T[:3, :3] @ (d * v) + T[:3, 3]
    n = -(T[:3, :3] @ v)
    n = n / np.linalg.norm(n)
    if 1.0 + n[2] < 1e-6:
        q = np.array([0.0, 1.0, 0.0, 0.0])
    else:
        q = np.array([1.0 + n[2], -n[1], n[0], 0.0])
        q /= np.linalg.norm(q)
    s = scale_k * d * math.sqrt(dgamma * dtheta)
    return (np.array([*mu, math.log(opacity / (1.0 - opacity))]), q,
            np.array([math.log(s), math.log(s)]))


def densify(views, Dt, D, O, n_d, refine=False, lambda_do=0.5, lambda_de=0.1, w0=0.05,
            w_cap=2.0, scale_k=2.0, opacity=0.5, seed=0, call=0):
    """Map growth over the packed pixels of several views (each (T_ws, rows, cols, elev_min,
    elev_max)): weights per view (densify_weights), one systematic draw of n_d samples over all
    packed pixels, and a new primitive per slot.  A pixel drawn k >= 1 times fills the first of
    its k slots; the other slots (all of them when no pixel is masked) are empty primitives
    (centre 0, opacity logit -30, identity rotation, log-scales 0).  Returns (pos_logit (n_d, 4),
    quat (n_d, 4), log_scale (n_d, 2), pixel of each slot (-1 for an empty slot))."""
    qs, geo = [], []
    off = 0
    for (T, rows, cols, emin, emax) in views:
        P = rows * cols
        sl = slice(off, off + P)
        qs.append(densify_weights(Dt[sl], None if D is None else D[sl],
                                  None if O is None else O[sl], rows, cols, refine, lambda_do,
                                  lambda_de, w0, w_cap))
        geo.append((T, rows, cols, emin, emax, off))
        off += P
    q = np.concatenate(qs)
    pl = np.zeros((n_d, 4))
    pl[:, 3] = DENSIFY_EMPTY_LOGIT
    qt = np.zeros((n_d, 4))
    qt[:, 0] = 1.0
    ls = np.zeros((n_d, 2))
    pix = np.full(n_d, -1, np.int64)
    Q = int(q.sum())
    if Q == 0 or n_d == 0:
        return pl, qt, ls, pix
    o = densify_offset(Q, seed, call)
    cnt, first = systematic_counts(q, n_d, o)
    Dt64 = np.asarray(Dt, np.float32).astype(np.float64)
    for (T, rows, cols, emin, emax, base) in geo:
        V = pixel_rays(rows, cols, emin, emax).reshape(-1, 3)
        dg = 2.0 * math.pi / cols
        dt = (emax - emin) / (rows - 1) if rows > 1 else dg
        for k in np.nonzero(cnt[base:base + rows * cols])[0]:
            j = int(first[base + k])
            pl[j], qt[j], ls[j] = init_primitive(Dt64[base + k], V[k], T, dg, dt, scale_k,
                                                 opacity)
            pix[j] = base + k
    return pl, qt, ls, pix


# ---- photometric registration residual (Sec. 3.3.3, Eq. L_photo) ---------------------------------

def _se3_right_jacobian_point(R, p):
    """d(R exp(xi^) p + t)/d xi at xi = 0 for xi = (rho, omega): R [I, -[p]x]  (3 x 6)."""
    px = np.array([[0.0, -p[2], p[1]], [p[2], 0.0, -p[0]], [-p[1], p[0], 0.0]])
    return R @ np.hstack([np.eye(3), -px])


def photometric_normal_eqs(D, O, Dq, T_qm, rows, cols, elev_min, elev_max, o_min, huber_delta,
                           band_px=None, band_r=None):
    """Photometric residual of the rendered range image against a query range image of the same
    sensor model, and its Gauss-Newton normal equations in the pose (Sec. 3.3.3, Eq. L_photo).
    Reading: pixel u of the render with O(u) >= o_min has range d = D / O and point p = d v(u);
    p' = T_qm p (render frame -> query frame); u' = phi(p') has the continuous column
    c' = (pi - atan2(y', x')) / dgamma - 1/2 and row r' = (elev_max - atan2(z', |x'y'|)) /
    dtheta; Dq is sampled bilinearly at u' (columns wrap; the four pixels must exist and have
    Dq > 0); the residual is r = |p'| - Dq(u') (at T_qm = I it is d(u) - Dq(u)).  The pose is
    perturbed on the right, T_qm exp(xi^), xi = (rho, omega); J = dr/dxi.  Huber weights
    w = min(1, delta / |r|) (IRLS), cost rho_H(r).  Returns a dict: H = sum w J J^T (6 x 6),
    g = sum w J r, cost, count, and per pixel r, w, J (P x 6), used (bool).  FP64.

    Ambiguity band (test infrastructure: the pixels on which a binary32 evaluation of the same
    residual may legitimately disagree), when band_px is given: band[i] is set for a pixel with
    O >= o_min whose u' lies within band_px of a cell edge in rows or columns (the floor of u'
    picks the bilinear cell, the validity of its four pixels and the slopes that enter J), or
    whose bilinear slopes move the sample by more than band_r when u' moves by band_px
    ((|dS/dc'| + |dS/dr'|) band_px > band_r)."""
    D = np.asarray(D, np.float64).ravel()
    O = np.asarray(O, np.float64).ravel()
    Dq = np.asarray(Dq, np.float64).reshape(rows, cols)
    T = np.asarray(T_qm, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    V = pixel_rays(rows, cols, elev_min, elev_max).reshape(-1, 3)
    dg = 2.0 * math.pi / cols
    dth = (elev_max - elev_min) / (rows - 1) if rows > 1 else dg
    P = rows * cols
    res = np.zeros(P)
    wts = np.zeros(P)
    J = np.zeros((P, 6))
    used = np.zeros(P, bool)
    band = np.zeros(P, bool)
    H = np.zeros((6, 6))
    g = np.zeros(6)
    cost = 0.0
    for i in range(P):
        if not (O[i] >= o_min):
            continue
        d = D[i] / O[i]
        p = d * V[i]
        q = R @ p + t
        x, y, z = q
        rxy2 = x * x + y * y
        rho = math.sqrt(rxy2 + z * z)
        if rxy2 == 0.0:
            continue
        rxy = math.sqrt(rxy2)
        cp = (math.pi - math.atan2(y, x)) / dg - 0.5
        rp = (elev_max - math.atan2(z, rxy)) / dth if rows > 1 else 0.0
        r0 = math.floor(rp)
        c0 = math.floor(cp)
        fr, fc = rp - r0, cp - c0
        if band_px is not None and ((rows > 1 and min(fr, 1.0 - fr) <= band_px)
                                    or min(fc, 1.0 - fc) <= band_px):
            band[i] = True
        if r0 < 0 or r0 + 1 >= rows:
            continue
        ca, cb = c0 % cols, (c0 + 1) % cols
        q00, q01, q10, q11 = Dq[r0, ca], Dq[r0, cb], Dq[r0 + 1, ca], Dq[r0 + 1, cb]
        if not (q00 > 0 and q01 > 0 and q10 > 0 and q11 > 0):
            continue
        sample = (1 - fr) * ((1 - fc) * q00 + fc * q01) + fr * ((1 - fc) * q10 + fc * q11)
        dS_dc = (1 - fr) * (q01 - q00) + fr * (q11 - q10)
        dS_dr = (1 - fc) * (q10 - q00) + fc * (q11 - q01)
        if band_px is not None and (abs(dS_dc) + abs(dS_dr)) * band_px > band_r:
            band[i] = True
        dc_dq = np.array([y, -x, 0.0]) / (dg * rxy2)
        dth_dq = np.array([-z * x / (rxy * rho * rho), -z * y / (rxy * rho * rho), rxy / (rho * rho)])
        dr_dq = -dth_dq / dth
        dres_dq = q / rho - (dS_dc * dc_dq + dS_dr * dr_dq)
        Ji = dres_dq @ _se3_right_jacobian_point(R, p)
        r = rho - sample
        a = abs(r)
        w = 1.0 if a <= huber_delta else huber_delta / a
        cost += 0.5 * r * r if a <= huber_delta else huber_delta * (a - 0.5 * huber_delta)
        H += w * np.outer(Ji, Ji)
        g += w * Ji * r
        res[i], wts[i], J[i], used[i] = r, w, Ji, True
    return {"H": H, "g": g, "cost": cost, "count": int(used.sum()), "r": res, "w": wts, "J": J,
            "used": used, "band": band}
