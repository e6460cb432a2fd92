"""Pins of the oracle's binary32 binning contract (Sec. 3.2.1 tiles and range sort, Sec. 3.2.3
bounding box; Supp. B).

* the series used for atan2 and exp stay within their error bounds;
* brute force: every (pixel, primitive) pair whose ray reaches the primitive (box test, in front,
  alpha >= alpha_min) lies in the primitive's pixel rectangle and in one of its tiles;
* hand-built cases: the +-pi seam behind the sensor, a splat over the pole, the sensor inside
  the 3-sigma box, an edge-on splat;
* the sorted key list is consistent: sorted by (tile, kappa bits, id), each primitive listed once
  per touched tile, tile ranges partition the list.
"""
import math

import numpy as np
import pytest

from paper_2503_17491_gb300 import scenes


def test_contract_atan2_bound(oracle_mod):
    rng = np.random.default_rng(0)
    ys = np.concatenate([rng.normal(size=4000) * 10 ** rng.uniform(-3, 3, 4000),
                         [0, 0, 1, -1, 1e-30, -1e-30, 3, -3]]).astype(np.float32)
    xs = np.concatenate([rng.normal(size=4000) * 10 ** rng.uniform(-3, 3, 4000),
                         [1, -1, 0, 0, -1, -1, 3, 3]]).astype(np.float32)
    worst = 0.0
    for y, x in zip(ys, xs):
        if x == 0 and y == 0:
            continue
        worst = max(worst, abs(oracle_mod.contract_atan2f(y, x) - math.atan2(float(y), float(x))))
    assert worst < 4e-7
    assert oracle_mod.contract_atan2f(0.0, 1.0) == 0.0
    assert oracle_mod.contract_atan2f(1.0, 0.0) == float(np.float32(math.pi / 2))
    assert oracle_mod.contract_atan2f(0.0, -1.0) == float(np.float32(math.pi))
    assert oracle_mod.contract_atan2f(-1e-30, -1.0) == -float(np.float32(math.pi))


def test_contract_exp_bound(oracle_mod):
    xs = np.linspace(-20, 10, 30001).astype(np.float32)
    rel = max(abs(oracle_mod.contract_expf(x) / math.exp(float(x)) - 1) for x in xs[::7])
    assert rel < 2e-7
    assert oracle_mod.contract_expf(0.0) == 1.0
    assert oracle_mod.contract_expf(1.0) == pytest.approx(math.e, rel=2e-7)


def test_contract_log_bound(oracle_mod):
    xs = np.exp(np.linspace(0.0, np.log(1e6), 20001)).astype(np.float32)
    # within a few float ulps of ln x (the series truncation is ~1e-9 at |z| <= 0.172)
    worst = max(abs(oracle_mod.contract_logf(x) - math.log(float(x))) / max(1.0, math.log(float(x)))
                for x in xs[::7])
    assert worst < 1.2e-7
    assert oracle_mod.contract_logf(1.0) == 0.0
    assert oracle_mod.contract_logf(2.0) == pytest.approx(math.log(2.0), abs=3e-7)


def test_low_opacity_primitive_reaches_nothing(oracle_mod):
    """A primitive whose opacity is below alpha_min can never contribute: no tiles."""
    pl, q, ls = _single((5.0, 0.0, 0.0), (0.5, 0.5, 0.5, 0.5), (0.3, 0.3), o=0.003)
    v = scenes.View(np.eye(4), 32, 512, scenes.deg(-15), scenes.deg(15))
    proj = oracle_mod.project_contract(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
    assert proj["count"][0] == 0


def test_pose_inverse(oracle_mod):
    T = scenes.random_pose(np.random.default_rng(1), 5.0, 40.0)
    R, t = oracle_mod.pose_inverse(T)
    Ti = np.eye(4)
    Ti[:3, :3], Ti[:3, 3] = R, t
    np.testing.assert_allclose(Ti @ T, np.eye(4), atol=1e-14)


def _in_cyclic(x, start, count, period):
    return ((x - start) % period) < count


def _check_coverage(oracle_mod, pl, q, ls, v, th=16, tw=16, min_pairs=1):
    proj = oracle_mod.project_contract(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min,
                                       v.elev_max, th, tw)
    params = oracle_mod.split_params(pl, q, ls)
    pix, prim = oracle_mod.reach_pairs(params, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
    assert len(pix) >= min_pairs
    r, c = pix // v.cols, pix % v.cols
    pr = proj["pix_rect"][prim]
    tr = proj["tile_rect"][prim]
    TC = -(-v.cols // tw)
    assert np.all(proj["count"][prim] > 0)
    assert np.all((r >= pr[:, 0]) & (r <= pr[:, 1]))
    assert np.all(_in_cyclic(c, pr[:, 2], pr[:, 3], v.cols))
    assert np.all((r // th >= tr[:, 0]) & (r // th <= tr[:, 1]))
    assert np.all(_in_cyclic(c // tw, tr[:, 2], tr[:, 3], TC))
    return proj, pix, prim


def test_coverage_workload0(oracle_mod):
    s = scenes.workload(0)
    v = s.views[0]
    proj, pix, prim = _check_coverage(oracle_mod, s.pos_logit, s.quat, s.log_scale, v,
                                      min_pairs=1000)
    # and the box is not wildly loose: the pixel rectangles hold at most ~6x the reached pixels
    area = (proj["pix_rect"][:, 1] - proj["pix_rect"][:, 0] + 1) * proj["pix_rect"][:, 3]
    area = np.where(proj["count"] > 0, area, 0).sum()
    assert area < 6 * len(pix)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8), (4, 64)])
def test_coverage_tiny_random(oracle_mod, seed, tile):
    s = scenes.tiny_scene(60, seed, rows=24, cols=200, fov_deg=35, dist=(0.6, 9.0),
                          spread=2.0, log_scale=(-3.0, -0.5))
    s.views[0].T_ws = scenes.random_pose(np.random.default_rng(seed + 10), 0.2, 30.0)
    _check_coverage(oracle_mod, s.pos_logit, s.quat, s.log_scale, s.views[0], *tile,
                    min_pairs=50)


def _single(mu, normal_q, s, o=0.9):
    pl = np.array([[*mu, math.log(o / (1 - o))]], np.float32)
    q = np.array([normal_q], np.float32)
    ls = np.array([[math.log(s[0]), math.log(s[1])]], np.float32)
    return pl, q, ls


def test_seam_behind_sensor(oracle_mod):
    """A splat straddling azimuth +-pi (behind the sensor): its columns wrap from W-1 to 0."""
    v = scenes.View(np.eye(4), 32, 512, scenes.deg(-15), scenes.deg(15))
    # at x = -4 facing the sensor: t_a = y, t_b = z, t_n = x (quaternion of 120 deg about 1,1,1)
    pl, q, ls = _single((-4.0, 0.05, 0.0), (0.5, 0.5, 0.5, 0.5), (0.3, 0.3))
    proj, pix, prim = _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=20)
    c = pix % v.cols
    assert c.min() == 0 and c.max() == v.cols - 1       # both image edges are reached
    c0, nc = proj["pix_rect"][0, 2], proj["pix_rect"][0, 3]
    assert c0 + nc > v.cols                              # the rectangle wraps
    assert proj["tile_rect"][0, 2] + proj["tile_rect"][0, 3] > v.cols // 16
    out = oracle_mod.full_view(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
    ref = oracle_mod.full_view(pl, q, ls, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max,
                               mode="brute")
    np.testing.assert_array_equal(out["D"], ref["D"])


def test_splat_over_the_pole(oracle_mod):
    """A horizontal splat above the sensor covers every azimuth of the top rows."""
    v = scenes.View(np.eye(4), 48, 256, scenes.deg(-80), scenes.deg(80))
    pl, q, ls = _single((0.3, -0.2, 2.0), (1.0, 0.0, 0.0, 0.0), (0.37, 0.3))
    proj, pix, prim = _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=100)
    assert proj["pix_rect"][0, 3] == v.cols and proj["pix_rect"][0, 0] == 0
    assert len(np.unique(pix % v.cols)) == v.cols


def test_sensor_inside_box(oracle_mod):
    """The sensor 0.1 m off the plane with its foot inside the 3-sigma box.  A vertical plane:
    the reached columns span nearly 180 degrees and stay inside the box.  A horizontal plane
    just below the sensor: every column."""
    v = scenes.View(np.eye(4), 32, 256, scenes.deg(-40), scenes.deg(40))
    pl, q, ls = _single((0.1, 0.2, -0.1), (0.5, 0.5, 0.5, 0.5), (0.35, 0.35))
    proj, pix, prim = _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=100)
    assert len(np.unique(pix % v.cols)) > 100
    pl, q, ls = _single((0.05, -0.1, -0.1), (1.0, 0.0, 0.0, 0.0), (0.35, 0.35))
    proj, pix, prim = _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=100)
    assert proj["pix_rect"][0, 3] == v.cols
    assert len(np.unique(pix % v.cols)) == v.cols


def test_edge_on_splat(oracle_mod):
    """A splat whose plane nearly contains the sensor: reached pixels form a thin sliver and
    stay inside the box."""
    v = scenes.View(np.eye(4), 64, 1024, scenes.deg(-20), scenes.deg(20))
    # plane y = 0.05 (normal +y): t_a = x, t_b = z -> rotation of -90 deg about x;
    # rays at azimuth 0.47-0.73 deg graze it (one column of a 1024-wide image)
    c, s_ = math.cos(-math.pi / 4), math.sin(-math.pi / 4)
    pl, q, ls = _single((5.0, 0.05, 0.0), (c, s_, 0.0, 0.0), (0.37, 0.37))
    _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=1)


def test_sorted_keys_and_ranges(oracle_mod):
    s = scenes.workload(0)
    v = s.views[0]
    th, tw = 16, 16
    proj = oracle_mod.project_contract(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                                       v.elev_min, v.elev_max, th, tw)
    keys, ids = oracle_mod.bin_pairs(proj, v.rows, v.cols, th, tw)
    assert len(keys) == proj["count"].sum()
    # sorted by (key, id); key = tile << 32 | bits(kappa)
    k2 = keys.astype(object) * (1 << 32) + ids.astype(object)
    assert all(k2[i] < k2[i + 1] for i in range(len(k2) - 1))
    np.testing.assert_array_equal((keys & 0xFFFFFFFF).astype(np.uint32),
                                  proj["kappa"][ids].view(np.uint32))
    # each primitive appears exactly once per tile of its rectangle
    TC = -(-v.cols // tw)
    tiles = (keys >> 32).astype(np.int64)
    for i in np.unique(ids)[:200]:
        t = np.sort(tiles[ids == i])
        tr = proj["tile_rect"][i]
        want = sorted(rr * TC + (tr[2] + k) % TC for rr in range(tr[0], tr[1] + 1)
                      for k in range(tr[3]))
        np.testing.assert_array_equal(t, want)
    n_tiles = -(-v.rows // th) * TC
    start, end = oracle_mod.tile_ranges(keys, n_tiles)
    nonempty = end > start
    assert (end - start)[nonempty].sum() == len(keys)
    assert np.all(tiles[start[nonempty]] == np.nonzero(nonempty)[0])


@pytest.mark.parametrize("o,bound", [(2.0 / 255.0, "reach"), (0.9, "box")])
def test_bbox_is_clipped_to_the_contributing_region(oracle_mod, o, bound):
    """A head-on splat at 5 m (t_a = y, t_b = z, 0.3 m scales): its columns span the angle where
    it can contribute, |s| <= a with a = min(sigma, r_o), r_o = sqrt(2 ln(o / alpha_min)) -- for
    o = 2 alpha_min that is r_o = 1.18 of the 3-sigma box, not the box (closed form, with the
    contract's small margins)."""
    v = scenes.View(np.eye(4), 33, 512, scenes.deg(-16), scenes.deg(16))
    d, s = 5.0, 0.3
    pl, q, ls = _single((d, 0.0, 0.0), (0.5, 0.5, 0.5, 0.5), (s, s), o=o)
    proj, pix, prim = _check_coverage(oracle_mod, pl, q, ls, v, min_pairs=10)
    a = min(3.0, math.sqrt(2.0 * math.log(o * 255.0))) if bound == "reach" else 3.0
    dg = 2 * math.pi / v.cols
    half = math.atan(a * s / d) / dg               # columns each side of the centre
    nc = int(proj["pix_rect"][0][3])
    assert 2 * half - 1 <= nc <= 2 * half * 1.003 + 3, (nc, half)


# ---- tightness against the exact FP64 footprint of the contributing region -------------------
#
# The binary32 contract bounds the part of the splat plane where a primitive can contribute
# (Sec. 3.2.3 reading: the 3-sigma square cut by o G(s) >= alpha_min, the disk |s| <= r_o).  The
# pins below compute that region's angular footprint independently, in FP64 from the parameters
# (quaternion -> axes, scales, sensor frame, densely sampled region boundary, exact corners), and
# bound the contract's pixel rectangle from both sides: it holds every pixel centre of the
# footprint, and it exceeds the footprint by at most one pixel of rounding beyond TIGHT_FRAC of
# the footprint's half-width.  The contract's polygon circumscribes the region with edges at most
# 1/cos(pi/8) - 1 = 8.2 % of its radius outside it (a regular octagon around a disk is the worst
# case), hence TIGHT_FRAC = 0.1.  Primitives whose region holds a pole ray, spans a quarter turn
# of azimuth or lies in a plane through the sensor are left to the hand-built cases above.

TIGHT_FRAC = 0.1


def _quat_axes(q):
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    ta = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    tb = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    return ta, tb


def _footprint(pl, q, ls, view, sigma=3.0, amin=1.0 / 255.0, K=2048):
    """Continuous pixel extent [r_lo, r_hi] x [c_lo, c_hi] of each primitive's contributing
    region seen from the view (FP64), and a mask of the primitives it is defined for."""
    pl, q, ls = (np.asarray(a, np.float64) for a in (pl, q, ls))
    Rws, tws = view.T_ws[:3, :3], view.T_ws[:3, 3]
    Rcw, tcw = Rws.T, -Rws.T @ tws
    ta, tb = _quat_axes(q)
    s = np.exp(ls)
    o = 1.0 / (1.0 + np.exp(-pl[:, 3]))
    ba = s[:, :1] * (ta @ Rcw.T)
    bb = s[:, 1:] * (tb @ Rcw.T)
    bc = pl[:, :3] @ Rcw.T + tcw
    ok = o > amin
    ro = np.sqrt(2.0 * np.log(np.maximum(o / amin, 1.0)))
    a = np.minimum(ro, sigma)
    # boundary of {|s|_inf <= a} n {|s| <= ro}: K directions plus the exact corners
    t = np.linspace(0.0, 2.0 * np.pi, K, endpoint=False)
    U = np.stack([np.cos(t), np.sin(t)], 1)
    out = {k: np.zeros(len(o)) for k in ("r_lo", "r_hi", "c_lo", "c_hi", "span")}
    for i0 in range(0, len(o), 256):
        sl = slice(i0, i0 + 256)
        rad = np.minimum(ro[sl, None], a[sl, None] / np.abs(U).max(1)[None])
        S = rad[..., None] * U[None]                                   # (m, K, 2)
        h = np.sqrt(np.maximum(ro[sl] ** 2 - a[sl] ** 2, 0.0))
        h = np.minimum(h, a[sl])
        corners = np.stack([np.stack([sa * a[sl], sb * h], 1) for sa in (-1, 1) for sb in (-1, 1)] +
                           [np.stack([sb * h, sa * a[sl]], 1) for sa in (-1, 1) for sb in (-1, 1)], 1)
        S = np.concatenate([S, corners], 1)
        X = bc[sl, None] + S[..., :1] * ba[sl, None] + S[..., 1:] * bb[sl, None]
        gam = np.arctan2(X[..., 1], X[..., 0])
        th = np.arctan2(X[..., 2], np.hypot(X[..., 0], X[..., 1]))
        gc = np.arctan2(bc[sl, 1], bc[sl, 0])
        d = (gam - gc[:, None] + np.pi) % (2.0 * np.pi) - np.pi
        dg = 2.0 * np.pi / view.cols
        dth = (view.elev_max - view.elev_min) / (view.rows - 1)
        out["c_lo"][sl] = (np.pi - (gc + d.max(1))) / dg - 0.5
        out["c_hi"][sl] = (np.pi - (gc + d.min(1))) / dg - 0.5
        out["r_lo"][sl] = (view.elev_max - th.max(1)) / dth
        out["r_hi"][sl] = (view.elev_max - th.min(1)) / dth
        out["span"][sl] = d.max(1) - d.min(1)
    # the z axis through the region (pole), a plane through the sensor
    det = ba[:, 0] * bb[:, 1] - ba[:, 1] * bb[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = -(bc[:, 0] * bb[:, 1] - bc[:, 1] * bb[:, 0]) / det
        v = -(ba[:, 0] * bc[:, 1] - ba[:, 1] * bc[:, 0]) / det
    pole = (np.abs(u) <= a * 1.01) & (np.abs(v) <= a * 1.01) & (u * u + v * v <= (1.01 * ro) ** 2)
    nrm = np.cross(ba, bb)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    through = np.abs(np.sum(nrm * bc, 1)) < 1e-3
    out["good"] = ok & ~pole & ~through & np.isfinite(det) & (out["span"] < np.pi / 2)
    return out


def _rect_excess(oracle_mod, pl, q, ls, view, th=16, tw=16):
    """Per selected primitive and edge (top, bottom, left, right): how far the contract's pixel
    rectangle reaches beyond the exact footprint (pixels, > -1 means every pixel centre of the
    footprint is inside), and the footprint's half-width along that axis."""
    proj = oracle_mod.project_contract(pl, q, ls, view.T_ws, view.rows, view.cols,
                                       view.elev_min, view.elev_max, th, tw)
    fp = _footprint(pl, q, ls, view)
    rect = proj["pix_rect"].astype(np.float64)
    H, W = view.rows, view.cols
    inside_rows = (fp["r_lo"] > 0) & (fp["r_hi"] < H - 1)    # no clipping at the image edge
    has_px = (np.ceil(fp["r_lo"]) <= np.floor(fp["r_hi"])) & \
             (np.ceil(fp["c_lo"]) <= np.floor(fp["c_hi"]))
    sel = fp["good"] & inside_rows & has_px
    assert np.all(proj["count"][sel] > 0)
    c0 = rect[:, 2] + W * np.round((fp["c_lo"] - rect[:, 2]) / W)   # unwrap to the footprint
    c1 = c0 + rect[:, 3] - 1
    ex = np.stack([fp["r_lo"] - rect[:, 0], rect[:, 1] - fp["r_hi"],
                   fp["c_lo"] - c0, c1 - fp["c_hi"]], 1)[sel]
    hr, hc = (fp["r_hi"] - fp["r_lo"]) / 2, (fp["c_hi"] - fp["c_lo"]) / 2
    hw = np.stack([hr, hr, hc, hc], 1)[sel]
    return ex, hw, proj, sel


def _tight_scenes():
    out = []
    for seed in range(3):
        s = scenes.tiny_scene(400, seed, rows=64, cols=1024, fov_deg=22.5, dist=(0.5, 12.0),
                              spread=1.5, log_scale=(-3.0, -0.5))
        s.views[0].T_ws = scenes.random_pose(np.random.default_rng(seed + 20), 0.5, 30.0)
        out.append(s)
    s = scenes.workload(1, n=4000)
    out.append(s)
    return out


@pytest.mark.parametrize("k", range(4))
def test_box_is_tight_around_the_exact_footprint(oracle_mod, k):
    """Random posed scenes (near, large splats on a 64 x 1024 image; a street): every edge of the
    contract's rectangle lies within 1 px + TIGHT_FRAC x half-width of the exact FP64 footprint
    of the contributing region, and no pixel centre of the footprint is outside it."""
    s = _tight_scenes()[k]
    v = s.views[0]
    ex, hw, proj, sel = _rect_excess(oracle_mod, s.pos_logit, s.quat, s.log_scale, v)
    assert sel.sum() >= 200 and (hw > 10).sum() >= 50       # large footprints are tested
    assert ex.min() > -1.0, ex.min()                          # coverage of every pixel centre
    worst = (ex - (1.0 + TIGHT_FRAC * hw)).max()
    assert worst <= 0.0, (worst, ex.max())


def test_rectangle_pixels_per_reached_pixel(oracle_mod):
    """Summed over the random posed scenes, the contract's rectangles hold at most 1.9 pixels per
    (pixel, primitive) pair whose ray reaches the primitive in FP64 (brute force)."""
    rect_px = reach = 0
    for s in _tight_scenes()[:3]:
        v = s.views[0]
        proj = oracle_mod.project_contract(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows,
                                           v.cols, v.elev_min, v.elev_max)
        params = oracle_mod.split_params(s.pos_logit, s.quat, s.log_scale)
        pix, prim = oracle_mod.reach_pairs(params, v.T_ws, v.rows, v.cols, v.elev_min, v.elev_max)
        pr = proj["pix_rect"].astype(np.int64)
        area = (pr[:, 1] - pr[:, 0] + 1) * pr[:, 3]
        rect_px += int(np.where(proj["count"] > 0, area, 0).sum())
        reach += len(pix)
    assert reach > 100_000
    assert rect_px <= 1.9 * reach, rect_px / reach


def test_contract_reach_radius_margin(oracle_mod):
    """The contract's radius of the contributing region is the closed form
    sqrt(2 ln(o / alpha_min)) (o exp(-r^2 / 2) = alpha_min) widened by 0.1 % + 0.002, to binary32
    rounding; nothing below alpha_min."""
    amin = 1.0 / 255.0
    for o in np.concatenate([np.linspace(0.0045, 0.99, 200), [amin * 1.0001, 0.5]]):
        o = float(np.float32(o))
        exact = math.sqrt(2.0 * math.log(o / float(np.float32(amin))))
        got = oracle_mod.contract_reach_radius(o, amin)
        assert abs(got - (exact * 1.001 + 0.002)) <= 2e-6 * max(exact, 1.0) + 1e-6, (o, got, exact)
    assert oracle_mod.contract_reach_radius(0.5 * amin, amin) == 0.0
