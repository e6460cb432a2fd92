"""Pins of the FP64 oracle's forward render (CPU only).

Each test checks the oracle against something other than itself: a closed form derived by hand,
an invariant of the blending equations (Sec. 3.2.1), a symmetry of the spherical grid, or brute
force.
"""
import math
import os

import numpy as np
import pytest

from paper_2503_17491_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
EMIN, EMAX = scenes.deg(-15.0), scenes.deg(15.0)


def one_splat(L, o, sa, sb, quat=(0.5, 0.5, 0.5, 0.5), mu=None):
    mu = (L, 0.0, 0.0) if mu is None else mu
    logit = math.log(o / (1 - o))
    pl = np.array([[mu[0], mu[1], mu[2], logit]], np.float32)
    q = np.array([quat], np.float32)
    ls = np.array([[math.log(sa), math.log(sb)]], np.float32)
    return pl, q, ls


def params64(pl, q, ls, oracle_mod):
    return oracle_mod.split_params(pl, q, ls)


def test_head_on_closed_form_golden(oracle_mod):
    """On-axis values D = o L, O = o, N = (-o,0,0) from tests/golden (hand derivation)."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "head_on_closed_form.txt"))
    H, W = 33, 513        # odd sizes: row 16 / column 256 look exactly along +x
    for L, o, sa, sb, D_ax, O_ax, Nx_ax in rows:
        pl, q, ls = one_splat(L, o, sa, sb)
        out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
        # the FP32-stored parameters are not exactly L, o, s: use their FP64 values
        o32 = 1.0 / (1.0 + math.exp(-float(pl[0, 3])))
        L32 = float(pl[0, 0])
        r, c = 16, 256
        assert abs(o32 - o) < 1e-6 and abs(L32 - L) < 1e-6
        assert out["D"][r, c] == pytest.approx(o32 * L32, rel=1e-13)
        assert out["O"][r, c] == pytest.approx(o32, rel=1e-13)
        assert out["N"][:, r, c] == pytest.approx([-o32, 0, 0], abs=1e-13)
        assert D_ax == pytest.approx(o * L) and O_ax == o and Nx_ax == -o


@pytest.mark.parametrize("L,o,sa,sb", [(10.0, 0.75, 0.5, 0.25), (3.0, 0.6, 0.2, 0.4)])
def test_head_on_closed_form_every_pixel(oracle_mod, L, o, sa, sb):
    """Every pixel of a single splat facing the sensor matches the hand-derived closed form
    (s_hat from the ray/plane hit, not from the two-plane intersection the oracle uses)."""
    H, W = 17, 256
    emin, emax = scenes.deg(-10), scenes.deg(10)
    pl, q, ls = one_splat(L, o, sa, sb)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, emin, emax, mode="brute")
    L64, o64 = float(pl[0, 0]), 1 / (1 + math.exp(-float(pl[0, 3])))
    sa64, sb64 = math.exp(float(ls[0, 0])), math.exp(float(ls[0, 1]))
    checked = 0
    for r in range(H):
        th = emax - r * (emax - emin) / (H - 1)
        for c in range(W):
            g = math.pi - 2 * math.pi * (c + 0.5) / W
            v = (math.cos(th) * math.cos(g), math.cos(th) * math.sin(g), math.sin(th))
            if v[0] <= 0:
                assert out["O"][r, c] == 0
                continue
            s1, s2 = L64 * v[1] / (v[0] * sa64), L64 * v[2] / (v[0] * sb64)
            a = o64 * math.exp(-0.5 * (s1 * s1 + s2 * s2))
            inside = max(abs(s1), abs(s2)) <= 3 and a >= 1 / 255
            if not inside:
                assert out["O"][r, c] == 0
                continue
            d = L64 / v[0]
            assert out["D"][r, c] == pytest.approx(a * d, rel=1e-11)
            assert out["O"][r, c] == pytest.approx(a, rel=1e-11)
            assert out["N"][0, r, c] == pytest.approx(-a, rel=1e-11)
            assert abs(out["N"][1, r, c]) < 1e-12 and abs(out["N"][2, r, c]) < 1e-12
            checked += 1
    assert checked > 20


def test_single_row_image_looks_along_elev_max(oracle_mod):
    """A one-row image has no row spacing: its rays sit at elev_max (the pixel-grid reading of
    Supp. A's K), so every column of a head-on splat follows the closed form at that elevation."""
    H, W = 1, 256
    emin, emax = float(np.float32(-0.2)), float(np.float32(0.03))   # the intrinsics are binary32
    L, o, sa, sb = 6.0, 0.8, 0.6, 0.3
    pl, q, ls = one_splat(L, o, sa, sb)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, emin, emax, mode="brute")
    L64, o64 = float(pl[0, 0]), 1 / (1 + math.exp(-float(pl[0, 3])))
    sa64, sb64 = math.exp(float(ls[0, 0])), math.exp(float(ls[0, 1]))
    hits = 0
    for c in range(W):
        g = math.pi - 2 * math.pi * (c + 0.5) / W
        v = (math.cos(emax) * math.cos(g), math.cos(emax) * math.sin(g), math.sin(emax))
        if v[0] <= 0:
            assert out["O"][0, c] == 0
            continue
        s1, s2 = L64 * v[1] / (v[0] * sa64), L64 * v[2] / (v[0] * sb64)
        a = o64 * math.exp(-0.5 * (s1 * s1 + s2 * s2))
        if not (max(abs(s1), abs(s2)) <= 3 and a >= 1 / 255):
            assert out["O"][0, c] == 0
            continue
        assert out["D"][0, c] == pytest.approx(a * L64 / v[0], rel=1e-11)
        assert out["O"][0, c] == pytest.approx(a, rel=1e-11)
        hits += 1
    assert hits >= 4


def test_two_splats_front_to_back_closed_form(oracle_mod):
    """Two coaxial splats: D = a1 d1 + (1-a1) a2 d2, O = 1 - (1-a1)(1-a2) on the axis
    (Eqs. ab_depth, ab_opacity); the nearer one composites first whatever the input order."""
    H, W = 33, 513
    for swap in (False, True):
        a = one_splat(5.0, 0.5, 0.5, 0.5)
        b = one_splat(8.0, 0.8, 0.5, 0.5)
        pl = np.concatenate([b[0], a[0]] if swap else [a[0], b[0]])
        q = np.concatenate([b[1], a[1]] if swap else [a[1], b[1]])
        ls = np.concatenate([b[2], a[2]] if swap else [a[2], b[2]])
        out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
        o1 = 1 / (1 + math.exp(-float(a[0][0, 3])))
        o2 = 1 / (1 + math.exp(-float(b[0][0, 3])))
        assert out["D"][16, 256] == pytest.approx(o1 * 5 + (1 - o1) * o2 * 8, rel=1e-12)
        assert out["O"][16, 256] == pytest.approx(1 - (1 - o1) * (1 - o2), rel=1e-12)
        assert out["n_contrib"][16, 256] == 2


def test_alpha_plus_transmittance_is_one(oracle_mod):
    """O + T_final = 1 within 1e-12 (telescoping product of Eq. ab_opacity)."""
    s = scenes.workload(0)
    v = s.views[0]
    out = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                               v.elev_min, v.elev_max)
    assert np.abs(out["O"] + out["T"] - 1).max() < 1e-12
    for seed in range(3):
        t = scenes.tiny_scene(40, seed)
        tv = t.views[0]
        o2 = oracle_mod.full_view(t.pos_logit, t.quat, t.log_scale, tv.T_ws, tv.rows, tv.cols,
                                  tv.elev_min, tv.elev_max, mode="brute")
        assert np.abs(o2["O"] + o2["T"] - 1).max() < 1e-12
        assert o2["O"].max() > 0.3


def test_input_order_invariance(oracle_mod):
    """Shuffling the primitives leaves the image unchanged: the composite order is the range
    sort (Sec. 3.2.1), not the input order."""
    s = scenes.workload(0)
    v = s.views[0]
    ref = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                               v.elev_min, v.elev_max)
    perm = np.random.default_rng(5).permutation(s.n)
    out = oracle_mod.full_view(s.pos_logit[perm], s.quat[perm], s.log_scale[perm], v.T_ws,
                               v.rows, v.cols, v.elev_min, v.elev_max)
    for k in ("D", "O", "N", "T"):
        np.testing.assert_allclose(out[k], ref[k], rtol=0, atol=1e-12)


def test_quarter_turn_is_a_column_shift(oracle_mod):
    """Rotating the sensor by +pi/2 about z (exact pose) shifts the image by W/4 columns with
    wrap-around: the +-pi seam is not special (Sec. 3.2.3)."""
    s = scenes.workload(0)
    v = s.views[0]
    W = v.cols
    ref = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, W,
                               v.elev_min, v.elev_max)
    T = np.eye(4)
    T[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]    # sensor x axis -> world y axis
    out = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, T, v.rows, W,
                               v.elev_min, v.elev_max)
    # column c of the turned sensor looks where column c - W/4 of the original did
    for k in ("D", "O"):
        np.testing.assert_allclose(out[k], np.roll(ref[k], W // 4, axis=1), atol=1e-9)
    assert ref["O"][:, :8].max() > 0 or ref["O"][:, -8:].max() > 0  # something near the seam


def test_disjoint_splats_add(oracle_mod):
    """Two splats that share no pixel render as the sum of their single images."""
    a = one_splat(6.0, 0.7, 0.2, 0.2)
    b = one_splat(6.0, 0.7, 0.2, 0.2, mu=(-6.0, 0.0, 0.0), quat=(0.5, -0.5, 0.5, -0.5))
    H, W = 33, 512
    ra = oracle_mod.full_view(*a, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    rb = oracle_mod.full_view(*b, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    pl = np.concatenate([a[0], b[0]])
    q = np.concatenate([a[1], b[1]])
    ls = np.concatenate([a[2], b[2]])
    rab = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    assert ((ra["O"] > 0) & (rb["O"] > 0)).sum() == 0
    assert ra["O"].sum() > 0 and rb["O"].sum() > 0
    for k in ("D", "O", "N"):
        np.testing.assert_allclose(rab[k], ra[k] + rb[k], atol=1e-14)


def test_cutoffs(oracle_mod):
    """The per-pixel cutoffs act as stated: nothing beyond the 3-sigma box, alpha clamped at
    alpha_max, stop once T would fall below t_min."""
    H, W = 33, 513
    # alpha_max: a near-opaque splat on the axis composites 0.99
    pl, q, ls = one_splat(5.0, 0.9999, 0.5, 0.5)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    assert out["O"][16, 256] == pytest.approx(0.99, abs=1e-15)
    # t_min: stacking opaque splats stops before T < 1e-4: 0.99^2 leaves T = 1e-4, a third
    # would take it to 1e-6 and is not composited
    stack = [one_splat(4.0 + k, 0.9999, 0.5, 0.5) for k in range(3)]
    pl = np.concatenate([s[0] for s in stack])
    q = np.concatenate([s[1] for s in stack])
    ls = np.concatenate([s[2] for s in stack])
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    nc = out["n_contrib"][16, 256]
    assert nc == 2 or (nc == 1 and out["T"][16, 256] >= 1e-4)
    assert out["T"][16, 256] >= 1e-4 * (1 - 1e-12)
    # 3-sigma box: a huge-opacity splat contributes only where max|s_hat| <= 3
    pl, q, ls = one_splat(2.0, 0.99, 0.05, 0.05)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, EMIN, EMAX, mode="brute")
    ang = math.atan(3 * 0.05 / 2.0) * 1.0001
    rr, cc = np.nonzero(out["O"] > 0)
    th = EMAX - rr * (EMAX - EMIN) / (H - 1)
    g = math.pi - 2 * math.pi * (cc + 0.5) / W
    assert np.all(np.abs(g) <= ang) and np.all(np.abs(th) <= ang * 1.01)


def test_culled_equals_brute_workload0(oracle_mod):
    """The tile-culled render equals the brute render bit for bit (binning is conservative)."""
    s = scenes.workload(0)
    v = s.views[0]
    a = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                             v.elev_min, v.elev_max, mode="culled")
    b = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                             v.elev_min, v.elev_max, mode="brute")
    for k in ("D", "O", "N", "T", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])


def test_culled_equals_brute_workload1_sample(oracle_mod):
    """Same on a pixel sample of the 100k-primitive street at a random pose."""
    s = scenes.workload(1)
    v = s.views[0]
    proj = oracle_mod.project_contract(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                                       v.elev_min, v.elev_max)
    params = oracle_mod.split_params(s.pos_logit, s.quat, s.log_scale)
    keys, ids = oracle_mod.bin_pairs(proj, v.rows, v.cols)
    cul = oracle_mod.Culled(keys, ids, v.rows, v.cols, 16, 16)
    rng = np.random.default_rng(3)
    px = np.stack([rng.integers(0, v.rows, 300), rng.integers(0, v.cols, 300)], 1)
    px = np.concatenate([px, [[0, 0], [0, v.cols - 1], [v.rows - 1, 0], [v.rows - 1, v.cols - 1]]])
    a = oracle_mod.render(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                          v.elev_max, culled=cul, pixels=px)
    order = oracle_mod.sort_order(proj["kappa"])
    b = oracle_mod.render(params, proj["flip"], order, v.T_ws, v.rows, v.cols, v.elev_min,
                          v.elev_max, pixels=px)
    for k in ("D", "O", "N", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])
    assert (a["O"] > 0.5).mean() > 0.3


@pytest.mark.parametrize("o,band,bits", [
    (0.8, (0.05, 0.002, 0.0, 0.0, 0.0), (1, 2)),      # box edge and alpha_min bands
    (0.995, (0.0, 0.0, 0.0, 0.0, 0.004), (16,)),     # alpha_max clamp band
])
def test_ambiguity_band_flags_follow_the_closed_form(oracle_mod, o, band, bits):
    """The band flags that take pixels out of the GPU comparison mark exactly the pixels whose
    decision quantity lies within the band of its threshold -- checked against the head-on
    closed form (s_hat and alpha by hand), so the parity tests exclude no more than that."""
    H, W = 17, 256
    emin, emax = scenes.deg(-10), scenes.deg(10)
    L, sa, sb = 6.0, 0.6, 0.3
    pl, q, ls = one_splat(L, o, sa, sb)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, emin, emax, band=band, mode="brute")
    L64, o64 = float(pl[0, 0]), 1 / (1 + math.exp(-float(pl[0, 3])))
    sa64, sb64 = math.exp(float(ls[0, 0])), math.exp(float(ls[0, 1]))
    a_min, a_max, sigma = 1 / 255, 0.99, 3.0
    flagged = {b: 0 for b in bits}
    for r in range(H):
        th = emax - r * (emax - emin) / (H - 1)
        for c in range(W):
            g = math.pi - 2 * math.pi * (c + 0.5) / W
            v = (math.cos(th) * math.cos(g), math.cos(th) * math.sin(g), math.sin(th))
            want = 0
            if v[0] != 0:
                s1, s2 = L64 * v[1] / (v[0] * sa64), L64 * v[2] / (v[0] * sb64)
                smax = max(abs(s1), abs(s2))
                edge = abs(abs(smax - sigma) - band[0] * sigma)
                if 1 in bits and edge < 1e-9:
                    continue                      # on the band's own edge: either answer
                if abs(smax - sigma) <= band[0] * sigma:
                    want |= 1
                if smax <= sigma and v[0] > 0:    # in front of the sensor
                    a_raw = o64 * math.exp(-0.5 * (s1 * s1 + s2 * s2))
                    if abs(a_raw - a_max) <= band[4]:
                        want |= 16
                    a = min(a_raw, a_max)
                    if abs(a - a_min) <= band[1]:
                        want |= 2
            got = int(out["band"][r, c])
            assert got == want, (r, c, got, want)
            for b in bits:
                flagged[b] += bool(got & b)
    assert all(n > 0 for n in flagged.values()), flagged


def test_ambiguity_band_flags_the_stop_on_t_min(oracle_mod):
    """Three coaxial splats of opacity 0.99: with alpha clamped at 0.99 the transmittance after
    two of them is at least 1e-4 = t_min, and the third takes it below near the axis.  The t_min
    band flags exactly the pixels whose running transmittance comes within the band of t_min
    (closed form), and the pixels that cross it stop before the crossing splat."""
    H, W = 33, 2049         # a fine grid around the axis (row 16 / column 1024 look along +x)
    emin, emax = scenes.deg(-1.5), scenes.deg(1.5)
    splats = [one_splat(L, 0.99, 0.5, 0.5) for L in (5.0, 8.0, 11.0)]
    pl, q, ls = (np.concatenate(x) for x in zip(*splats))
    band = (0.0, 0.0, 0.5, 0.0, 0.0)
    out = oracle_mod.full_view(pl, q, ls, np.eye(4), H, W, emin, emax, band=band, mode="brute")
    t_min, a_min = 1e-4, 1 / 255
    flagged = stopped = stopped_in_band = 0
    for r in range(H):
        th = emax - r * (emax - emin) / (H - 1)
        for c in range(W):
            g = math.pi - 2 * math.pi * (c + 0.5) / W
            v = (math.cos(th) * math.cos(g), math.cos(th) * math.sin(g), math.sin(th))
            want, T, n = 0, 1.0, 0
            if v[0] > 0:
                for P in splats:
                    L64 = float(P[0][0, 0])
                    o64 = 1 / (1 + math.exp(-float(P[0][0, 3])))
                    s64 = math.exp(float(P[2][0, 0]))
                    s1, s2 = L64 * v[1] / (v[0] * s64), L64 * v[2] / (v[0] * s64)
                    if max(abs(s1), abs(s2)) > 3:
                        continue
                    al = min(o64 * math.exp(-0.5 * (s1 * s1 + s2 * s2)), 0.99)
                    if al < a_min:
                        continue
                    tt = T * (1 - al)
                    if abs(tt - t_min) <= band[2] * t_min:
                        want |= 4
                    if tt < t_min:
                        stopped += 1
                        stopped_in_band += want != 0
                        break
                    T, n = tt, n + 1
            assert int(out["band"][r, c]) == want, (r, c)
            assert int(out["n_contrib"][r, c]) == n, (r, c)
            flagged += want != 0
    assert flagged > 0 and stopped > 0 and stopped_in_band > 0
