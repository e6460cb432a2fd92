"""Pins of the oracle's map growth (Sec. 3.3.1 local model initialisation, Sec. 3.3.2
densification masks): weights, masks, systematic sampling and the new primitives."""
import math

import numpy as np
import pytest

import oracle


def test_counts_match_brute_force_enumeration():
    """The closed-form counts equal an enumeration of every sample point s_j located in the
    cumulative weights by a library search, and each count is floor or ceil of n_d q_i / Q."""
    rng = np.random.default_rng(0)
    for trial in range(20):
        P = int(rng.integers(1, 400))
        q = rng.integers(0, 3000, P).astype(np.uint64)
        q[rng.uniform(size=P) < 0.3] = 0
        Q = int(q.sum())
        if Q == 0:
            continue
        n_d = int(rng.integers(1, 2 * P + 5))
        o = int(rng.integers(0, Q))
        cnt, first = oracle.systematic_counts(q, n_d, o)
        s = [(j * Q + o) // n_d for j in range(n_d)]
        upper = np.cumsum(q.astype(np.int64))
        owner = np.searchsorted(upper, s, side="right")
        ref = np.bincount(owner, minlength=P)
        np.testing.assert_array_equal(cnt, ref)
        assert cnt.sum() == n_d
        for i in np.nonzero(cnt)[0]:
            assert owner[first[i]] == i and (first[i] == 0 or owner[first[i] - 1] < i)
        e = n_d * q.astype(np.float64) / Q
        assert ((cnt == np.floor(e)) | (cnt == np.ceil(e))).all()


def test_flat_weights_pick_evenly_spaced_pixels():
    P, n_d = 1200, 40
    q = np.full(P, 7, np.uint64)
    for o in (0, 1, 7 * 30 - 1, 8399):
        cnt, first = oracle.systematic_counts(q, n_d, o)
        sel = np.nonzero(cnt)[0]
        assert len(sel) == n_d and (cnt <= 1).all()
        assert (np.diff(sel) == P // n_d).all()


def test_weights_masks_and_a_step_edge():
    """A wall at 10 m with a box at 6 m in front of it: the weight is w0 off the edges and
    w0 + 4 at the pixel before the box's left edge (capped by w_cap); invalid pixels and, in
    refinement, pixels outside M_n or M_e weigh 0."""
    rows, cols = 6, 20
    Dt = np.full((rows, cols), 10.0, np.float32)
    Dt[:, 8:12] = 6.0
    Dt[0, 0] = 0.0
    q = oracle.densify_weights(Dt, None, None, rows, cols, False, 0, 0, 0.25, 16.0)
    q = q.reshape(rows, cols).astype(np.int64)
    assert q[3, 3] == 64                               # 0.25 m * 256
    assert q[3, 7] == math.floor((0.25 + 4.0) * 256)   # g_x = 6 - 10
    assert q[3, 11] == math.floor((0.25 + 4.0) * 256)  # g_x = 10 - 6
    assert q[0, 0] == 0 and q[0, 19] == 64             # wrap neighbour invalid: g_x = 0
    qc = oracle.densify_weights(Dt, None, None, rows, cols, False, 0, 0, 0.25, 1.0)
    assert qc.reshape(rows, cols)[3, 7] == 256
    D = Dt.copy()
    O = np.ones_like(Dt)
    O[1, :] = 0.2          # M_n
    D[2, 5] += 0.3         # M_e
    D[4, 6] += 0.05        # below lambda_de
    qr = oracle.densify_weights(Dt, D, O, rows, cols, True, 0.5, 0.1, 0.25, 16.0)
    qr = qr.reshape(rows, cols)
    on = np.zeros((rows, cols), bool)
    on[1, :] = True
    on[2, 5] = True
    on[0, 0] = False
    on[1, :] &= Dt[1, :] > 0
    np.testing.assert_array_equal(qr > 0, on)


def test_selection_frequencies_follow_the_weights():
    """Over many calls the mean count of a pixel is n_d q_i / Q (the offset is uniform)."""
    q = np.array([1, 0, 5, 2, 9, 3, 0, 4], np.uint64) * 256
    n_d = 3
    Q = int(q.sum())
    acc = np.zeros(len(q))
    calls = 3000
    for call in range(calls):
        o = oracle.densify_offset(Q, 11, call)
        assert 0 <= o < Q
        acc += oracle.systematic_counts(q, n_d, o)[0]
    np.testing.assert_allclose(acc / calls, n_d * q / Q, atol=0.04)


def _pose(rng):
    a = rng.normal(size=3)
    th = np.linalg.norm(a)
    k = a / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    T = np.eye(4)
    T[:3, :3] = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    T[:3, 3] = rng.normal(0, 5, 3)
    return T


def _quat_rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_new_primitives_round_trip():
    """Two posed views: every filled slot's centre projects back to its pixel's ray at the
    target range, its normal (third rotation column) points at the sensor, its scale and opacity
    follow the definition; empty slots are exactly the duplicate draws."""
    rng = np.random.default_rng(5)
    views = [(_pose(rng), 8, 64, -0.3, 0.2), (_pose(rng), 5, 40, -0.1, 0.4)]
    P = sum(r * c for _, r, c, _, _ in views)
    Dt = rng.uniform(2, 30, P).astype(np.float32)
    Dt[rng.uniform(size=P) < 0.2] = 0
    n_d = 150
    pl, qt, ls, pix = oracle.densify(views, Dt, None, None, n_d, w0=0.05, w_cap=8.0, scale_k=1.5,
                                     opacity=0.3, seed=3, call=2)
    filled = pix >= 0
    assert filled.sum() > 100
    off = 0
    for (T, rows, cols, emin, emax) in views:
        V = oracle.pixel_rays(rows, cols, emin, emax).reshape(-1, 3)
        Ti = np.linalg.inv(T)
        dg, dt = 2 * math.pi / cols, (emax - emin) / (rows - 1)
        for j in np.nonzero((pix >= off) & (pix < off + rows * cols))[0]:
            k = pix[j] - off
            ps = Ti[:3, :3] @ pl[j, :3] + Ti[:3, 3]
            d = float(Dt[off + k])
            np.testing.assert_allclose(ps, d * V[k], atol=1e-9 * d)
            n = _quat_rot(qt[j])[:, 2]
            np.testing.assert_allclose(n, -(T[:3, :3] @ V[k]), atol=1e-12)
            assert np.dot(n, T[:3, 3] - pl[j, :3]) > 0
            np.testing.assert_allclose(ls[j], math.log(1.5 * d * math.sqrt(dg * dt)), rtol=1e-12)
            assert pl[j, 3] == pytest.approx(math.log(0.3 / 0.7))
        off += rows * cols
    assert (pl[~filled, 3] == oracle.DENSIFY_EMPTY_LOGIT).all()
    assert len(set(pix[filled].tolist())) == filled.sum()
    assert Dt[pix[filled]].min() > 0


def test_nothing_masked_gives_empty_slots():
    views = [(np.eye(4), 4, 16, -0.1, 0.1)]
    pl, qt, ls, pix = oracle.densify(views, np.zeros(64, np.float32), None, None, 10)
    assert (pix == -1).all() and (pl[:, 3] == oracle.DENSIFY_EMPTY_LOGIT).all()


def test_normal_straight_down_uses_the_fallback_rotation():
    T = np.eye(4)
    pl, q, ls = oracle.init_primitive(5.0, np.array([0.0, 0.0, 1.0]), T, 0.01, 0.01, 1.0, 0.5)
    np.testing.assert_allclose(_quat_rot(q)[:, 2], [0, 0, -1], atol=1e-15)


def test_invalid_lower_neighbour_gives_no_vertical_gradient():
    """A ray drop below a valid pixel contributes no range gradient (it is not a surface edge)."""
    rows, cols = 6, 20
    Dt = np.full((rows, cols), 10.0, np.float32)
    Dt[3, 5] = 0.0
    q = oracle.densify_weights(Dt, None, None, rows, cols, False, 0, 0, 0.25, 16.0)
    q = q.reshape(rows, cols).astype(np.int64)
    assert q[2, 5] == 64 and q[3, 4] == 64 and q[3, 5] == 0


def test_offset_is_one_quantile_of_every_total():
    """The draw's offset is the quantile x / 2^32 of the total weight: doubling the total doubles
    the offset (up to the floor), whatever the call."""
    for call in range(50):
        for Q in (1000, 77777, 123456789):
            o1 = oracle.densify_offset(Q, 5, call)
            o2 = oracle.densify_offset(2 * Q, 5, call)
            assert o2 in (2 * o1, 2 * o1 + 1)
