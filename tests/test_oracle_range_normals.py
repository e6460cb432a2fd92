"""Pins of the oracle's self-regularised normal term (Eq. loss_normal: rendered normals against
the normals of the rendered range map)."""
import numpy as np
import pytest

import oracle


def _plane_range(rows, cols, emin, emax, n, d0):
    """Range map of the plane n . p = d0 (n the unit normal facing away from the sensor side)."""
    V = oracle.pixel_rays(rows, cols, emin, emax)
    nv = V @ n
    D = np.where(nv > 1e-3, d0 / np.where(nv > 1e-3, nv, 1.0), 0.0)
    return D


@pytest.mark.parametrize("n", [np.array([1.0, 0.0, 0.0]),
                               np.array([0.8, 0.36, 0.48]) / np.linalg.norm([0.8, 0.36, 0.48])])
def test_planar_range_map_gives_the_plane_normal(n):
    """On a planar range map every stencil's normal is the plane's normal turned towards the
    sensor (-n): with N = -k n the term is 1 - k per stencil, with gradient -lambda n_D."""
    rows, cols, emin, emax = 8, 64, -0.3, 0.3
    D = _plane_range(rows, cols, emin, emax, n, 6.0)
    Dt = D.copy()
    k = 0.7
    N = np.broadcast_to((-k * n)[:, None, None], (3, rows, cols)).copy()
    val, gD, gN = oracle.range_normal_loss(D, N, Dt, rows, cols, emin, emax, lambda_n=2.0)
    valid = (Dt[:-1] > 0) & (np.roll(Dt, -1, 1)[:-1] > 0) & (Dt[1:] > 0)
    cnt = int(valid.sum())
    assert cnt > 50
    assert val == pytest.approx(2.0 * (1 - k) * cnt, rel=1e-9)
    np.testing.assert_allclose(gN[:, :-1][:, valid], np.repeat((2.0 * n)[:, None], cnt, 1),
                               atol=1e-9)


def test_finite_differences_in_depth_and_normal():
    """Central differences of the term in every D and N entry (a smooth random range map with the
    azimuth wrap inside the image)."""
    rows, cols, emin, emax = 5, 12, -0.4, 0.4
    rng = np.random.default_rng(3)
    D = 6.0 + rng.normal(0, 0.3, (rows, cols))
    N = rng.normal(0, 1, (3, rows, cols))
    Dt = np.ones((rows, cols))
    Dt[2, 5] = 0.0
    val, gD, gN = oracle.range_normal_loss(D, N, Dt, rows, cols, emin, emax, lambda_n=1.3)
    h = 1e-6
    for r in range(rows):
        for c in range(cols):
            a, b = D.copy(), D.copy()
            a[r, c] += h
            b[r, c] -= h
            fd = (oracle.range_normal_loss(a, N, Dt, rows, cols, emin, emax, 1.3)[0] -
                  oracle.range_normal_loss(b, N, Dt, rows, cols, emin, emax, 1.3)[0]) / (2 * h)
            assert abs(fd - gD[r, c]) <= 1e-6 * max(1.0, abs(gD[r, c])), (r, c, fd, gD[r, c])
    for (k, r, c) in [(0, 0, 0), (1, 3, 11), (2, 1, 6), (0, 4, 3)]:
        a, b = N.copy(), N.copy()
        a[k, r, c] += h
        b[k, r, c] -= h
        fd = (oracle.range_normal_loss(D, a, Dt, rows, cols, emin, emax, 1.3)[0] -
              oracle.range_normal_loss(D, b, Dt, rows, cols, emin, emax, 1.3)[0]) / (2 * h)
        assert abs(fd - gN[k, r, c]) <= 1e-7 * max(1.0, abs(gN[k, r, c]))
    assert gD[2, 5] != 0.0 or gD[1, 5] != 0.0   # invalid target only removes its own stencils


def test_zero_rendered_range_removes_its_stencils():
    """A pixel with D = 0 sits at the sensor: the stencils that use it (as u, x or y) do not
    count, and no gradient reaches it from them."""
    rows, cols, emin, emax = 4, 10, -0.2, 0.2
    rng = np.random.default_rng(9)
    D = 5.0 + rng.normal(0, 0.2, (rows, cols))
    N = rng.normal(0, 1, (3, rows, cols))
    Dt = np.ones((rows, cols))
    D[1, 4] = 0.0
    val, gD, gN = oracle.range_normal_loss(D, N, Dt, rows, cols, emin, emax)
    for (r, c) in [(1, 4), (1, 3), (0, 4)]:   # u, the stencil whose x it is, whose y it is
        assert (gN[:, r, c] == 0).all()
    assert gD[1, 4] == 0.0
    full = (rows - 1) * cols
    assert np.isfinite(val)
    cnt = int((np.abs(gN).sum(0) > 0).sum())
    assert cnt == full - 3
