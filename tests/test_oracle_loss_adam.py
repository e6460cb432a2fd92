"""Pins of the oracle's loss (Eqs. loss_range, loss_normal, loss_opacity over the valid mask M_v)
and Adam step, against hand-computed values and Adam's known closed-form behaviour."""
import math

import numpy as np
import pytest


def test_loss_hand_values(oracle_mod):
    # 4 pixels; the last has target range 0 (ray drop: outside M_v)
    D = np.array([2.0, 5.0, 1.0, 7.0])
    Dt = np.array([1.5, 5.0, 3.0, 0.0])
    N = np.array([[0.0, 1.0, 0.6, 1.0], [0.0, 0.0, 0.8, 0.0], [-1.0, 0.0, 0.0, 0.0]])
    Nt = np.array([[0.0, 0.0, 0.6, 1.0], [0.0, 1.0, 0.8, 0.0], [-1.0, 0.0, 0.0, 0.0]])
    O = np.array([0.5, 1.0, 0.25, 0.9])
    L, gD, gN, gO = oracle_mod.loss(D, N, O, Dt, Nt, lambda_n=0.5, lambda_o=0.1)
    # L_d = 0.5 + 0 + 2 ; L_n = 0.5 * ((1-1) + (1-0) + (1-1)) ; L_o = 0.1 * (ln 2 + 0 + ln 4)
    want = 2.5 + 0.5 * 1.0 + 0.1 * (math.log(2) + math.log(4))
    assert L == pytest.approx(want, rel=1e-14)
    np.testing.assert_array_equal(gD, [1.0, 0.0, -1.0, 0.0])
    np.testing.assert_allclose(gN[:, :3], -0.5 * Nt[:, :3])
    assert np.all(gN[:, 3] == 0)
    np.testing.assert_allclose(gO, [-0.1 / 0.5, -0.1, -0.1 / 0.25, 0.0])


def test_adam_first_step_is_lr_times_sign(oracle_mod):
    """With bias correction, Adam's first update is -lr * g / |g| (m_hat = g, v_hat = g^2)."""
    rng = np.random.default_rng(0)
    p = rng.normal(size=100)
    g = rng.normal(size=100) * 10 ** rng.uniform(-4, 4, 100)
    p0 = p.copy()
    m = np.zeros(100)
    v = np.zeros(100)
    oracle_mod.adam(p, g, m, v, lr=1e-2, eps=1e-15, step=1)
    np.testing.assert_allclose(p - p0, -1e-2 * np.sign(g), rtol=1e-9)


def test_adam_constant_gradient(oracle_mod):
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step: each update is
    -lr * sign(g) again."""
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -3.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 6):
        before = p.copy()
        oracle_mod.adam(p, g, m, v, lr=0.1, b1=0.9, b2=0.99, eps=1e-15, step=t)
        np.testing.assert_allclose(p - before, -0.1 * np.sign(g), rtol=1e-9)


def test_loss_wrapper_with_converted_inputs(oracle_mod):
    """float32 inputs are converted to float64 copies by the wrapper; those copies must stay alive
    through the C call (a large case, so a freed copy would be overwritten)."""
    rng = np.random.default_rng(0)
    P = 5000
    D = rng.uniform(0, 50, P).astype(np.float32)
    N = rng.normal(size=(3, P)).astype(np.float32)
    O = rng.uniform(0, 1, P).astype(np.float32)
    Dt = np.where(rng.uniform(size=P) < 0.2, 0, rng.uniform(1, 50, P)).astype(np.float32)
    Nt = rng.normal(size=(3, P)).astype(np.float32)
    L, gD, gN, gO = oracle_mod.loss(D, N, O, Dt, Nt, lambda_n=0.5, lambda_o=0.1)
    L2, *_ = oracle_mod.loss(D.astype(np.float64), N.astype(np.float64), O.astype(np.float64),
                             Dt.astype(np.float64), Nt.astype(np.float64), lambda_n=0.5,
                             lambda_o=0.1)
    assert L == L2
    v = Dt > 0
    assert np.array_equal(gD != 0, v & (D != Dt))


def test_scale_regularizer_values_and_gradient(oracle_mod):
    """Hand values of the scale term and central differences of its gradient away from the
    threshold and from ties."""
    import math
    ls = np.log(np.array([[2.0, 1.0], [0.3, 0.4], [0.5, 3.0], [1.2, 1.2]]))
    v, g = oracle_mod.scale_regularizer(ls, 0.5, 1.0)
    assert math.isclose(v, 0.5 * ((2.0 - 1.0) + 0.0 + (3.0 - 1.0) + (1.2 - 1.0)), rel_tol=1e-12)
    np.testing.assert_allclose(g, [[1.0, 0.0], [0.0, 0.0], [0.0, 1.5], [0.6, 0.0]], rtol=1e-12)
    rng = np.random.default_rng(4)
    ls = rng.uniform(-1.5, 1.5, (30, 2))
    _, g = oracle_mod.scale_regularizer(ls, 0.7, 1.3)
    for i in range(30):
        for k in range(2):
            h = 1e-6
            a, b = ls.copy(), ls.copy()
            a[i, k] += h
            b[i, k] -= h
            fd = (oracle_mod.scale_regularizer(a, 0.7, 1.3)[0] -
                  oracle_mod.scale_regularizer(b, 0.7, 1.3)[0]) / (2 * h)
            if abs(math.exp(ls[i, k]) - 1.3) > 1e-3 and abs(ls[i, 0] - ls[i, 1]) > 1e-3:
                assert abs(fd - g[i, k]) <= 1e-6 * max(1.0, abs(g[i, k])), (i, k, fd, g[i, k])


def test_range_weight_rho_d(oracle_mod):
    """rho_d = Dt^p: with p = -1 the range term is the sum of relative errors (hand values), and
    p = 0 is the plain L1 term."""
    D = np.array([12.0, 9.0, 5.0, 3.0])
    Dt = np.array([10.0, 10.0, 0.0, 2.0])
    N = np.zeros((3, 4))
    O = np.ones(4)
    L, gD, gN, gO = oracle_mod.loss(D, N, O, Dt, N, lambda_n=0.0, rho_exp=-1.0)
    assert L == pytest.approx(0.2 + 0.1 + 0.5)
    np.testing.assert_allclose(gD, [0.1, -0.1, 0.0, 0.5])
    L0, gD0, _, _ = oracle_mod.loss(D, N, O, Dt, N, lambda_n=0.0, rho_exp=0.0)
    assert L0 == pytest.approx(2.0 + 1.0 + 1.0)
    np.testing.assert_allclose(gD0, [1.0, -1.0, 0.0, 1.0])
    L2, gD2, _, _ = oracle_mod.loss(D, N, O, Dt, N, lambda_n=0.0, rho_exp=2.0)
    assert L2 == pytest.approx(100 * 2 + 100 * 1 + 4 * 1)


def test_opacity_term_is_flat_below_its_floor(oracle_mod):
    """-log max(O, o_eps) is constant for O below o_eps, so its gradient is zero there, and
    the value is -log o_eps (hand values)."""
    D = np.array([1.0, 1.0])
    Dt = np.array([1.0, 1.0])
    Z = np.zeros((3, 2))
    O = np.array([1e-8, 0.5])
    L, gD, gN, gO = oracle_mod.loss(D, Z, O, Dt, Z, lambda_n=0.0, lambda_o=2.0, o_eps=1e-6)
    assert L == pytest.approx(2.0 * (-math.log(1e-6) - math.log(0.5)))
    np.testing.assert_allclose(gO, [0.0, -4.0])
