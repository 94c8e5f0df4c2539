"""Pins for the oracle's fitting layer: parameter maps, their inverses and slopes,
and Adam (the published algorithm) on closed-form cases."""
import numpy as np
import pytest

from oracle import optim as oo

CODES = [oo.IDENT, oo.ALPHA, oo.SOFTPLUS, oo.RATIO, oo.NEGSP, oo.ATTACK]


@pytest.mark.parametrize("code", CODES)
def test_map_inverse_round_trip_and_slope(rng, code):
    th = rng.uniform(-4, 4, 50)
    p = oo.to_param(th, code)
    np.testing.assert_allclose(oo.to_theta(p, code), th, rtol=1e-8, atol=1e-8)
    h = 1e-6
    fd = (oo.to_param(th + h, code) - oo.to_param(th - h, code)) / (2 * h)
    np.testing.assert_allclose(oo.dparam_dtheta(th, code), fd, rtol=1e-7, atol=1e-10)


def test_map_ranges():
    th = np.linspace(-30, 30, 1001)
    a = oo.to_param(th, oo.ALPHA)
    assert a.min() >= 0.9 and a.max() <= 0.9999
    assert oo.to_param(th, oo.SOFTPLUS).min() > 0
    assert oo.to_param(th, oo.RATIO).min() > 1
    assert oo.to_param(th, oo.NEGSP).max() < 0
    b = oo.to_param(th, oo.ATTACK)
    assert b.min() >= 0.5 and b.max() <= 0.9999


def test_adam_first_step_moves_by_lr(rng):
    """At t = 1 the bias-corrected step is g/|g| (up to eps): every coordinate moves lr."""
    th = rng.standard_normal(20)
    g = rng.standard_normal(20)
    new, m, v = oo.adam_step(th, np.zeros(20), np.zeros(20), g, 1, lr=0.05, eps=0.0)
    np.testing.assert_allclose(th - new, 0.05 * np.sign(g), rtol=1e-12)


def test_adam_minimises_quadratic(rng):
    c = rng.standard_normal(10)
    th, m, v = np.zeros(10), np.zeros(10), np.zeros(10)
    for t in range(1, 3001):
        th, m, v = oo.adam_step(th, m, v, 2 * (th - c), t, lr=1e-2)
    np.testing.assert_allclose(th, c, atol=1e-3)


def test_param_codes_layout():
    assert list(oo.param_codes(6, 4)) == [oo.ALPHA, oo.IDENT, oo.SOFTPLUS, oo.RATIO]
    rc = oo.param_codes(8, 50)
    assert list(rc[12:24]) == [oo.NEGSP] * 12 and list(rc[36:48]) == [oo.NEGSP] * 12
    assert list(rc[:12]) == [oo.IDENT] * 12 and rc[48] == rc[49] == oo.IDENT
    assert list(oo.param_codes(13, 5)) == [oo.ATTACK, oo.ALPHA, oo.IDENT, oo.SOFTPLUS, oo.RATIO]


def test_delay_z_pair_layout():
    c = oo.param_codes(7, 176)
    assert list(c[:22]) == [oo.ZRE, oo.ZIM] + [oo.IDENT] * 20 and np.array_equal(c[22:44], c[:22])
    assert list(oo.param_codes(7, 880)[::22]) == [oo.ZRE] * 40


def test_delay_z_penalty_gradient_by_finite_differences(rng):
    # with a zero loss gradient the update direction is the penalty's gradient alone
    codes = oo.param_codes(7, 44)
    th = rng.uniform(-1.5, 1.5, (5, 44))
    g = oo.delay_z_grad(th, np.zeros_like(th), codes)
    h = 1e-6
    for j in (0, 22):
        for d in (0, 1):
            tp, tm = th.copy(), th.copy()
            tp[:, j + d] += h
            tm[:, j + d] -= h
            fd = (oo.z_penalty(tp[:, j], tp[:, j + 1]) - oo.z_penalty(tm[:, j], tm[:, j + 1])) / (2 * h)
            np.testing.assert_allclose(g[:, j + d], fd, rtol=1e-6, atol=1e-12)
    assert np.array_equal(g[:, 2:22], np.zeros((5, 20)))


def test_delay_z_penalty_closed_form():
    codes = oo.param_codes(7, 22)
    th = np.zeros(22)
    th[0] = 2.0                                     # z = 2: 2 lam (2 - 1) (1, 0)
    g = oo.delay_z_grad(th, np.zeros(22), codes)
    np.testing.assert_allclose(g[:2], [2 * oo.LAMBDA_Z, 0.0], rtol=1e-15)
    th[0], th[1] = 0.6, 0.8                         # on the unit circle: no pull
    np.testing.assert_allclose(oo.delay_z_grad(th, np.zeros(22), codes)[:2], [0.0, 0.0], atol=1e-15)


def test_delay_z_normalisation_is_scale_invariant_and_unit(rng):
    codes = oo.param_codes(7, 176)
    ang = rng.uniform(-np.pi, np.pi, (6, 8))
    th = rng.standard_normal((6, 176))
    th[:, 0::22], th[:, 1::22] = np.cos(ang), np.sin(ang)      # |z| = 1: penalty gradient 0
    g = rng.standard_normal((6, 176))
    a = oo.delay_z_grad(th, g, codes)
    for c in (1e-6, 3.0, 1e5):
        np.testing.assert_allclose(oo.delay_z_grad(th, c * g, codes), np.where(codes == oo.IDENT, c * g, a),
                                   rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.hypot(a[:, 0::22], a[:, 1::22]), 1.0, rtol=1e-12)
    # the direction is the raw gradient's, and the other columns are untouched
    cosv = (a[:, 0::22] * g[:, 0::22] + a[:, 1::22] * g[:, 1::22]) / np.hypot(g[:, 0::22], g[:, 1::22])
    np.testing.assert_allclose(cosv, 1.0, rtol=1e-12)
    assert np.array_equal(a[:, codes == oo.IDENT], g[:, codes == oo.IDENT])
    z = np.zeros((1, 22))
    assert np.array_equal(oo.delay_z_grad(th[:1, :22], z, codes[:22])[:, :2], np.zeros((1, 2)))
