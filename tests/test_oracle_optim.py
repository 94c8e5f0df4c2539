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
