"""Pins for the oracle's noisegate (Eq. 13): the gate curve's regions, continuity and
partials, the R = 1 identity, the settled gain on a constant input, and the analytic
backward pass against central finite differences."""
import numpy as np

from oracle import processors as op


def test_gate_curve_regions_and_continuity():
    T, W, R = -5.0, 0.7, 3.0
    Gu = np.array([T + W + 1.0, T + W, T, T - W, T - W - 2.0])
    Gy, dGu, dT, dW, dR = op.gate_curve(Gu, T, W, R)
    assert Gy[0] == Gu[0] and dGu[0] == 1.0                     # open: unchanged
    assert np.isclose(Gy[4], T + R * (Gu[4] - T))                # closed: expansion by R
    assert np.isclose(dGu[4], R) and np.isclose(dT[4], 1 - R)
    # the knee meets both lines with matching value and slope at T - W and T + W
    for edge, inner in ((T + W, T + W - 1e-9), (T - W, T - W + 1e-9)):
        a = op.gate_curve(np.array([edge - 1e-12, edge + 1e-12]), T, W, R)
        assert abs(a[0][0] - a[0][1]) < 1e-9 and abs(a[1][0] - a[1][1]) < 1e-6
    assert np.isclose(Gy[2], T + (1 - R) * W / 4.0)             # centre of the knee: d = -W


def test_gate_curve_partials_finite_differences():
    rng = np.random.Generator(np.random.PCG64(4))
    T, W, R = -3.0, 0.9, 2.5
    Gu = rng.uniform(T - 3, T + 3, 50)
    _, dGu, dT, dW, dR = op.gate_curve(Gu, T, W, R)
    h = 1e-6
    f = lambda *a: op.gate_curve(*a)[0]
    np.testing.assert_allclose(dGu, (f(Gu + h, T, W, R) - f(Gu - h, T, W, R)) / (2 * h), atol=1e-6)
    np.testing.assert_allclose(dT, (f(Gu, T + h, W, R) - f(Gu, T - h, W, R)) / (2 * h), atol=1e-6)
    np.testing.assert_allclose(dW, (f(Gu, T, W + h, R) - f(Gu, T, W - h, R)) / (2 * h), atol=1e-6)
    np.testing.assert_allclose(dR, (f(Gu, T, W, R + h) - f(Gu, T, W, R - h)) / (2 * h), atol=1e-6)


def test_ratio_one_is_identity():
    rng = np.random.Generator(np.random.PCG64(5))
    u = rng.standard_normal((2, 3000)) * 0.1
    y = op.noisegate_fwd(u, [0.99, -4.0, 0.69, 1.0])
    np.testing.assert_allclose(y, u, rtol=1e-13, atol=1e-15)


def test_constant_input_settles_on_the_static_curve():
    a, n = 0.01, 20000
    u = np.full((2, n), a)
    alpha, T, W, R = 0.99, np.log(0.05), 0.3, 2.0
    y = op.noisegate_fwd(u, [alpha, T, W, R])
    x = (2 * a) ** 2                       # the settled envelope (Eq. 8 fixed point)
    Gu = np.log(x + op.COMP_EPS)
    assert Gu < T - W                      # a quiet input is below the knee: expanded
    want = a * np.exp(T + R * (Gu - T) - Gu)
    assert np.isclose(y[0, -1], want, rtol=1e-9) and np.isclose(y[1, -1], want, rtol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(6))
    L = 600
    u = rng.standard_normal((2, L)) * np.linspace(0.001, 0.3, L)   # crosses the knee
    p = np.array([0.97, np.log(0.01), 0.4, 2.2])
    ybar = rng.standard_normal((2, L))
    ubar, pbar = op.noisegate_bwd(u, p, ybar)
    f = lambda uu, pp: np.sum(ybar * op.noisegate_fwd(uu, pp))
    for i in range(4):
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        assert np.isclose(pbar[i], (f(u, pp) - f(u, pm)) / (2 * h), rtol=1e-5, atol=1e-8), i
    for (c, t) in ((0, 10), (1, 300), (0, 599)):
        h = 1e-7
        up, um = u.copy(), u.copy()
        up[c, t] += h
        um[c, t] -= h
        assert np.isclose(ubar[c, t], (f(up, p) - f(um, p)) / (2 * h), rtol=1e-5, atol=1e-8)
