"""Pins for the oracle's attack/release ballistics (Sec. 3, Eq. 8 with different attack
and release coefficients, the form the paper describes before restricting it to one)."""
import numpy as np

import synth
from oracle import processors as op, render as orr
from tests.helpers import random_dag


def fd(f, x, i, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp.flat[i] += h
    xm.flat[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_equal_coefficients_reduce_to_the_one_pole_filter(rng):
    x = rng.uniform(0, 1, 3000) ** 3
    g, _ = op.envelope_ar(x, 0.97, 0.97)
    np.testing.assert_allclose(g, op.envelope(x, 0.97), rtol=1e-12, atol=1e-15)
    u = rng.standard_normal((2, 3000)) * 0.2
    p = [0.98, np.log(0.01), 0.4, 3.0]
    np.testing.assert_allclose(op.ballistic_fwd(u, [0.98, 0.98] + p[1:]), op.compressor_fwd(u, p), rtol=1e-12)


def test_step_input_closed_forms():
    """x = 1 for n < 200 then 0: the attack rise 1 - aa^(n+1), then the release decay
    g[199] ar^(m+1)."""
    aa, ar = 0.9, 0.999
    x = np.concatenate([np.ones(200), np.zeros(300)])
    g, att = op.envelope_ar(x, aa, ar)
    n = np.arange(200)
    np.testing.assert_allclose(g[:200], 1 - aa ** (n + 1), rtol=1e-12)
    m = np.arange(300)
    np.testing.assert_allclose(g[200:], g[199] * ar ** (m + 1), rtol=1e-12)
    assert att[:200].all() and not att[200:].any()


def test_ballistic_gradients_fd(rng):
    L = 400
    u = rng.standard_normal((2, L)) * np.concatenate([np.linspace(0.01, 0.4, L // 2), np.linspace(0.4, 0.01, L // 2)])
    p = np.array([0.9, 0.995, np.log(0.01), 0.5, 3.0])
    w = rng.standard_normal((2, L))
    ub, pb = op.ballistic_bwd(u, p, w)
    f = lambda pp: np.sum(w * op.ballistic_fwd(u, pp))
    for i in range(5):
        h = 1e-7 * max(1.0, abs(p[i]))
        assert np.isclose(pb[i], fd(f, p, i, h), rtol=1e-5, atol=1e-8), i
    fu = lambda uu: np.sum(w * op.ballistic_fwd(uu.reshape(2, -1), p))
    for i in rng.choice(2 * L, 6, replace=False):
        assert np.isclose(ub.flat[i], fd(fu, u.reshape(-1), i, 1e-7), rtol=1e-5, atol=1e-8)


def test_graphs_with_ballistics_scheduled_equals_one_by_one(rng):
    g = random_dag(rng, 2, 8, kinds=(synth.A, synth.G, synth.C, synth.M))
    P = synth.random_params(g, 3)
    src = 0.2 * rng.standard_normal((g.count(synth.I), 2, 900))
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P))
    got = orr.render_scheduled(g.types, g.edges, src, P)[0]
    np.testing.assert_allclose(got, want, atol=1e-12)
