"""Pins for the oracle's multi-port nodes (Sec. 2 Definitions, Eq. 1a/1b with M inputs
and N outputs and typed edges): split, merge and the sidechain compressor, and the
port-aware renders and backward pass."""
import numpy as np
import pytest

import synth
from oracle import graph as og, processors as op, render as orr
from tests.helpers import permute_graph, random_mimo_dag

P, J, K = synth.P, synth.J, synth.K


def fd(f, x, i, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp.flat[i] += h
    xm.flat[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_split_closed_form_and_merge_inverts_it(rng):
    u = rng.standard_normal((2, 300))
    y0, y1 = op.split_fwd(u)
    m, s = (u[0] + u[1]) / 2, (u[0] - u[1]) / 2
    np.testing.assert_array_equal(y0, np.stack([m, m]))
    np.testing.assert_array_equal(y1, np.stack([s, s]))
    np.testing.assert_allclose(op.merge_fwd([y0, y1]), u, atol=1e-15)


def test_split_and_merge_adjoints_are_transposes(rng):
    """<split(u), w> = <u, split^T(w)> and likewise for merge (both are linear)."""
    u = rng.standard_normal((2, 200))
    w0, w1 = rng.standard_normal((2, 2, 200))
    ys = op.split_fwd(u)
    lhs = np.sum(ys[0] * w0) + np.sum(ys[1] * w1)
    assert np.isclose(lhs, np.sum(u * op.split_bwd(u, [w0, w1])[0]), rtol=1e-13)
    a, b = rng.standard_normal((2, 2, 200))
    w = rng.standard_normal((2, 200))
    ub = op.merge_bwd([a, b], w)
    assert np.isclose(np.sum(op.merge_fwd([a, b]) * w), np.sum(a * ub[0]) + np.sum(b * ub[1]), rtol=1e-13)


def test_sidechain_silent_key_passes_main_through(rng):
    """A silent key keeps the envelope at 0: G_u = ln(eps) lies below every threshold
    of the synthetic range, so the gain is exactly 1."""
    u = rng.standard_normal((2, 1000))
    p = np.array([0.99, np.log(0.01), 0.7, 4.0])
    np.testing.assert_allclose(op.sidechain_fwd([u, np.zeros((2, 1000))], p), u, rtol=1e-15)


def test_sidechain_constant_key_settles_on_the_static_curve(rng):
    a, n = 0.3, 30000
    key = np.full((2, n), a)
    u = rng.standard_normal((2, n))
    alpha, T, W, R = 0.99, np.log(0.02), 0.3, 4.0
    y = op.sidechain_fwd([u, key], [alpha, T, W, R])
    x = (2 * a) ** 2                               # the settled envelope (Eq. 8 fixed point)
    Gu = np.log(x + op.COMP_EPS)
    assert Gu > T + W                              # a loud key is above the knee
    gain = np.exp(T + (Gu - T) / R - Gu)           # Eq. 10 above the knee, Eq. 12
    np.testing.assert_allclose(y[:, -1], gain * u[:, -1], rtol=1e-9)


def test_sidechain_adjoint_fd(rng):
    L = 500
    u = rng.standard_normal((2, L)) * 0.3
    key = rng.standard_normal((2, L)) * np.linspace(0.01, 0.4, L)   # crosses the knee
    p = np.array([0.97, np.log(0.01), 0.5, 3.0])
    w = rng.standard_normal((2, L))
    (ub, kb), pb = op.sidechain_bwd([u, key], p, w)
    f = lambda uu, kk, pp: np.sum(w * op.sidechain_fwd([uu, kk], pp))
    for i in range(4):
        h = 1e-6 * max(1.0, abs(p[i]))
        assert np.isclose(pb[i], fd(lambda pp: f(u, key, pp), p, i, h), rtol=1e-5, atol=1e-8), i
    for i in rng.choice(2 * L, 5, replace=False):
        assert np.isclose(ub.flat[i], fd(lambda uu: f(uu, key, p), u, i), rtol=1e-6, atol=1e-8)
        assert np.isclose(kb.flat[i], fd(lambda kk: f(u, kk, p), key, i, 1e-7), rtol=1e-5, atol=1e-8)


def test_ports_are_validated():
    types = [synth.I, P, J, synth.O]
    edges = [(0, 1), (1, 2), (1, 2), (2, 3)]
    og.validate(types, edges, ports=[(0, 0), (0, 0), (1, 1), (0, 0)])
    for bad in ([(0, 0), (2, 0), (1, 1), (0, 0)],      # split has outputs 0, 1
                [(0, 0), (0, 0), (1, 2), (0, 0)],      # merge has inputs 0, 1
                [(1, 0), (0, 0), (1, 1), (0, 0)]):     # a source has one output
        with pytest.raises(og.GraphError):
            og.validate(types, edges, ports=bad)


def test_mid_side_processing_round_trip(rng):
    """i -> split -> (mid: gain 0 dB, side: gain 0 dB) -> merge -> o renders the input."""
    g = synth.Graph()
    i = g.add(synth.I)
    sp = g.add(P)
    gm, gs = g.add(synth.G), g.add(synth.G)
    mg = g.add(J)
    o = g.add(synth.O)
    g.connect(i, sp)
    g.connect(sp, gm, 0, 0)
    g.connect(sp, gs, 1, 0)
    g.connect(gm, mg, 0, 0)
    g.connect(gs, mg, 0, 1)
    g.connect(mg, o)
    src = rng.standard_normal((1, 2, 400))
    P_ = {synth.G: np.zeros((2, 2))}
    y = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P_, ports=g.ports))
    np.testing.assert_allclose(y[0], src[0], atol=1e-14)
    # a side gain of -inf dB keeps only the mid: both channels (l + r) / 2
    P_[synth.G][1] = -60.0
    y = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P_, ports=g.ports))
    m = (src[0, 0] + src[0, 1]) / 2
    np.testing.assert_allclose(y[0], np.stack([m, m]), atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_mimo_scheduled_equals_one_by_one(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = random_mimo_dag(rng, 3, 12, 2)
    P_ = synth.random_params(g, seed)
    src = 0.2 * rng.standard_normal((g.count(synth.I), 2, 700))
    hp = dict(eq_taps=31)
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P_, hp, ports=g.ports))
    for m in ("beam", "greedy", "one_by_one"):
        got = orr.render_scheduled(g.types, g.edges, src, P_, hp, method=m, ports=g.ports)[0]
        np.testing.assert_allclose(got[:, 0] if got.ndim == 4 else got, want, atol=1e-12)


def test_mimo_relabelling_invariance(rng):
    g = random_mimo_dag(rng, 2, 10, 1)
    perm = list(rng.permutation(g.n_nodes))
    h = permute_graph(g, perm)
    P_ = synth.random_params(g, 3)
    src = 0.2 * rng.standard_normal((g.count(synth.I), 2, 500))
    hp = dict(eq_taps=31)
    yg = orr.render_ports(g.types, g.edges, src, P_, hp, g.ports)
    # the permuted graph's inputs and parameter rows follow its own node order
    ins_g = [v for v in range(g.n_nodes) if g.types[v] == synth.I]
    ins_h = sorted(ins_g, key=lambda v: perm[v])
    src_h = src[[ins_g.index(v) for v in ins_h]]
    P_h = {}
    for t, tab in P_.items():
        rows_g = [v for v in range(g.n_nodes) if g.types[v] == t]
        P_h[t] = tab[[rows_g.index(v) for v in sorted(rows_g, key=lambda v: perm[v])]]
    yh = orr.render_ports(h.types, h.edges, src_h, P_h, hp, h.ports)
    for v in range(g.n_nodes):
        for k in range(len(yg[v])):
            np.testing.assert_allclose(yh[perm[v]][k], yg[v][k], atol=1e-12)


def test_mimo_graph_backward_fd(rng):
    g = random_mimo_dag(rng, 2, 7, 1)
    P_ = synth.random_params(g, 5)
    L = 300
    src = 0.3 * rng.standard_normal((g.count(synth.I), 2, L))
    hp = dict(eq_taps=15)
    w = rng.standard_normal((1, 2, L))
    dP, dS = orr.backward(g.types, g.edges, src, P_, w, hp, ports=g.ports)

    def loss(s, p):
        return np.sum(w * orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, s, p, hp, ports=g.ports)))
    for i in rng.choice(src.size, 4, replace=False):
        assert np.isclose(dS.flat[i], fd(lambda s: loss(s, P_), src, i), rtol=1e-5, atol=1e-8)
    for t, tab in P_.items():
        for i in rng.choice(tab.size, min(3, tab.size), replace=False):
            def f(x, t=t):
                q = dict(P_)
                q[t] = x
                return loss(src, q)
            num = fd(f, np.asarray(tab, dtype=np.float64), i, 1e-6 * max(1.0, abs(float(tab.flat[i]))))
            assert np.isclose(dP[t].flat[i], num, rtol=1e-4, atol=1e-7), (t, i)
