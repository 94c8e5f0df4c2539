"""Pins for the oracle's processors, adjoints and loss against closed forms, brute
force and central finite differences (Sec. 3 Eq. 2-12; Sec. 4 loss reading)."""
import numpy as np
import pytest

import synth
from oracle import processors as op, render as orr, loss as ol, graph as og
from tests.helpers import random_dag, permute_graph


def fd_grad(f, x, idx, rel=1e-6):
    x = np.array(x, dtype=np.float64)
    h = rel * max(1.0, abs(x.flat[idx]))
    xp, xm = x.copy(), x.copy()
    xp.flat[idx] += h
    xm.flat[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def sig(rng, L, scale=0.3):
    return scale * rng.standard_normal((2, L))


# ------------------------------------------------------------------ gain / imager
def test_gain_closed_form_on_gain_only_graph(rng):
    """Gain-only graph: each output is sum over paths of prod exp(p) times the source."""
    I, O, M, G = 0, 1, 2, 3
    g = synth.Graph()
    i0, i1 = g.add(I), g.add(I)
    a, b = g.add_serial_chain([G, G])
    c = g.add(G)
    m = g.add(M)
    o = g.add(O)
    for s, d in [(i0, a), (i1, c), (i0, c), (b, m), (c, m), (m, o)]:
        g.connect(s, d)
    L = 64
    src = rng.standard_normal((2, 2, L)).astype(np.float32)
    P = {G: rng.uniform(-1, 1, (3, 2)).astype(np.float32)}
    e = np.exp(P[G].astype(np.float64))
    s0, s1 = src.astype(np.float64)
    want = (e[0] * e[1])[:, None] * s0 + e[2][:, None] * (s1 + s0)
    Y = orr.render_one_by_one(g.types, g.edges, src, P)
    np.testing.assert_allclose(orr.outputs_of(g.types, Y)[0], want, rtol=1e-14, atol=1e-14)


def test_gradient_term_magnitudes(rng):
    """The magnitude sums bound the gradients (triangle inequality) and equal them when
    every term has the same sign (ybar = u makes the gain's terms u^2 >= 0)."""
    u = sig(rng, 500)
    p = np.array([0.3, -0.2])
    ub, pb = op.gain_bwd(u, p, u)
    np.testing.assert_allclose(op.gain_bwd_abs(u, p, u), pb, rtol=1e-13)
    w = sig(rng, 500)
    _, pb = op.gain_bwd(u, p, w)
    assert np.all(op.gain_bwd_abs(u, p, w) >= np.abs(pb))
    q = np.array([0.4])
    _, pb = op.imager_bwd(u, q, w)
    assert op.imager_bwd_abs(u, q, w)[0] >= abs(pb[0])
    # ybar with sidebar = (l - r): all imager terms are squares
    d = u[0] - u[1]
    yb = np.stack([d, -d])
    _, pb = op.imager_bwd(u, q, yb)
    np.testing.assert_allclose(op.imager_bwd_abs(u, q, yb), pb, rtol=1e-13)


def test_imager_identity_and_mono(rng):
    u = sig(rng, 128)
    np.testing.assert_allclose(op.imager_fwd(u, [0.0]), u, atol=1e-15)
    mono = op.imager_fwd(u, [-80.0])
    np.testing.assert_allclose(mono[0], (u[0] + u[1]) / 2, atol=1e-15)
    np.testing.assert_allclose(mono[1], (u[0] + u[1]) / 2, atol=1e-15)


# ------------------------------------------------------------------ EQ
@pytest.mark.parametrize("N", [15, 255, 1023])
def test_eq_flat_is_identity(N):
    h = op.eq_taps_from_bands(np.zeros(8), N)
    d = np.zeros(N)
    d[(N - 1) // 2] = 1.0
    np.testing.assert_allclose(h, d, atol=1e-13)


@pytest.mark.parametrize("N", [15, 255])
def test_eq_taps_match_library_idft_and_are_even(rng, N):
    logmag = rng.uniform(-1.5, 1.5, (N + 1) // 2)
    A = np.exp(logmag)
    full = np.concatenate([A, A[1:][::-1]])         # A_{N-k} = A_k
    h0 = np.real(np.fft.ifft(full))                  # (1/N) sum_k A_k w^{kn}
    H = (N - 1) // 2
    h0c = np.concatenate([h0[-H:], h0[:H + 1]])      # n = -H..H
    want = op.hann_sym(N) * h0c
    h = op.zerophase_taps(logmag, N)
    np.testing.assert_allclose(h, want, atol=1e-14)
    np.testing.assert_allclose(h, h[::-1], atol=1e-15)
    # the window vanishes just past the printed bounds +-(N+1)/2
    assert abs(0.5 * (1 + np.cos(2 * np.pi * ((N + 1) / 2) / (N + 1)))) < 1e-15


def test_eq_impulse_returns_taps(rng):
    N, L, t0 = 63, 200, 77
    bands = rng.uniform(-12, 12, 8)
    h = op.eq_taps_from_bands(bands, N)
    u = np.zeros((2, L))
    u[:, t0] = 1.0
    y = op.eq_fwd(u, bands, N)
    H = (N - 1) // 2
    np.testing.assert_allclose(y[0, t0 - H:t0 + H + 1], h, atol=1e-14)
    assert np.abs(y[0, :t0 - H]).max() < 1e-14 and np.abs(y[0, t0 + H + 1:]).max() < 1e-14


def test_eq_band_matrix():
    B = op.eq_band_matrix(1023)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-15)
    assert B[0, 0] == 1.0 and B[-1, -1] == 1.0
    # constant dB over all bands gives that dB at every bin
    np.testing.assert_allclose(op.eq_logmag(np.full(8, 6.0), 1023), 6.0 * np.log(10) / 20, atol=1e-14)


@pytest.mark.parametrize("N", [15, 255, 1023, 2047])
def test_eq_window_is_the_hann_window_through_the_printed_bounds(N):
    """The window of Eq. 4 is the symmetric Hann window whose zeros fall on the printed
    bounds -(N+1)/2 and (N+1)/2: numpy's (N+2)-point Hann window without its two zero
    end points."""
    full = np.hanning(N + 2)
    assert full[0] == 0.0 and full[-1] == 0.0
    np.testing.assert_allclose(op.hann_sym(N), full[1:-1], rtol=0, atol=1e-15)


def test_eq_band_design_is_linear_in_log_frequency():
    """Band gains that are linear in log2 f come back exactly at every bin between the
    first and last band centre (linear interpolation in log2 f reproduces a linear
    function), and the end bands' gains hold beyond the end centres."""
    N, fs = 1023, 44100
    c = op.eq_band_centres()
    a, slope = -3.0, 1.7
    db = a + slope * np.log2(c)
    got = op.eq_band_matrix(N, fs) @ db
    f = np.arange((N + 1) // 2) * fs / N
    inner = (f > c[0]) & (f < c[-1])
    np.testing.assert_allclose(got[inner], a + slope * np.log2(f[inner]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[f <= c[0]], db[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[f >= c[-1]], db[-1], rtol=0, atol=1e-12)
    # the centres are log-spaced over 20 Hz .. 20 kHz, one per eighth of the three decades
    np.testing.assert_allclose(np.log10(c / 20.0), (np.arange(8) + 0.5) * 3 / 8, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N, L", [(9, 30), (9, 3), (63, 5), (63, 1)])
def test_fir_centred_brute_force(rng, N, L):
    """Brute-force sums, including signals shorter than the filter (lags beyond the
    signal carry no pair of samples)."""
    h = rng.standard_normal(N)
    u = rng.standard_normal((2, L))
    H = (N - 1) // 2
    y = np.zeros((2, L))
    for t in range(L):
        for m in range(-H, H + 1):
            if 0 <= t - m < L:
                y[:, t] += h[m + H] * u[:, t - m]
    np.testing.assert_allclose(op.fir_centred(u, h), y, atol=1e-13)
    yb = rng.standard_normal((2, L))
    hb = np.zeros(N)
    ub = np.zeros((2, L))
    for t in range(L):
        for m in range(-H, H + 1):
            if 0 <= t - m < L:
                hb[m + H] += np.sum(yb[:, t] * u[:, t - m])
                ub[:, t - m] += h[m + H] * yb[:, t]
    np.testing.assert_allclose(op.fir_centred_taps_grad(u, yb, H), hb, atol=1e-12)
    np.testing.assert_allclose(op.fir_centred_adjoint(yb, h), ub, atol=1e-12)


# ------------------------------------------------------------------ compressor
def test_envelope_constant_input_closed_form():
    alpha, c, L = 0.99, 0.3, 500
    x = np.full(L, 4 * c * c)
    g = op.envelope(x, alpha)
    n = np.arange(L)
    np.testing.assert_allclose(g, 4 * c * c * (1 - alpha ** (n + 1)), rtol=1e-12)


def test_envelope_equals_direct_fir(rng):
    alpha, L = 0.93, 60
    x = rng.random(L)
    h = (1 - alpha) * alpha ** np.arange(L)                 # Eq. 9, FIR as long as x
    direct = np.array([sum(h[k] * x[n - k] for k in range(n + 1)) for n in range(L)])
    np.testing.assert_allclose(op.envelope(x, alpha), direct, rtol=1e-12)
    # the reverse recursion is the transpose of the (1/(1-alpha)) forward filter
    Mx = np.array([[alpha ** (n - k) if n >= k else 0.0 for k in range(L)] for n in range(L)])
    a = rng.standard_normal(L)
    np.testing.assert_allclose(op.envelope_reverse(a, alpha), Mx.T @ a, rtol=1e-11, atol=1e-12)


def test_compressor_settles_on_static_curve():
    alpha, c, L = 0.95, 0.2, 4000
    T, W, R = np.log(0.01), 0.6908, 4.0
    u = np.full((2, L), c)
    y = op.compressor_fwd(u, [alpha, T, W, R])
    Gu = np.log(4 * c * c + op.COMP_EPS)
    Gy = op.knee(np.array([Gu]), T, W, R)[0][0]
    np.testing.assert_allclose(y[:, -1], c * np.exp(Gy - Gu), rtol=1e-12)
    assert Gu > T + W  # compressing branch: T + (Gu - T)/R
    np.testing.assert_allclose(Gy, T + (Gu - T) / R, rtol=1e-14)


def test_compressor_ratio_one_is_identity(rng):
    u = sig(rng, 300)
    np.testing.assert_allclose(op.compressor_fwd(u, [0.97, -3.0, 0.7, 1.0]), u, rtol=1e-14)


def test_knee_continuity():
    T, W, R = -2.0, 0.5, 3.0
    for b in (T - W, T + W):
        lo, hi = np.array([b - 1e-9]), np.array([b + 1e-9])
        kl, kh = op.knee(lo, T, W, R), op.knee(hi, T, W, R)
        assert abs(kl[0][0] - kh[0][0]) < 1e-8          # value
        assert abs(kl[1][0] - kh[1][0]) < 1e-8          # slope
    # below the knee the curve leaves the level alone, above it it divides the excess by R
    below = np.array([T - W - 3.0, T - W - 0.1])
    kv, ks = op.knee(below, T, W, R)[:2]
    np.testing.assert_array_equal(kv, below)
    np.testing.assert_array_equal(ks, np.ones(2))
    above = np.array([T + W + 0.1, T + W + 3.0])
    kv, ks = op.knee(above, T, W, R)[:2]
    np.testing.assert_allclose(kv, T + (above - T) / R, rtol=1e-15)
    np.testing.assert_allclose(ks, np.full(2, 1 / R), rtol=1e-15)


# ------------------------------------------------------------------ adjoints by FD
CASES = [
    (3, lambda r: r.uniform(-1, 1, 2)),
    (4, lambda r: r.uniform(-1, 1, 1)),
    (5, lambda r: r.uniform(-12, 12, 8)),
    (6, lambda r: np.array([r.uniform(0.9, 0.99), np.log(0.02), 0.6908, r.uniform(1.5, 6)])),
]


@pytest.mark.parametrize("t,pgen", CASES)
def test_processor_adjoints_fd(rng, t, pgen):
    L = 400
    hp = dict(orr.DEFAULT_HP, eq_taps=31)
    u = sig(rng, L)
    p = pgen(rng)
    w = rng.standard_normal((2, L))
    ubar, pbar = orr.process_bwd(t, u, p, w, hp)
    f_p = lambda pp: np.sum(w * orr.process(t, u, pp, hp))
    for k in range(len(p)):
        assert np.isclose(pbar[k], fd_grad(f_p, p, k), rtol=2e-6, atol=1e-8), (t, k)
    f_u = lambda uu: np.sum(w * orr.process(t, uu.reshape(2, L), p, hp))
    for idx in rng.choice(2 * L, 12, replace=False):
        assert np.isclose(ubar.flat[idx], fd_grad(f_u, u, idx), rtol=2e-6, atol=1e-8), (t, idx)


# ------------------------------------------------------------------ renders
def _random_setup(rng, n_mid=8, L=256, n_out=1):
    g = random_dag(rng, n_inputs=3, n_mid=n_mid, n_outputs=n_out)
    K = g.count(0)
    src = (0.3 * rng.standard_normal((K, 2, L))).astype(np.float32)
    P = synth.random_params(g, int(rng.integers(0, 1 << 30)))
    return g, src, P


@pytest.mark.parametrize("seed", range(6))
def test_scheduled_equals_one_by_one(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g, src, P = _random_setup(rng, n_out=2)
    hp = dict(eq_taps=31)
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P, hp))
    for m in ("one_by_one", "greedy", "beam"):
        got = orr.render_scheduled(g.types, g.edges, src, P, hp, method=m)[0]
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_relabelling_invariance_of_outputs(rng):
    g, src, P = _random_setup(rng, n_out=2)
    hp = dict(eq_taps=31)
    perm = list(rng.permutation(g.n_nodes))
    h = permute_graph(g, perm)
    # sources and parameter rows follow their nodes
    def reorder(graph_from, graph_to, table_t, t):
        ids_from = [v for v in range(graph_from.n_nodes) if graph_from.types[v] == t]
        ids_to = [v for v in range(graph_to.n_nodes) if graph_to.types[v] == t]
        pos = {perm[v]: k for k, v in enumerate(ids_from)}
        return np.stack([table_t[pos[v]] for v in ids_to])
    src_h = reorder(g, h, src, 0)
    P_h = {t: reorder(g, h, P[t], t) for t in P}
    yg = orr.render_one_by_one(g.types, g.edges, src, P, hp)
    yh = orr.render_one_by_one(h.types, h.edges, src_h, P_h, hp)
    for v in range(g.n_nodes):
        np.testing.assert_allclose(yh[perm[v]], yg[v], rtol=1e-12, atol=1e-13)


def test_union_equals_per_graph(rng):
    hp = dict(eq_taps=31)
    setups = [_random_setup(rng, n_mid=6) for _ in range(3)]
    types, edges, _ = og.union([s[0] for s in setups])
    src = np.concatenate([s[1] for s in setups])
    P = {}
    for t in range(9):
        rows = [s[2][t] for s in setups if t in s[2]]
        if rows:
            P[t] = np.concatenate(rows)
    got = orr.render_scheduled(types, edges, src, P, hp)[0]
    want = np.concatenate([orr.outputs_of(s[0].types, orr.render_one_by_one(s[0].types, s[0].edges, s[1], s[2], hp))
                           for s in setups])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_graph_backward_fd(rng):
    g, src, P = _random_setup(rng, n_mid=7, L=300, n_out=2)
    hp = dict(eq_taps=31)
    W = rng.standard_normal((2, 2, 300))

    def loss_of(Pm):
        return np.sum(W * orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, Pm, hp)))
    dP, dS = orr.backward(g.types, g.edges, src, P, W, hp)
    for t in P:
        for idx in range(min(P[t].size, 6)):
            def f(x, t=t):
                Pm = dict(P)
                Pm[t] = x.reshape(P[t].shape)
                return loss_of(Pm)
            assert np.isclose(dP[t].flat[idx], fd_grad(f, P[t].astype(np.float64), idx),
                              rtol=1e-5, atol=1e-8), (t, idx)
    f_s = lambda x: np.sum(W * orr.outputs_of(
        g.types, orr.render_one_by_one(g.types, g.edges, x.reshape(src.shape), P, hp)))
    for idx in rng.choice(src.size, 6, replace=False):
        assert np.isclose(dS.flat[idx], fd_grad(f_s, src.astype(np.float64), idx), rtol=1e-5, atol=1e-8)


# ------------------------------------------------------------------ loss
def test_loss_zero_at_target(rng):
    t = rng.standard_normal((1, 2, 4096))
    assert ol.mrstft(t, t) == 0.0


def test_spec_matches_direct_dft(rng):
    M, L = 16, 64
    x = rng.standard_normal(L)
    S = ol.spec(x, M)
    w = ol.hann_periodic(M)
    n = np.arange(M)
    for f in range(S.shape[0]):
        fr = x[f * 4:f * 4 + M] * w
        for k in range(M // 2 + 1):
            assert abs(S[f, k] - np.sum(fr * np.exp(-2j * np.pi * k * n / M))) < 1e-12


def test_loss_grad_fd(rng):
    res = (16, 32)
    y = rng.standard_normal((1, 2, 160))
    t = rng.standard_normal((1, 2, 160))
    g = ol.mrstft_grad(y, t, res)
    for idx in rng.choice(y.size, 10, replace=False):
        f = lambda x: ol.mrstft(x.reshape(y.shape), t, res)
        assert np.isclose(g.flat[idx], fd_grad(f, y, idx), rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("M", [512, 1024, 2048])
def test_spec_of_bin_centred_cosine(M):
    """A cosine of amplitude a on bin k0 seen through the periodic Hann window: the
    window's DFT is M/2 at bin 0, -M/4 at bins +-1 and zero elsewhere, so every frame
    holds a M/4 at k0, a M/8 at k0 +- 1 and nothing in any other bin (a symmetric Hann
    window would leak into every bin)."""
    a, k0, hop = 0.7, 37, M // 4
    n = np.arange(M + 3 * hop)
    S = np.abs(ol.spec(a * np.cos(2 * np.pi * k0 * n / M + 0.3), M))
    expect = np.zeros(M // 2 + 1)
    expect[k0] = a * M / 4
    expect[k0 - 1] = expect[k0 + 1] = a * M / 8
    assert S.shape == (4, M // 2 + 1)
    np.testing.assert_allclose(S, np.broadcast_to(expect, S.shape), rtol=0, atol=1e-10 * M)


def test_frames_start_at_multiples_of_the_hop():
    """No centre padding: frame f covers [f M/4, f M/4 + M) and only whole frames count,
    F = 1 + (L - M) // (M/4)."""
    M, hop = 64, 16
    for L, F in [(64, 1), (79, 1), (80, 2), (144, 6), (159, 6)]:
        fr, nf = ol.frames(np.arange(L, dtype=np.float64), M)
        assert nf == F and fr.shape == (F, M)
        np.testing.assert_array_equal(fr[:, 0], np.arange(F) * hop)
        np.testing.assert_array_equal(fr[:, -1], np.arange(F) * hop + M - 1)


def test_loss_of_a_doubled_target_in_closed_form(rng):
    """With y = 2 t every bin has |Y| = 2 |T|: spectral convergence is || |T| || / || |T| || = 1
    against the target t and 1/2 the other way round, the log term ln 2 either way (up to
    the 1e-7 floor), and the row loss is their mean over resolutions and channels, so
    mrstft(2t, t) = 1 + ln 2 and mrstft(t, 2t) = 1/2 + ln 2 for one row (twice that for two)."""
    t = rng.standard_normal((1, 2, 3 * 2048))
    assert abs(ol.mrstft(2 * t, t) - (1 + np.log(2))) < 1e-6
    assert abs(ol.mrstft(t, 2 * t) - (0.5 + np.log(2))) < 1e-6
    t2 = rng.standard_normal((2, 2, 3 * 2048))
    assert abs(ol.mrstft(2 * t2, t2) - 2 * (1 + np.log(2))) < 2e-6
    # a common scale leaves the loss unchanged (again up to the floor)
    y = rng.standard_normal((1, 2, 3 * 2048))
    assert abs(ol.mrstft(8 * y, 8 * t) - ol.mrstft(y, t)) < 1e-6
