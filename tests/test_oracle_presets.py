"""Pins for the oracle's processors in the paper's own settings (Sec. 3): the EQ
parameterised by its log-magnitudes (N = 2047, 1024 values), the multitap delay
with one tap per 100 ms slot (20 taps per channel, 880 values) and the reverb with
FFT 384 / hop 192 and 192 log-magnitudes per filter (768 values)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import processors as op, render as orr
from tests.helpers import random_dag

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_param_sizes.json")


def fd(f, x, i, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_widths_match_the_paper():
    gold = json.load(open(GOLD))
    assert synth.PAPER_PARAM_COLS[synth.E] == gold["eq_params"] == (gold["eq_taps"] + 1) // 2
    assert synth.PAPER_PARAM_COLS[synth.D] == gold["delay_params"]
    assert gold["delay_params"] == gold["delay_delays"] * (2 + gold["delay_mags"])
    assert op.DELAY_PAPER_TAPS * 2 == gold["delay_delays"] and op.DELAY_K == gold["delay_mags"]
    assert synth.PAPER_PARAM_COLS[synth.R] == gold["reverb_params"] == op.rv_cols(op.RV_PAPER)
    assert op.RV_PAPER["rv_nfft"] // 2 == gold["reverb_mags"]
    hp = orr.paper_hp()
    assert hp["eq_taps"] == gold["eq_taps"] and hp["delay_slot"] == 4410 and hp["delay_taps"] == 20


# ------------------------------------------------------------------ EQ, log-magnitude parameter
def test_eq_flat_logmag_is_a_scaled_identity():
    """All A_k = e^c: the cosine sum is the Dirichlet kernel, N delta[n], so h = e^c delta."""
    N = 2047
    h = op.zerophase_taps(np.full(1024, 0.3), N)
    want = np.zeros(N)
    want[(N - 1) // 2] = np.exp(0.3)
    np.testing.assert_allclose(h, want, atol=1e-13)


def test_eq_design_interpolates_the_magnitudes_exactly(rng):
    """Before the window the design is the exact inverse DFT: its N-point DFT (a
    library FFT) gives back A_k at every bin, mirrored."""
    N = 2047
    lm = rng.uniform(-1.5, 1.5, 1024)
    h = op.zerophase_taps(lm, N)
    h0 = h / op.hann_sym(N)
    X = np.fft.fft(np.fft.ifftshift(h0))
    A = np.exp(lm)
    np.testing.assert_allclose(X.real[:1024], A, rtol=1e-11)
    np.testing.assert_allclose(X.real[1024:], A[1:][::-1], rtol=1e-11)
    assert np.max(np.abs(X.imag)) < 1e-11


def test_eq_logmag_matches_the_band_mode_and_its_chain_rule(rng):
    N, L = 63, 500
    bands = rng.uniform(-12, 12, 8)
    lm = op.eq_logmag(bands, N)
    u = rng.standard_normal((2, L))
    w = rng.standard_normal((2, L))
    np.testing.assert_allclose(op.eq_fwd_logmag(u, lm, N), op.eq_fwd(u, bands, N), atol=1e-13)
    ub1, pb_lm = op.eq_bwd_logmag(u, lm, w, N)
    ub2, pb_b = op.eq_bwd(u, bands, w, N)
    np.testing.assert_allclose(ub1, ub2, atol=1e-13)
    np.testing.assert_allclose(op.eq_band_matrix(N).T @ pb_lm * op.LN10 / 20, pb_b, rtol=1e-12)


def test_eq_logmag_gradients_fd(rng):
    N, L = 31, 300
    lm = rng.uniform(-1, 1, 16)
    u = rng.standard_normal((2, L))
    w = rng.standard_normal((2, L))
    ubar, pbar = op.eq_bwd_logmag(u, lm, w, N)
    f = lambda q: np.sum(w * op.eq_fwd_logmag(u, q, N))
    for k in (0, 1, 7, 15):
        assert np.isclose(pbar[k], fd(f, lm, k), rtol=1e-7, atol=1e-9), k
    fu = lambda uu: np.sum(w * op.eq_fwd_logmag(uu.reshape(2, -1), lm, N))
    for i in rng.choice(2 * L, 5, replace=False):
        assert np.isclose(ubar.flat[i], fd(fu, u.reshape(-1), i), rtol=1e-7, atol=1e-9)


# ------------------------------------------------------------------ delay, one tap per slot
TAPS, SLOT = 20, 64       # the paper's 20 slots, shortened to 64 samples for speed


def delay_params(rng, on_circle=True):
    p = np.zeros((2, TAPS, 2 + op.DELAY_K))
    d = rng.integers(0, SLOT, (2, TAPS))
    ang = -2 * np.pi * d / SLOT
    r = 1.0 if on_circle else 0.97
    p[..., 0], p[..., 1] = r * np.cos(ang), r * np.sin(ang)
    p[..., 2:] = rng.uniform(-1.2, 0.2, (2, TAPS, op.DELAY_K))
    return p.reshape(-1), d


def test_slot_delays_stay_in_their_slots_and_fir_brute_force(rng):
    p, dd = delay_params(rng)
    z, lm = op.delay_split(p, TAPS)
    d = op.delay_samples(z, SLOT, SLOT)
    np.testing.assert_array_equal(d, dd + SLOT * np.arange(TAPS)[None, :])
    assert np.all((d >= SLOT * np.arange(TAPS)) & (d < SLOT * (np.arange(TAPS) + 1)))
    L = 1500
    u = rng.standard_normal((2, L))
    y = op.delay_fwd(u, p, SLOT, TAPS, SLOT)
    H = (op.DELAY_FIR - 1) // 2
    want = np.zeros_like(u)
    for x in range(2):
        for m in range(TAPS):
            c = op.zerophase_taps(lm[x, m], op.DELAY_FIR)
            for j in range(-H, H + 1):
                s = d[x, m] + j
                for t in range(max(s, 0), L):
                    if t - s < L:
                        want[x, t] += c[j + H] * u[x, t - s]
    np.testing.assert_allclose(y, want, atol=1e-12)


def test_slot_surrogate_is_exact_on_the_unit_circle(rng):
    p, _ = delay_params(rng)
    u = rng.standard_normal((2, 1500))
    np.testing.assert_allclose(op.delay_fwd_surrogate(u, p, SLOT, TAPS, SLOT),
                               op.delay_fwd(u, p, SLOT, TAPS, SLOT), atol=1e-10)


def test_slot_delay_gradients_fd(rng):
    p, _ = delay_params(rng)
    L = 1400
    u = rng.standard_normal((2, L))
    w = rng.standard_normal((2, L))
    ubar, pbar = op.delay_bwd(u, p, w, SLOT, TAPS, SLOT)
    W = 2 + op.DELAY_K
    f_u = lambda uu: np.sum(w * op.delay_fwd(uu.reshape(2, -1), p, SLOT, TAPS, SLOT))
    for i in rng.choice(u.size, 5, replace=False):
        assert np.isclose(ubar.flat[i], fd(f_u, u.reshape(-1), i), rtol=1e-6, atol=1e-8)
    f_p = lambda pp: np.sum(w * op.delay_fwd(u, pp, SLOT, TAPS, SLOT))
    for x, m, k in [(0, 0, 3), (1, 19, 0), (0, 11, 19)]:
        i = (x * TAPS + m) * W + 2 + k
        assert np.isclose(pbar[i], fd(f_p, p, i), rtol=1e-6, atol=1e-8), (x, m, k)
    f_s = lambda pp: np.sum(w * op.delay_fwd_surrogate(u, pp, SLOT, TAPS, SLOT))
    for x, m in [(0, 0), (1, 19), (0, 7)]:
        for c in (0, 1):
            i = (x * TAPS + m) * W + c
            assert np.isclose(pbar[i], fd(f_s, p, i, h=1e-7), rtol=1e-4, atol=1e-6), (x, m, c)


# ------------------------------------------------------------------ reverb, the paper's STFT and masks
HPR = dict(rv_len=1000, rv_nfft=48, rv_hop=24, rv_mode="paper")   # shortened 384 / 192


def rv_params(rng, K=24):
    q = np.zeros((2, 2, K))
    q[:, 0] = rng.uniform(-1, 0, (2, K))
    q[:, 1] = -rng.uniform(0.01, 0.1, (2, K))
    return q.reshape(-1)


def test_paper_masks_follow_eq7_and_drop_nyquist(rng):
    p = rv_params(rng)
    Ms = op.rv_masks(p, 48, 10, mode="paper")
    q = p.reshape(2, 2, 24)
    for x in range(2):
        assert Ms[x].shape == (10, 25)
        np.testing.assert_allclose(np.log(Ms[x][4, :24]), q[x, 0] + 4 * q[x, 1], atol=1e-12)
        assert np.all(Ms[x][:, 24] == 0.0)


def test_paper_ir_brute_force_dft(rng):
    """The IR from explicit DFT sums: per centred frame, the windowed noise's one-sided
    spectrum (direct sum), times exp(H0 + m Hd) on bins 0..K-1 and 0 at Nyquist, the
    one-sided inverse sum, the window again, overlap-add over the frames, division by
    the window envelope, then (mid +- side) / 2."""
    N, hop, Ln = 48, 24, 1000
    K = N // 2
    nz = rng.uniform(-1, 1, (2, Ln))
    p = rv_params(rng)
    q = p.reshape(2, 2, K)
    F = 1 + Ln // hop
    j = np.arange(N)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * j / N)
    hms = []
    for x in range(2):
        acc = np.zeros(Ln)
        env = np.zeros(Ln)
        for m in range(F):
            t = m * hop + j - N // 2
            ok = (t >= 0) & (t < Ln)
            fr = np.zeros(N)
            fr[ok] = nz[x, t[ok]] * w[ok]
            X = [sum(fr[n] * np.exp(-2j * np.pi * k * n / N) for n in range(N)) for k in range(K + 1)]
            Y = [X[k] * np.exp(q[x, 0, k] + m * q[x, 1, k]) if k < K else 0.0 for k in range(K + 1)]
            y = np.array([(Y[0].real + 2 * sum((Y[k] * np.exp(2j * np.pi * k * n / N)).real for k in range(1, K)))
                          / N for n in range(N)])
            acc[t[ok]] += y[ok] * w[ok]
            env[t[ok]] += w[ok] ** 2
        hms.append(acc / env)
    h = op.rv_ir(p, nz, HPR)
    np.testing.assert_allclose(h[0], (hms[0] + hms[1]) / 2, atol=1e-12)
    np.testing.assert_allclose(h[1], (hms[0] - hms[1]) / 2, atol=1e-12)


def test_paper_reverb_is_wet_only(rng):
    nz = rng.uniform(-1, 1, (2, 1000))
    p = rv_params(rng)
    u = np.zeros((2, 700))
    u[:, 0] = 1.0
    y = op.reverb_fwd(u, p, nz, HPR)
    np.testing.assert_allclose(y, op.rv_ir(p, nz, HPR)[:, :700], atol=1e-13)


def test_unit_masks_reconstruct_at_384_192(rng):
    """The paper's STFT size is not a power of two: the pair still reconstructs."""
    nz = rng.uniform(-1, 1, (2, 5000))
    hp = dict(rv_len=5000, rv_nfft=384, rv_hop=192)
    h = op.rv_ir(np.zeros(50), nz, hp)
    np.testing.assert_allclose(h[0] + h[1], nz[0], atol=1e-12)
    np.testing.assert_allclose(h[0] - h[1], nz[1], atol=1e-12)


def test_paper_reverb_gradients_fd(rng):
    nz = rng.uniform(-1, 1, (2, 1000))
    p = rv_params(rng)
    u = rng.standard_normal((2, 300))
    w = rng.standard_normal((2, 300))
    ubar, pbar = op.reverb_bwd(u, p, w, nz, HPR)
    assert pbar.shape == (96,)
    f = lambda pp: np.sum(w * op.reverb_fwd(u, pp, nz, HPR))
    for i in [0, 5, 23, 24, 40, 47, 48, 60, 71, 72, 90, 95]:
        assert np.isclose(pbar[i], fd(f, p, i), rtol=1e-5, atol=1e-9), i
    fu = lambda uu: np.sum(w * op.reverb_fwd(uu.reshape(2, -1), p, nz, HPR))
    for i in rng.choice(600, 5, replace=False):
        assert np.isclose(ubar.flat[i], fd(fu, u.reshape(-1), i), rtol=1e-6, atol=1e-9)


# ------------------------------------------------------------------ whole graphs in the paper's settings
def test_paper_settings_scheduled_equals_one_by_one(rng):
    g = random_dag(rng, 2, 6, kinds=(synth.E, synth.D, synth.R, synth.G))
    types, edges = g.types, g.edges
    P = synth.random_params(g, 5, preset="paper")
    K = types.count(synth.I)
    L = 6000
    src = 0.1 * rng.standard_normal((K, 2, L))
    hp = orr.paper_hp()
    hp["reverb_noise"] = synth.reverb_noise(11)
    Y = orr.render_one_by_one(types, edges, src, P, hp)
    ys, _, _ = orr.render_scheduled(types, edges, src, P, hp)
    np.testing.assert_allclose(ys, orr.outputs_of(types, Y), atol=1e-12)
