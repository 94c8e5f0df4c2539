"""Seeded physical processor parameters, one float32 table per type.

Rows follow the original node order of each type (Sec. 2: the l-th row of P[t]
belongs to the l-th type-t node of T_V).  Distributions:
  g: ln-gain per channel from U(-6, 6) dB
  s: U(-1, 1)
  e: 8 band gains U(-12, 12) dB
  c: alpha U(0.9, 0.9999); T from U(-40, 0) dB (energy, natural-log units);
     W = 3 dB (0.6908 ln units); R U(1, 8)
  d: per channel and tap, an integer delay U{1 ms .. 500 ms} placed on the unit
     circle as z = exp(-2 pi j d / 32768); 20 ln-magnitudes from U(-12, 0) dB
  r: H0 from U(-6, 0) dB per band; H_delta a per-frame ln decay from an RT60
     U(0.3, 1.5) s at hop 256 / 44.1 kHz; q_dry U(-1, 0), q_wet U(-3, -1)
"""
import numpy as np

from .types import G, S, E, C, D, R, N, PARAM_COLS

LN10 = np.log(10.0)
DELAY_FFT = 32768
DELAY_TAPS = 4
DELAY_MAGS = 20
REVERB_BANDS = 12


def _db_amp_ln(db):
    return db * LN10 / 20.0


def _rows(rng, t, n, fs=44100):
    if t == G:
        return _db_amp_ln(rng.uniform(-6, 6, (n, 2)))
    if t == S:
        return rng.uniform(-1, 1, (n, 1))
    if t == E:
        return rng.uniform(-12, 12, (n, 8))
    if t == C:
        p = np.empty((n, 4))
        p[:, 0] = rng.uniform(0.9, 0.9999, n)
        p[:, 1] = rng.uniform(-40, 0, n) * LN10 / 10.0
        p[:, 2] = 3.0 * LN10 / 10.0
        p[:, 3] = rng.uniform(1, 8, n)
        return p
    if t == N:
        # noisegate: threshold -60..-30 dB, expansion ratio 1..4, W = 3 dB
        p = np.empty((n, 4))
        p[:, 0] = rng.uniform(0.9, 0.9999, n)
        p[:, 1] = rng.uniform(-60, -30, n) * LN10 / 10.0
        p[:, 2] = 3.0 * LN10 / 10.0
        p[:, 3] = rng.uniform(1, 4, n)
        return p
    if t == D:
        p = np.empty((n, 2, DELAY_TAPS, 2 + DELAY_MAGS))
        d = rng.integers(int(0.001 * fs), int(0.5 * fs) + 1, (n, 2, DELAY_TAPS))
        ang = -2 * np.pi * d / DELAY_FFT
        p[..., 0] = np.cos(ang)
        p[..., 1] = np.sin(ang)
        p[..., 2:] = _db_amp_ln(rng.uniform(-12, 0, (n, 2, DELAY_TAPS, DELAY_MAGS)))
        return p.reshape(n, -1)
    if t == R:
        p = np.empty((n, 50))
        h0 = _db_amp_ln(rng.uniform(-6, 0, (n, 2, REVERB_BANDS)))
        rt60 = rng.uniform(0.3, 1.5, (n, 2, REVERB_BANDS))
        hd = -3.0 * LN10 * 256.0 / (rt60 * fs)
        p[:, :48] = np.stack([h0, hd], axis=2).reshape(n, 48)
        p[:, 48] = rng.uniform(-1, 0, n)
        p[:, 49] = rng.uniform(-3, -1, n)
        return p
    raise ValueError(t)


def random_params(graph, seed: int):
    """Dict type -> float32 [|V_t|, N_t] for every parameterised type in ``graph``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for t in sorted(set(graph.types)):
        if PARAM_COLS[t] == 0:
            continue
        out[t] = _rows(rng, t, graph.types.count(t)).astype(np.float32)
    return out


def neutral_params(graph):
    """Parameters that make g, s, e and c (nearly) transparent: 0 dB gains, flat EQ,
    ratio 1; reverb fully dry; delay keeps drawn-free unit taps at 1 ms."""
    out = {}
    for t in sorted(set(graph.types)):
        n = graph.types.count(t)
        if PARAM_COLS[t] == 0:
            continue
        p = np.zeros((n, PARAM_COLS[t]))
        if t in (C, N):
            p[:, 0] = 0.99
            p[:, 2] = 3.0 * LN10 / 10.0
            p[:, 3] = 1.0
        if t == D:
            q = p.reshape(n, 2, DELAY_TAPS, 2 + DELAY_MAGS)
            ang = -2 * np.pi * 44 / DELAY_FFT
            q[..., 0] = np.cos(ang)
            q[..., 1] = np.sin(ang)
            q[..., 2:] = np.log(0.25)
        if t == R:
            p[:, 24:48] = -0.05
            p[:, 49] = -30.0
        out[t] = p.astype(np.float32)
    return out
