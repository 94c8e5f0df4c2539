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
The paper's own settings (preset "paper", widths in ``types.PAPER_PARAM_COLS``):
  e: 1024 ln-magnitudes (bin k at k fs / 2047 Hz) of a smooth random curve: 8 gains
     U(-12, 12) dB at log-spaced centres 20 * 1000^((b+0.5)/8) Hz, each a Gaussian
     bump of 0.6 octaves in log2 frequency
  d: per channel 20 taps, tap m at m * 100 ms + U{0 .. 100 ms - 1 sample} placed on
     the unit circle of its slot, z = exp(-2 pi j d' / 4410); ln-magnitudes from
     U(-30, -12) dB
  r: per bin H0 from a smooth random curve around -36 dB (+-6 dB), H_delta the
     per-frame ln decay (hop 192) of a smooth random RT60 curve in 0.3 .. 1.5 s
"""
import numpy as np

from .types import G, S, E, C, D, R, N, K, A, PARAM_COLS, param_cols

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
    if t == K:
        # sidechain compressor: the compressor's distributions
        return _rows(rng, C, n, fs)
    if t == A:
        # attack/release: a fast attack U(0.5, 0.99), a slow release U(0.999, 0.9999), the
        # compressor's T, W, R
        q = _rows(rng, C, n, fs)
        p = np.empty((n, 5))
        p[:, 0] = rng.uniform(0.5, 0.99, n)
        p[:, 1] = rng.uniform(0.999, 0.9999, n)
        p[:, 2:] = q[:, 1:]
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


def _smooth_curve(rng, n, freqs, lo, hi):
    """[n, len(freqs)] random smooth curves in dB: 8 gains U(lo, hi) at log-spaced
    centres, each a Gaussian bump of 0.6 octaves in log2 frequency."""
    cb = np.log2(20.0 * 1000.0 ** ((np.arange(8) + 0.5) / 8))
    lf = np.log2(np.maximum(freqs, 10.0))
    bumps = np.exp(-0.5 * ((lf[None, :] - cb[:, None]) / 0.6) ** 2)   # [8, K]
    return rng.uniform(lo, hi, (n, 8)) @ bumps


def _rows_paper(rng, t, n, fs=44100):
    if t == E:
        K = 1024
        return _db_amp_ln(_smooth_curve(rng, n, np.arange(K) * fs / 2047.0, -12, 12))
    if t == D:
        taps, slot = 20, fs // 10
        p = np.empty((n, 2, taps, 2 + DELAY_MAGS))
        d = rng.integers(0, slot, (n, 2, taps))
        ang = -2 * np.pi * d / slot
        p[..., 0] = np.cos(ang)
        p[..., 1] = np.sin(ang)
        p[..., 2:] = _db_amp_ln(rng.uniform(-30, -12, (n, 2, taps, DELAY_MAGS)))
        return p.reshape(n, -1)
    if t == R:
        K, hop = 192, 192
        f = np.arange(K) * fs / 384.0
        h0 = _db_amp_ln(-36.0 + _smooth_curve(rng, 2 * n, f, -6, 6)).reshape(n, 2, K)
        rt60 = np.clip(0.9 + 0.1 * _smooth_curve(rng, 2 * n, f, -6, 6), 0.3, 1.5).reshape(n, 2, K)
        hd = -3.0 * LN10 * hop / (rt60 * fs)
        return np.stack([h0, hd], axis=2).reshape(n, 4 * K)
    return _rows(rng, t, n, fs)


def random_params(graph, seed: int, preset="compact"):
    """Dict type -> float32 [|V_t|, N_t] for every parameterised type in ``graph``."""
    cols = param_cols(preset)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for t in sorted(set(graph.types)):
        if cols[t] == 0:
            continue
        n = graph.types.count(t)
        rows = _rows_paper(rng, t, n) if preset == "paper" else _rows(rng, t, n)
        out[t] = rows.astype(np.float32)
    return out


def union_params(graphs, seed: int, preset="compact"):
    """One table per type over a batch of graphs (the union's original order: graph by
    graph), graph k's rows drawn by ``random_params(graphs[k], seed + k)``."""
    tabs = {}
    for k, g in enumerate(graphs):
        for t, a in random_params(g, seed + k, preset=preset).items():
            tabs.setdefault(t, []).append(a)
    return {t: np.concatenate(v) for t, v in tabs.items()}


def neutral_params(graph, preset="compact"):
    """Parameters that make g, s, e and c (nearly) transparent: 0 dB gains, flat EQ,
    ratio 1; reverb fully dry (compact) or a short quiet tail (paper: no dry path);
    delay keeps drawn-free quiet taps near the start of each slot."""
    cols = param_cols(preset)
    out = {}
    for t in sorted(set(graph.types)):
        n = graph.types.count(t)
        if cols[t] == 0:
            continue
        p = np.zeros((n, cols[t]))
        if t == A:
            p[:, 0], p[:, 1], p[:, 3], p[:, 4] = 0.9, 0.999, 3.0 * LN10 / 10.0, 1.0
        if t in (C, N, K):
            p[:, 0] = 0.99
            p[:, 2] = 3.0 * LN10 / 10.0
            p[:, 3] = 1.0
        if t == D:
            taps = cols[D] // (2 * (2 + DELAY_MAGS))
            nf = 4410 if preset == "paper" else DELAY_FFT
            q = p.reshape(n, 2, taps, 2 + DELAY_MAGS)
            ang = -2 * np.pi * 44 / nf
            q[..., 0] = np.cos(ang)
            q[..., 1] = np.sin(ang)
            q[..., 2:] = np.log(1.0 / taps)
        if t == R:
            if preset == "paper":
                q = p.reshape(n, 2, 2, 192)
                q[:, :, 0] = _db_amp_ln(-36.0)
                q[:, :, 1] = -3.0 * LN10 * 192 / (0.5 * 44100)
            else:
                p[:, 24:48] = -0.05
                p[:, 49] = -30.0
        out[t] = p.astype(np.float32)
    return out
