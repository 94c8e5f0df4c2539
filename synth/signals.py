"""Seeded synthetic stereo source tracks (the stand-in for multitrack stems).

Each track is pink noise (white Gaussian shaped by 1/sqrt(f) in the rFFT domain),
independent per channel, multiplied by an envelope: a constant bed of 0.05
(about -26 dB below a unit note; recorded stems carry room tone and bleed, so
they are never digitally silent) plus a sum of notes with Poisson onsets at
2 notes/s, amplitude U(0.3, 1) and decay exp(-t/tau), tau ~ U(0.05, 1.0) s.
Each track is scaled to a peak of 0.5/sqrt(K) for K tracks so that mixes stay
near full scale.
"""
import numpy as np


def _pink(rng, n):
    w = rng.standard_normal(n)
    spec = np.fft.rfft(w)
    f = np.arange(spec.shape[0], dtype=np.float64)
    f[0] = 1.0
    spec = spec / np.sqrt(f)
    spec[0] = 0.0
    return np.fft.irfft(spec, n)


NOISE_BED = 0.05


def _envelope(rng, n, fs):
    env = np.full(n, NOISE_BED)
    dur = n / fs
    n_notes = max(1, int(rng.poisson(2.0 * dur)))
    t = np.arange(n) / fs
    for _ in range(n_notes):
        onset = rng.uniform(0.0, dur)
        amp = rng.uniform(0.3, 1.0)
        tau = rng.uniform(0.05, 1.0)
        k0 = int(onset * fs)
        env[k0:] += amp * np.exp(-(t[k0:] - t[k0]) / tau)
    return env


def sources(seed: int, K: int, L: int, fs: int = 44100, pitch: int = None) -> np.ndarray:
    """K stereo tracks of L samples as float32 ``[K, 2, pitch]`` (pitch >= L, tail zero)."""
    if pitch is None:
        pitch = L
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((K, 2, pitch), dtype=np.float32)
    peak = 0.5 / np.sqrt(max(K, 1))
    for k in range(K):
        env = _envelope(rng, L, fs)
        x = np.stack([_pink(rng, L), _pink(rng, L)]) * env[None, :]
        m = np.max(np.abs(x))
        if m > 0:
            x = x * (peak / m)
        out[k, :, :L] = x.astype(np.float32)
    return out


def reverb_noise(seed: int = 8, length: int = 88200) -> np.ndarray:
    """The two uniform noise buffers (mid, side) of the filtered-noise reverb, U(-1, 1),
    float32 [2, length] (2 s at 44.1 kHz by default)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, (2, length)).astype(np.float32)
