"""Pins for the oracle's multitap delay (Sec. 3 "Multitap delay", Eq. 14-15)."""
import numpy as np
import pytest

from oracle import processors as op

NF = 256          # a short surrogate transform keeps the checks fast


def params(rng, nf=NF, on_circle=True):
    p = np.zeros((2, op.DELAY_TAPS, 2 + op.DELAY_K))
    d = rng.integers(1, nf, (2, op.DELAY_TAPS))
    ang = -2 * np.pi * d / nf
    r = 1.0 if on_circle else 0.97
    p[..., 0], p[..., 1] = r * np.cos(ang), r * np.sin(ang)
    p[..., 2:] = rng.uniform(-1.2, 0.2, (2, op.DELAY_TAPS, op.DELAY_K))
    return p.reshape(-1), d


def fd(f, x, i, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_delay_map_and_sparse_fir_brute_force(rng):
    p, d = params(rng)
    z, lm = op.delay_split(p)
    assert np.array_equal(op.delay_samples(z, NF), d)
    u = rng.standard_normal((2, 700))
    y = op.delay_fwd(u, p, NF)
    H = (op.DELAY_FIR - 1) // 2
    want = np.zeros_like(u)
    for x in range(2):
        for m in range(op.DELAY_TAPS):
            c = op.zerophase_taps(lm[x, m], op.DELAY_FIR)
            for j in range(-H, H + 1):
                s = d[x, m] + j
                if s >= 0:
                    want[x, s:] += c[j + H] * u[x, :700 - s]
                else:
                    want[x, :700 + s] += c[j + H] * u[x, -s:]
    np.testing.assert_allclose(y, want, atol=1e-12)


def test_surrogate_is_exact_on_the_unit_circle(rng):
    """Eq. 15 at |z| = 1 with integer phase is the DFT pair of a unit impulse."""
    p, _ = params(rng)
    u = rng.standard_normal((2, 600))
    np.testing.assert_allclose(op.delay_fwd_surrogate(u, p, NF), op.delay_fwd(u, p, NF), atol=1e-10)


def test_delay_gradients_fd(rng):
    p, _ = params(rng)
    u = rng.standard_normal((2, 500))
    w = rng.standard_normal((2, 500))
    ubar, pbar = op.delay_bwd(u, p, w, NF)
    q = pbar.reshape(2, op.DELAY_TAPS, 2 + op.DELAY_K)
    f_u = lambda uu: np.sum(w * op.delay_fwd(uu.reshape(2, -1), p, NF))
    for i in rng.choice(u.size, 8, replace=False):
        assert np.isclose(ubar.flat[i], fd(f_u, u.reshape(-1), i), rtol=1e-6, atol=1e-8)
    # FIR log-magnitudes through the exact forward
    f_p = lambda pp: np.sum(w * op.delay_fwd(u, pp, NF))
    for x, m, k in [(0, 0, 3), (1, 2, 0), (1, 3, 19), (0, 1, 10)]:
        i = (x * op.DELAY_TAPS + m) * (2 + op.DELAY_K) + 2 + k
        assert np.isclose(pbar[i], fd(f_p, p, i), rtol=1e-6, atol=1e-8), (x, m, k)
    # z through the surrogate forward (straight-through estimator)
    f_s = lambda pp: np.sum(w * op.delay_fwd_surrogate(u, pp, NF))
    for x, m in [(0, 0), (1, 3), (0, 2)]:
        for c in (0, 1):
            i = (x * op.DELAY_TAPS + m) * (2 + op.DELAY_K) + c
            assert np.isclose(pbar[i], fd(f_s, p, i, h=1e-7), rtol=1e-4, atol=1e-6), (x, m, c)
