"""Pins for the oracle's filtered-noise reverb (Sec. 3 "Reverb", Eq. 6-7), on reduced
STFT sizes so that brute force and finite differences stay cheap."""
import numpy as np
import pytest

from oracle import processors as op

HP = dict(rv_len=1500, rv_nfft=64, rv_hop=16)


def noise(rng, n=1500):
    return rng.uniform(-1, 1, (2, n))


def params(rng):
    p = np.zeros(50)
    p[0:12] = rng.uniform(-1, 0, 12)
    p[12:24] = -rng.uniform(0.01, 0.1, 12)
    p[24:36] = rng.uniform(-1, 0, 12)
    p[36:48] = -rng.uniform(0.01, 0.1, 12)
    p[48], p[49] = -0.3, -1.5
    return p


def test_unit_mask_reconstructs_the_noise(rng):
    nz = noise(rng)
    h = op.rv_ir(np.zeros(50), nz, HP)
    hm, hs = h[0] + h[1], h[0] - h[1]
    D = op.rv_ola_norm(1500, 64, 16)
    assert D.min() > 0.5                      # centred frames: the envelope is bounded below
    np.testing.assert_allclose(hm, nz[0], atol=1e-12)
    np.testing.assert_allclose(hs, nz[1], atol=1e-12)


def test_stft_matches_direct_dft(rng):
    x = rng.standard_normal(200)
    S = op.rv_stft(x, 32, 8)
    w = op.rv_window(32)
    n = np.arange(32)
    xp = np.zeros((S.shape[0] - 1) * 8 + 32)
    xp[16:216] = x                            # centred frames: N/2 zeros before the signal
    assert S.shape[0] == 1 + 200 // 8
    for m in (0, 5, S.shape[0] - 1):
        fr = xp[m * 8:m * 8 + 32] * w
        for k in (0, 3, 16):
            assert abs(S[m, k] - np.sum(fr * np.exp(-2j * np.pi * k * n / 32))) < 1e-12


def test_masks_follow_eq7(rng):
    p = params(rng)
    Ms = op.rv_masks(p, 64, 10)
    B = op.rv_band_matrix(64)
    np.testing.assert_allclose(np.log(Ms[1][3]), B @ p[24:36] + 3 * (B @ p[36:48]), atol=1e-12)


def test_dry_limit_and_brute_force_convolution(rng):
    nz = noise(rng)
    p = params(rng)
    u = rng.standard_normal((2, 120))
    y = op.reverb_fwd(u, p, nz, HP)
    h = op.rv_ir(p, nz, HP)
    want = np.exp(p[48]) * u.copy()
    for x in range(2):
        for t in range(120):
            want[x, t] += np.exp(p[49]) * sum(h[x, n] * u[x, t - n] for n in range(t + 1))
    np.testing.assert_allclose(y, want, atol=1e-11)
    p2 = p.copy()
    p2[49] = -60.0
    np.testing.assert_allclose(op.reverb_fwd(u, p2, nz, HP), np.exp(p[48]) * u, atol=1e-20)


def test_reverb_gradients_fd(rng):
    nz = noise(rng)
    p = params(rng)
    u = rng.standard_normal((2, 300))
    w = rng.standard_normal((2, 300))
    ubar, pbar = op.reverb_bwd(u, p, w, nz, HP)
    f = lambda pp: np.sum(w * op.reverb_fwd(u, pp, nz, HP))
    for i in [0, 5, 11, 12, 17, 23, 24, 30, 40, 47, 48, 49]:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        assert np.isclose(pbar[i], (f(pp) - f(pm)) / (2 * h), rtol=1e-5, atol=1e-9), i
    fu = lambda uu: np.sum(w * op.reverb_fwd(uu.reshape(2, -1), p, nz, HP))
    for i in rng.choice(600, 6, replace=False):
        uu, um = u.reshape(-1).copy(), u.reshape(-1).copy()
        uu[i] += 1e-6
        um[i] -= 1e-6
        assert np.isclose(ubar.flat[i], (fu(uu) - fu(um)) / 2e-6, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("n", [64, 384, 1024])
def test_stft_window_is_the_periodic_hann_window(n):
    """The reverb's STFT window is the periodic Hann window (scipy's 'hann' with
    fftbins): unit-mask reconstruction alone would hold for any window, since the
    overlap-add divides by the window envelope."""
    import scipy.signal
    np.testing.assert_allclose(op.rv_window(n), scipy.signal.get_window("hann", n, fftbins=True),
                               rtol=0, atol=1e-15)


def test_band_filters_are_linear_in_log_frequency():
    """Band log-magnitudes that are linear in log2 f come back exactly at every bin
    between the first and last band centre and hold the end bands' values beyond them."""
    n, fs = 1024, 44100
    c = 20.0 * 1000.0 ** ((np.arange(op.RV_BANDS) + 0.5) / op.RV_BANDS)
    a, slope = 0.4, -0.9
    got = op.rv_band_matrix(n, fs) @ (a + slope * np.log2(c))
    f = np.arange(n // 2 + 1) * fs / n
    inner = (f > c[0]) & (f < c[-1])
    np.testing.assert_allclose(got[inner], a + slope * np.log2(f[inner]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[f <= c[0]], a + slope * np.log2(c[0]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[f >= c[-1]], a + slope * np.log2(c[-1]), rtol=0, atol=1e-12)
