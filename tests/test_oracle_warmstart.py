"""Pins for the oracle's warm-start network: parameter count, mel features on tones,
and the analytic backward pass against central finite differences."""
import numpy as np
import pytest

from oracle import warmstart as ow


def test_parameter_count_about_1p2m():
    assert 1.15e6 < ow.n_params() < 1.25e6


def test_mel_filterbank_shape_and_partition():
    W = ow.mel_filterbank()
    assert W.shape == (128, 1025)
    assert W.max() <= 1.0 + 1e-12
    # adjacent triangles overlap to a partition of unity between the first and last centre
    s = W.sum(axis=0)
    c = ow.mel_to_hz(np.linspace(0, ow.hz_to_mel(22050), 130))
    f = np.arange(1025) * 44100 / 2048
    inner = (f > c[1]) & (f < c[-2])
    np.testing.assert_allclose(s[inner], 1.0, atol=1e-12)


def test_logmel_of_a_tone_peaks_at_its_band():
    t = np.arange(20000) / 44100
    for f0 in (300.0, 2500.0, 9000.0):
        x = np.stack([np.sin(2 * np.pi * f0 * t)] * 2)
        lm = ow.logmel(x)
        band = int(np.argmax(lm.mean(axis=1)))
        c = ow.mel_to_hz(np.linspace(0, ow.hz_to_mel(22050), 130))[1:-1]
        assert abs(np.log(c[band] / f0)) < 0.15, (f0, c[band])


def test_backward_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(3))
    flat = ow.init_params(1)
    feats = rng.standard_normal((256, 12))
    for t in (6, 7):
        out, cache = ow.forward(flat, feats, t)
        d = rng.standard_normal(out.shape[0])
        g = ow.backward(flat, cache, t, d)
        shapes = ow.param_shapes()
        offs = np.cumsum([0] + [int(np.prod(s)) for _, s in shapes])
        names = [n for n, _ in shapes]
        picks = []
        for name in ("conv0.w", "conv0.b", "conv3.w", f"h{t}.w1", f"h{t}.b2", f"h{t}.w3", f"h{t}.b3"):
            i = names.index(name)
            picks += list(rng.integers(offs[i], offs[i + 1], 3))
        for i in picks:
            h = 1e-5
            fp, fm = flat.copy(), flat.copy()
            fp[i] += h
            fm[i] -= h
            num = (d @ ow.forward(fp, feats, t)[0] - d @ ow.forward(fm, feats, t)[0]) / (2 * h)
            assert np.isclose(g[i], num, rtol=1e-5, atol=1e-8), (names, i)


def test_bf16_round_ties_to_even_and_matches_torch():
    import torch
    one = 1.0
    # 1 + 2^-8 is half an ulp of bfloat16 at 1: ties go to the even neighbour 1.0;
    # 1 + 3*2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert ow.bf16_round(np.float32(one + 2.0 ** -8)) == 1.0
    assert ow.bf16_round(np.float32(one + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    assert ow.bf16_round(np.float32(one + 2.0 ** -8 + 2.0 ** -20)) == 1.0 + 2.0 ** -7
    assert ow.bf16_round(np.float32(-3.0)) == -3.0
    rng = np.random.Generator(np.random.PCG64(11))
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-60, 60, 200000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ow.bf16_round(x), ref)


def test_conv1d_is_cross_correlation_with_zero_padding():
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.standard_normal((3, 9))
    w = rng.standard_normal((2, 3, 5))
    b = rng.standard_normal(2)
    y = ow.conv1d(x, w, b)
    for o in range(2):
        want = b[o] + sum(np.correlate(np.pad(x[c], 2), w[o, c], mode="valid") for c in range(3))
        np.testing.assert_allclose(y[o], want, rtol=1e-12, atol=1e-12)


def test_masked_mse_brute_force():
    rng = np.random.Generator(np.random.PCG64(6))
    out, tgt = rng.standard_normal((4, 176)), rng.standard_normal((4, 176))
    n_out = [2, 176, 8, 50]
    loss, d = ow.masked_mse(out, tgt, n_out)
    per = []
    for i, n in enumerate(n_out):
        per.append(sum((out[i, j] - tgt[i, j]) ** 2 for j in range(n)) / n)
    assert np.isclose(loss, sum(per) / 4, rtol=1e-13)
    for i, n in enumerate(n_out):
        np.testing.assert_allclose(d[i, :n], 2 * (out[i, :n] - tgt[i, :n]) / (4 * n), rtol=1e-13)
        assert not d[i, n:].any()
    # central differences of the loss in a few coordinates
    for i, j in ((0, 1), (1, 100), (3, 49)):
        h = 1e-6
        op, om = out.copy(), out.copy()
        op[i, j] += h
        om[i, j] -= h
        num = (ow.masked_mse(op, tgt, n_out)[0] - ow.masked_mse(om, tgt, n_out)[0]) / (2 * h)
        assert np.isclose(d[i, j], num, rtol=1e-6)


def test_logmel_parseval_and_pooling():
    rng = np.random.Generator(np.random.PCG64(8))
    L = 2048 + 3 * 512 + 100                      # 4 frames, fewer than the 32 pooled slots
    x = rng.standard_normal((2, L)) * 0.1
    lm = ow.logmel(x)
    m = 0.5 * (x[0] + x[1])
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(2048) / 2048)
    W = ow.mel_filterbank()
    frames = []
    for f in range(4):
        seg = m[f * 512:f * 512 + 2048] * w
        # direct DFT of the one-sided bins; Parseval over the full spectrum
        k = np.arange(1025)[:, None]
        X = (seg[None, :] * np.exp(-2j * np.pi * k * np.arange(2048)[None, :] / 2048)).sum(axis=1)
        P = np.abs(X) ** 2
        full = P.sum() + P[1:1024].sum()
        assert np.isclose(full, 2048 * (seg ** 2).sum(), rtol=1e-10)
        frames.append(np.log(W @ P + 1e-5))
    frames = np.array(frames)
    # 4 frames over 32 slots: slot i averages frame floor(4 i / 32) alone
    for i in range(32):
        np.testing.assert_allclose(lm[:, i], frames[(4 * i) // 32], rtol=1e-9, atol=1e-9)


def test_backward_all_heads_finite_differences():
    rng = np.random.Generator(np.random.PCG64(9))
    flat = ow.init_params(2)
    feats = rng.standard_normal((256, 6))
    shapes = ow.param_shapes()
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in shapes])
    names = [n for n, _ in shapes]
    for t in (3, 4, 5, 8):
        out, cache = ow.forward(flat, feats, t)
        d = rng.standard_normal(out.shape[0])
        g = ow.backward(flat, cache, t, d)
        # the other heads get exactly zero gradient
        for u in ow.HEAD_TYPES:
            if u != t:
                i = names.index(f"h{u}.w1")
                assert not g[offs[i]:offs[i + 6]].any()
        for name in ("conv1.w", "conv2.b", f"h{t}.w2", f"h{t}.b1", f"h{t}.w3"):
            i = names.index(name)
            for j in rng.integers(offs[i], offs[i + 1], 2):
                h = 1e-5
                fp, fm = flat.copy(), flat.copy()
                fp[j] += h
                fm[j] -= h
                num = (d @ ow.forward(fp, feats, t)[0] - d @ ow.forward(fm, feats, t)[0]) / (2 * h)
                assert np.isclose(g[j], num, rtol=1e-5, atol=1e-8), (name, j)


def _stereo(rng, L):
    return rng.standard_normal((2, L))


def test_xgain_of_a_scaled_copy_is_the_scale(rng):
    # target = a * u on both channels: every band's gain is a (mid and side)
    u = _stereo(rng, 2 ** 14)
    for a in (0.25, 1.0, 3.0):
        np.testing.assert_allclose(ow.xgain(u, a * u), np.log(a + ow.XG_FLOOR), rtol=1e-12, atol=1e-12)
    # a phase-inverted copy has a negative gain, floored
    np.testing.assert_allclose(ow.xgain(u, -u), np.log(ow.XG_FLOOR), rtol=1e-12)


def test_xgain_separates_mid_and_side(rng):
    # an imager-like target: mid kept, side scaled by b (Eq. 3 keeps the mid)
    u = _stereo(rng, 2 ** 14)
    b = 0.4
    mid, side = 0.5 * (u[0] + u[1]), 0.5 * (u[0] - u[1])
    T = np.stack([mid + b * side, mid - b * side])
    f = ow.xgain(u, T)
    np.testing.assert_allclose(f[:ow.XG_BANDS], np.log(1.0 + ow.XG_FLOOR), rtol=1e-12)
    np.testing.assert_allclose(f[ow.XG_BANDS:], np.log(b + ow.XG_FLOOR), rtol=1e-12)


def test_xgain_ignores_an_independent_source(rng):
    # the node's path plus an independent track: the estimate tends to the path's gain
    L = 2 ** 17
    u, n = _stereo(rng, L), _stereo(rng, L)
    f = ow.xgain(u, 2.0 * u + n)
    # wide high bands average many bins and frames: close to ln(2.01)
    assert abs(np.median(f[40:64]) - np.log(2.0 + ow.XG_FLOOR)) < 0.05


def test_xgain_sums_against_a_direct_dft(rng):
    # one frame, one band pair, computed with explicit DFT sums
    L = ow.MEL_NFFT
    u, T = _stereo(rng, L), _stereo(rng, L)
    f = ow.xgain(u, T, T_slots=1)
    n = np.arange(L)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * n / L)
    W = ow.mel_filterbank()
    um, tm = 0.5 * (u[0] + u[1]) * w, 0.5 * (T[0] + T[1]) * w
    k = np.arange(L // 2 + 1)
    E = np.exp(-2j * np.pi * np.outer(k, n) / L)
    U, Y = E @ um, E @ tm
    band = 10
    C = (W[2 * band] + W[2 * band + 1]) @ np.real(Y * np.conj(U))
    P = (W[2 * band] + W[2 * band + 1]) @ np.abs(U) ** 2
    assert abs(f[band, 0] - np.log(max(C / P, 0.0) + ow.XG_FLOOR)) < 1e-10
