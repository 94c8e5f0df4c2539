"""Warm-start network on the GPU against the FP64 oracle (oracle/warmstart.py).

Tolerances, derived from the arithmetic:
* BF16 GEMM against the float64 product of the same BF16-rounded operands: only the
  float32 accumulation differs, |err| <= K 2^-22 sum_k |a_k b_k| (a worst-case bound
  with a factor 2 for truncating accumulation).
* Network against the exact float64 oracle: each product rounds both operands to 8
  significant bits (relative error up to 2^-9 each, about 2^-9 sqrt(2) = 2.8e-3 per layer
  for sums of random sign), compounded over 7 layers forward (sqrt(7) x 2.8e-3 = 7e-3)
  and the longer backward chain: 2e-2 normwise per tensor, cosine >= 0.9995.
* Network against the oracle with the same BF16 operand rounding: the two sides round
  float32 and float64 intermediates, which differ by the float32 error delta (1e-6 after
  the first product); an operand rounds differently with probability ~2 delta / 2^-8 and
  then moves by 2^-8, so the next layer differs by ~sqrt(4 delta 2^8) 2^-8 = sqrt(delta)/8
  (1e-6 -> 1.3e-4 -> 1.4e-3 -> ...), capped by the rounding error itself: 1e-2 normwise.
* Log-mel: float32 FFT error per bin is at most ~u log2(N) sqrt(N) ||x_w||, which moves
  ln(mel + 1e-5) by at most 2 sqrt(mel) delta / (mel + 1e-5); the test evaluates that
  bound per frame (with the packed partner frame's energy) and pools it.
"""
import numpy as np
import pytest

import synth
from oracle import warmstart as ow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2408_03204_b300 as gx
    return gx, torch


def _bf16_gemm_ref(A, B):
    Ar, Br = ow.bf16_round(A), ow.bf16_round(B)
    return Ar @ Br, np.abs(Ar) @ np.abs(Br)


@pytest.mark.parametrize("M,N,K,ta,tb,split", [(1, 1, 1, 0, 0, 0), (70, 130, 45, 0, 0, 0), (64, 64, 32, 1, 0, 0),
                                               (129, 65, 1280, 0, 1, 0), (200, 288, 3, 1, 1, 0),
                                               (5, 176, 288, 0, 1, 0), (128, 640, 4096, 1, 0, 1),
                                               (130, 260, 2000, 1, 1, 1), (257, 129, 999, 0, 0, 1)])
def test_gemm_bf16_matches_rounded_product(env, M, N, K, ta, tb, split):
    gx, torch = env
    rng = np.random.Generator(np.random.PCG64(M * 1000 + N + K))
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    # A stored as [M][K] (ta=0) or [K][M] (ta=1); B as [K][N] (tb=0) or [N][K] (tb=1)
    Ad = torch.tensor(A.T.copy() if ta else A, device="cuda")
    Bd = torch.tensor(B.T.copy() if tb else B, device="cuda")
    sam, sak = (1, M) if ta else (K, 1)
    sbk, sbn = (1, K) if tb else (N, 1)
    C = torch.tensor(C0, device="cuda")
    scratch = torch.empty(64 * M * N, device="cuda") if split else None
    gx.gemm_bf16_raw(M, N, K, Ad, sam, sak, Bd, sbk, sbn, C, N, 0.5, 2.0, gx._stream(torch, C.device), scratch)
    torch.cuda.synchronize()
    want, mag = _bf16_gemm_ref(A, B)
    want = 0.5 * want + 2.0 * C0.astype(np.float64)
    err = np.abs(C.cpu().numpy() - want)
    bound = K * 2.0 ** -22 * 0.5 * mag + 2.0 ** -22 * (0.5 * mag + 2.0 * np.abs(C0)) + 1e-30
    assert (err <= bound).all(), float((err / bound).max())


def test_gemm_bf16_rejects_bad_shapes(env):
    gx, torch = env
    a = torch.zeros(4, device="cuda")
    with pytest.raises(gx.GrafxError):
        gx.gemm_bf16_raw(2, 2, 1, a, 1, 1, a, 1, 1, a, 1, 1.0, 0.0, gx._stream(torch, a.device))


def _logmel_bound(x):
    """Per-(band, slot) bound on |ln(mel_gpu + eps) - ln(mel_ref + eps)| for a [2, L] row."""
    m = 0.5 * (x[0].astype(np.float64) + x[1].astype(np.float64))
    F = 1 + (m.shape[0] - 2048) // 512
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(2048) / 2048)
    W = ow.mel_filterbank()
    seg = np.stack([m[f * 512:f * 512 + 2048] * w for f in range(F)])
    P = np.abs(np.fft.rfft(seg, axis=-1)) ** 2
    mel = P @ W.T
    e = (seg ** 2).sum(axis=1)
    partner = np.array([e[f ^ 1] if (f ^ 1) < F else 0.0 for f in range(F)])
    delta = 8 * 2.0 ** -24 * 11 * np.sqrt(2048) * np.sqrt(e + partner)
    per = 2 * np.sqrt(mel) * delta[:, None] / (mel + 1e-5) + 4 * 2.0 ** -24 * np.abs(np.log(mel + 1e-5)) + 1e-6
    out = np.zeros((128, 32))
    for i in range(32):
        a, b = (i * F) // 32, ((i + 1) * F) // 32
        out[:, i] = per[a:max(b, a + 1)].mean(axis=0)
    return out


@pytest.mark.parametrize("L", [2048, 2048 + 511, 2048 + 512, 44100, 65536 + 1000])
def test_logmel_matches_oracle(env, L):
    gx, torch = env
    n_rows = 3
    P = (L + 3) // 4 * 4
    src = synth.sources(40 + L % 97, n_rows, L, pitch=P)          # [rows, 2, P]
    src[1] *= 1e-3                                                  # a quiet row
    src[2, :, L // 3: L // 2] = 0.0                                 # digital silence in part
    net = gx.WarmStartNet(max_batch=4, max_rows=n_rows, max_len=L)
    rows = torch.tensor(src.reshape(-1), device="cuda")
    feats = torch.full((n_rows, 256, 32), float("nan"), device="cuda")
    st = gx._stream(torch, rows.device)
    net.logmel_raw(rows, n_rows, 2 * P, P, L, None, n_rows, 0, feats, st)
    # mix rows broadcast to samples through a row map (sample i takes row map[i])
    rmap = torch.tensor([2, 0, 1], dtype=torch.int32, device="cuda")
    net.logmel_raw(rows, n_rows, 2 * P, P, L, rmap, n_rows, 128, feats, st)
    torch.cuda.synchronize()
    got = feats.cpu().numpy()
    for r in range(n_rows):
        x = src[r, :, :L]
        want = ow.logmel(x)
        bound = _logmel_bound(x)
        err = np.abs(got[r, :128] - want)
        assert (err <= bound).all(), (r, float((err / bound).max()), float(err.max()))
        r2 = [2, 0, 1][r]
        np.testing.assert_array_equal(got[r, 128:], got[r2, :128])


@pytest.mark.parametrize("L", [2048, 44100 + 3])
def test_xgain_matches_oracle(env, L):
    """Cross-spectral band gain of node inputs against target rows through a row map:
    an exact copy at -6 dB, a filtered copy plus an independent track, and a sample whose
    target index is out of range (zero target)."""
    gx, torch = env
    P = (L + 3) // 4 * 4
    u = synth.sources(70 + L % 13, 3, L, pitch=P)                    # node inputs [3, 2, P]
    other = synth.sources(90, 1, L, pitch=P)[0]
    T = np.zeros((2, 2, P), np.float32)
    T[0] = 0.5 * u[0]
    k = np.array([0.5, 0.3, 0.2])                                     # a short FIR on sample 1's input
    for ch in range(2):
        T[1, ch, :L] = np.convolve(u[1, ch, :L], k)[:L] + other[ch, :L]
    rmap = [0, 1, 7]
    net = gx.WarmStartNet(max_batch=4, max_rows=8, max_len=L)
    ud = torch.tensor(u.reshape(-1), device="cuda")
    td = torch.tensor(T.reshape(-1), device="cuda")
    feats = torch.full((3, 256, 32), float("nan"), device="cuda")
    rm = torch.tensor(rmap, dtype=torch.int32, device="cuda")
    st = gx._stream(torch, ud.device)
    net.xgain_raw(ud, 3, 2 * P, td, 2, 2 * P, rm, P, L, 128, feats, st)
    torch.cuda.synchronize()
    got = feats.cpu().numpy()[:, 128:]
    for i, r in enumerate(rmap):
        tgt = T[r, :, :L] if r < 2 else np.zeros((2, L))
        want = ow.xgain(u[i, :, :L], tgt)
        # FP32 spectra: the ratio of two band sums to about 1e-5, at most 1e-3 after the log
        np.testing.assert_allclose(got[i], want, rtol=0, atol=1e-3, err_msg=f"sample {i}")
    np.testing.assert_allclose(got[0], np.log(0.5 + ow.XG_FLOOR), atol=1e-4)
    np.testing.assert_allclose(got[2], np.log(ow.XG_FLOOR), rtol=0, atol=1e-5)   # FP32 logf


def test_logmel_rejects_short_rows_and_small_workspace(env):
    gx, torch = env
    net = gx.WarmStartNet(max_batch=2, max_rows=1, max_len=4096)
    rows = torch.zeros(2 * 8192 * 2, device="cuda")
    feats = torch.zeros(2, 256, 32, device="cuda")
    st = gx._stream(torch, rows.device)
    with pytest.raises(gx.GrafxError):
        net.logmel_raw(rows, 1, 4096, 2048, 2047, None, 1, 0, feats, st)
    with pytest.raises(gx.GrafxError):      # 2 rows of 8192 need more frame scratch than bound
        net.logmel_raw(rows, 2, 16384, 8192, 8192, None, 2, 0, feats, st)


HEADS = ow.HEAD_TYPES


def _batch(seed, counts):
    """Weights, features and d_out for a batch sorted by head (counts per head)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = ow.init_params(seed)
    shapes = ow.param_shapes()
    flat[:int(np.prod(shapes[0][1]))] *= 0.125          # conv0 sees log-mel values of ~-6 +- 3
    for i, (name, sh) in enumerate(shapes):              # nonzero biases exercise their paths
        if ".b" in name:
            o = sum(int(np.prod(s)) for _, s in shapes[:i])
            flat[o:o + int(np.prod(sh))] = 0.1 * rng.standard_normal(int(np.prod(sh)))
    flat = flat.astype(np.float32).astype(np.float64)
    B = sum(counts)
    feats = (-6.0 + 3.0 * rng.standard_normal((B, 256, 32))).astype(np.float32).astype(np.float64)
    types = [t for t, c in zip(HEADS, counts) for _ in range(c)]
    d_out = np.zeros((B, 176))
    for i, t in enumerate(types):
        d_out[i, :ow.HEAD_OUT[t]] = rng.standard_normal(ow.HEAD_OUT[t])
    d_out = d_out.astype(np.float32).astype(np.float64)
    return flat, feats, types, d_out


def _oracle(flat, feats, types, d_out, rnd):
    outs, grad = np.zeros((len(types), 176)), np.zeros_like(flat)
    for i, t in enumerate(types):
        o, cache = ow.forward(flat, feats[i], t, rnd)
        outs[i, :o.shape[0]] = o
        grad += ow.backward(flat, cache, t, d_out[i, :o.shape[0]])
    return outs, grad


def _gpu(gx, torch, flat, feats, counts, d_out):
    B = sum(counts)
    net = gx.WarmStartNet(max_batch=B + 3, max_rows=1, max_len=2048)
    assert net.n_params == flat.shape[0]
    W = torch.tensor(flat, dtype=torch.float32, device="cuda")
    Fd = torch.tensor(feats, dtype=torch.float32, device="cuda")
    out = torch.full((B, 176), float("nan"), device="cuda")
    dW = torch.full_like(W, float("nan"))
    st = gx._stream(torch, W.device)
    net.forward_raw(W, Fd, counts, out, st)
    net.backward_raw(W, Fd, counts, torch.tensor(d_out, dtype=torch.float32, device="cuda"), dW, st)
    net.sync_status(st)
    return out.cpu().numpy().astype(np.float64), dW.cpu().numpy().astype(np.float64)


def _blocks(v):
    o = 0
    for name, sh in ow.param_shapes():
        n = int(np.prod(sh))
        yield name, v[o:o + n]
        o += n


# 133 samples: 34 row tiles (the last one ragged), 67 k-tiles in the weight gradients
# (the last one half past the batch) split over CTAs and summed through the permutation;
# 512: the training step's minibatch (128 row tiles, 256 k-tiles, every head populated)
@pytest.mark.parametrize("counts", [(2, 1, 1, 1, 1, 1), (0, 0, 3, 0, 2, 0), (1, 0, 0, 0, 0, 0),
                                    (40, 20, 30, 20, 13, 10), (100, 90, 110, 105, 60, 47)])
def test_network_matches_bf16_oracle(env, counts):
    gx, torch = env
    flat, feats, types, d_out = _batch(sum(counts) + 17, counts)
    got_o, got_g = _gpu(gx, torch, flat, feats, list(counts), d_out)
    want_o, want_g = _oracle(flat, feats, types, d_out, ow.bf16_round)
    assert np.linalg.norm(got_o - want_o) <= 1e-2 * np.linalg.norm(want_o)
    for i, t in enumerate(types):                      # unused output columns stay zero
        assert not got_o[i, ow.HEAD_OUT[t]:].any()
    for (name, g), (_, w) in zip(_blocks(got_g), _blocks(want_g)):
        nw = np.linalg.norm(w)
        if nw == 0:
            assert not g.any(), name                    # heads without samples: zero gradient
        else:
            assert np.linalg.norm(g - w) <= 1e-2 * nw, (name, np.linalg.norm(g - w) / nw)


def test_network_matches_exact_oracle_within_bf16_error(env):
    gx, torch = env
    counts = (1, 1, 2, 1, 1, 1)
    flat, feats, types, d_out = _batch(5, counts)
    got_o, got_g = _gpu(gx, torch, flat, feats, list(counts), d_out)
    want_o, want_g = _oracle(flat, feats, types, d_out, None)
    assert np.linalg.norm(got_o - want_o) <= 2e-2 * np.linalg.norm(want_o)
    for (name, g), (_, w) in zip(_blocks(got_g), _blocks(want_g)):
        nw = np.linalg.norm(w)
        assert np.linalg.norm(g - w) <= 2e-2 * nw, name
        assert g @ w >= 0.9995 * np.linalg.norm(g) * nw, name


def test_network_rejects_bad_head_counts(env):
    gx, torch = env
    net = gx.WarmStartNet(max_batch=4, max_rows=1, max_len=2048)
    W = torch.zeros(net.n_params, device="cuda")
    Fd = torch.zeros(5, 256, 32, device="cuda")
    out = torch.zeros(5, 176, device="cuda")
    st = gx._stream(torch, W.device)
    with pytest.raises(gx.GrafxError):
        net.forward_raw(W, Fd, [5, 0, 0, 0, 0, 0], out, st)      # above max_batch
    with pytest.raises(gx.GrafxError):
        net.forward_raw(W, Fd, [-1, 2, 0, 0, 0, 0], out, st)


def test_masked_mse_matches_oracle(env):
    gx, torch = env
    rng = np.random.Generator(np.random.PCG64(12))
    B = 37
    out = rng.standard_normal((B, 176)).astype(np.float32)
    tgt = rng.standard_normal((B, 176)).astype(np.float32)
    n_out = rng.choice([2, 1, 8, 4, 176, 50], B).astype(np.int32)
    o, t = torch.tensor(out, device="cuda"), torch.tensor(tgt, device="cuda")
    loss = torch.zeros(1, device="cuda")
    d = torch.full_like(o, float("nan"))
    gx.WarmStartNet.mse_raw(o, t, torch.tensor(n_out, device="cuda"), loss, d, gx._stream(torch, o.device))
    torch.cuda.synchronize()
    wl, wd = ow.masked_mse(out, tgt, n_out)
    assert abs(loss.item() - wl) <= 1e-5 * wl
    np.testing.assert_allclose(d.cpu().numpy(), wd, rtol=1e-5, atol=1e-9)


def test_node_inputs_match_oracle_render(env):
    gx, torch = env
    from gpu_common import DeviceRun, assert_out_close, flat_sources, union_params
    from oracle import render as orr
    g = synth.console_cfg1()
    L = 5003
    src_flat, per = flat_sources([g], [L], [71])
    P = union_params([g], 72)
    run = DeviceRun([g], [L], P, src_flat, eq_taps=255)
    out = run.render()
    ids = [v for v, t in enumerate(g.types) if t != synth.I]
    pitch = (L + 3) // 4 * 4 + 8
    dst = torch.full((len(ids), 2, pitch), float("nan"), device="cuda")
    run.plan.node_inputs_raw(run.src, out, ids, dst, pitch, gx._stream(torch, dst.device))
    torch.cuda.synchronize()
    got = dst.cpu().numpy()
    Y = orr.render_one_by_one(g.types, g.edges, per[0][:, :, :L], P, {"eq_taps": 255})
    for i, v in enumerate(ids):
        u = sum(Y[s] for s, d in g.edges if d == v)
        assert_out_close(got[i, :, :L], u)
        assert not got[i, :, L:].any()
    with pytest.raises(gx.GrafxError):                   # input nodes have no node input
        run.plan.node_inputs_raw(run.src, out, [0], dst, pitch, gx._stream(torch, dst.device))


def test_standardise_round_trip(env):
    """grafx_ws_standardise: per-row head statistics, masked columns, both directions."""
    gx, torch = env
    rng = np.random.Generator(np.random.PCG64(12))
    B, cols, heads = 37, 176, 6
    x = rng.standard_normal((B, cols)).astype(np.float32)
    head = rng.integers(0, heads, B).astype(np.int32)
    n_out = np.array([ow.HEAD_OUT[ow.HEAD_TYPES[h]] for h in head], np.int32)
    mu = rng.standard_normal((heads, cols)).astype(np.float32)
    sd = rng.uniform(0.2, 3.0, (heads, cols)).astype(np.float32)
    d = lambda a: torch.tensor(a, device="cuda")
    xd, hd, nd, mud, sdd = d(x), d(head), d(n_out), d(mu), d(sd)
    y, z = torch.empty_like(xd), torch.empty_like(xd)
    lib, st = gx.lib(), gx._stream(torch, xd.device)
    p = gx._ptr
    assert lib.grafx_ws_standardise(p(xd), p(hd), p(nd), p(mud), p(sdd), B, cols, 0, p(y), st) == 0
    assert lib.grafx_ws_standardise(p(y), p(hd), p(nd), p(mud), p(sdd), B, cols, 1, p(z), st) == 0
    torch.cuda.synchronize()
    mask = np.arange(cols)[None, :] < n_out[:, None]
    want = np.where(mask, (x - mu[head]) / sd[head], 0.0)
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(z.cpu().numpy(), np.where(mask, x, 0.0), rtol=1e-5, atol=1e-6)
