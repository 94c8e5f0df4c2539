"""Learned warm-start network in float64 (oracle; test infrastructure only, see
``oracle/__init__``).

The paper motivates parameter estimation by a trained network (Sec. 1) and GNN use
of its graphs, without fixing an architecture.  Reading used here (about 1.2 M
parameters):
  features  log-mel of a mono signal (l + r)/2: frames of 2048 with hop 512 (no
            padding), periodic Hann, power spectrum, 128 triangular mel filters on
            the HTK mel scale 2595 log10(1 + f/700) between 0 Hz and fs/2, ln(mel +
            1e-5); frames average-pooled to T = 32 (frame i of the pool averages
            frames [floor(i F/T), floor((i+1) F/T)) of F).  A node's input is the
            concatenation of the log-mel of its input signal (rendered with neutral
            parameters) and of the cross-spectral band gain ``xgain`` of that input
            against the target mix: 256 x T.
  encoder   4 conv1d layers, kernel 5, zero padding 2 ('same'), 256->128->128->128->128,
            bias, exact GELU 0.5 x (1 + erf(x / sqrt 2)); mean over time -> e in R^128.
  heads     one MLP per parameterised type: 128 -> 288 -> 288 -> N_t (GELU, GELU,
            linear); output = the unconstrained parameters theta of the fit.
  loss      squared error averaged over the N_t outputs of each sample, then over the
            samples.

``forward``/``backward`` take an optional operand rounding ``rnd`` applied to both
operands of every matrix product (``bf16_round`` reproduces the operand precision of a
BF16 tensor-core product; with ``rnd=None`` everything is float64).
"""
import numpy as np
from scipy.special import erf

N_MEL = 128
MEL_NFFT = 2048
MEL_HOP = 512
MEL_EPS = 1e-5
T_POOL = 32
CONV_CH = (256, 128, 128, 128, 128)
KW = 5
HID = 288
HEAD_TYPES = (3, 4, 5, 6, 7, 8)               # g, s, e, c, d, r
HEAD_OUT = {3: 2, 4: 1, 5: 8, 6: 4, 7: 176, 8: 50}


def hz_to_mel(f):
    return 2595.0 * np.log10(1.0 + np.asarray(f, dtype=np.float64) / 700.0)


def mel_to_hz(m):
    return 700.0 * (10.0 ** (np.asarray(m, dtype=np.float64) / 2595.0) - 1.0)


def mel_filterbank(fs=44100, nfft=MEL_NFFT, n_mel=N_MEL):
    """[n_mel, nfft/2+1] triangles with peaks 1 at mel-spaced centres."""
    edges = mel_to_hz(np.linspace(0.0, hz_to_mel(fs / 2.0), n_mel + 2))
    f = np.arange(nfft // 2 + 1) * fs / nfft
    W = np.zeros((n_mel, f.shape[0]))
    for b in range(n_mel):
        lo, c, hi = edges[b], edges[b + 1], edges[b + 2]
        up = (f - lo) / (c - lo)
        dn = (hi - f) / (hi - c)
        W[b] = np.maximum(0.0, np.minimum(up, dn))
    return W


def logmel(x, fs=44100, T=T_POOL):
    """x: [2, L] stereo -> [128, T] pooled log-mel of the mono mix."""
    m = 0.5 * (np.asarray(x[0], np.float64) + np.asarray(x[1], np.float64))
    F = 1 + (m.shape[0] - MEL_NFFT) // MEL_HOP
    idx = np.arange(F)[:, None] * MEL_HOP + np.arange(MEL_NFFT)[None, :]
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(MEL_NFFT) / MEL_NFFT)
    P = np.abs(np.fft.rfft(m[idx] * w[None, :], axis=-1)) ** 2
    mel = np.log(P @ mel_filterbank(fs).T + MEL_EPS)          # [F, 128]
    out = np.zeros((N_MEL, T))
    for i in range(T):
        a, b = (i * F) // T, ((i + 1) * F) // T
        out[:, i] = mel[a:max(b, a + 1)].mean(axis=0)
    return out


XG_BANDS = 64          # band pairs of the 128 mel triangles
XG_FLOOR = 1e-2


def _frames(m):
    F = 1 + (m.shape[0] - MEL_NFFT) // MEL_HOP
    idx = np.arange(F)[:, None] * MEL_HOP + np.arange(MEL_NFFT)[None, :]
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(MEL_NFFT) / MEL_NFFT)
    return np.fft.rfft(m[idx] * w[None, :], axis=-1), F


def xgain(u, T, fs=44100, T_slots=T_POOL):
    """Cross-spectral band gain of a node's path to the output (a reading: the network's
    second input block, in place of the target mix's log-mel).  u: the node's input
    [2, L], T: the target mix [2, L].  For the mid (l + r)/2 and the side (l - r)/2 of
    both, per frame (the log-mel framing) and mel triangle: C = sum_k w Re(T_k conj(U_k))
    and P = sum_k w |U_k|^2; adjacent triangles summed in pairs (64 bands); per pooling
    slot (the log-mel's frame ranges) the sums over its frames give the gain C / P, and
    the feature is ln(max(C / P, 0) + 1e-2).  Because the sources of a mix are independent,
    the part of the target correlated with the node's input is the node's own path
    (its processor and everything downstream) applied to it: C / P estimates that path's
    gain in the band.  Returns [128, T]: 64 mid bands, then 64 side bands."""
    u = np.asarray(u, np.float64)
    T = np.asarray(T, np.float64)
    W = mel_filterbank(fs)
    out = np.zeros((2 * XG_BANDS, T_slots))
    for half, sgn in ((0, 1.0), (1, -1.0)):
        U, F = _frames(0.5 * (u[0] + sgn * u[1]))
        Y, _ = _frames(0.5 * (T[0] + sgn * T[1]))
        C = (np.real(Y * np.conj(U)) @ W.T)                       # [F, 128]
        P = ((np.abs(U) ** 2) @ W.T)
        C = C[:, 0::2] + C[:, 1::2]                               # [F, 64]
        P = P[:, 0::2] + P[:, 1::2]
        for i in range(T_slots):
            a, b = (i * F) // T_slots, ((i + 1) * F) // T_slots
            b = max(b, a + 1)
            g = C[a:b].sum(axis=0) / np.maximum(P[a:b].sum(axis=0), 1e-20)
            out[half * XG_BANDS:(half + 1) * XG_BANDS, i] = np.log(np.maximum(g, 0.0) + XG_FLOOR)
    return out


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64.  bfloat16 is the
    upper half of the float32 bit pattern: 8 exponent bits, 7 fraction bits."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _id(x):
    return x


def masked_mse(out, target, n_out):
    """Mean over rows of the mean squared error over each row's first n_out[i] entries
    (every sample weighs the same whatever its head's width), and its gradient with
    respect to out."""
    out = np.asarray(out, np.float64)
    target = np.asarray(target, np.float64)
    n_out = np.asarray(n_out)
    mask = np.arange(out.shape[1])[None, :] < n_out[:, None]
    r = np.where(mask, out - target, 0.0)
    B = out.shape[0]
    loss = float(((r * r).sum(axis=1) / n_out).sum() / B)
    return loss, 2.0 * r / (B * n_out[:, None])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi)


def param_shapes():
    """(name, shape) of every tensor, in the flat order used by the GPU buffers."""
    s = []
    for l in range(4):
        s.append((f"conv{l}.w", (CONV_CH[l + 1], CONV_CH[l], KW)))
        s.append((f"conv{l}.b", (CONV_CH[l + 1],)))
    for t in HEAD_TYPES:
        s += [(f"h{t}.w1", (HID, CONV_CH[-1])), (f"h{t}.b1", (HID,)), (f"h{t}.w2", (HID, HID)),
              (f"h{t}.b2", (HID,)), (f"h{t}.w3", (HEAD_OUT[t], HID)), (f"h{t}.b3", (HEAD_OUT[t],))]
    return s


def n_params():
    return sum(int(np.prod(sh)) for _, sh in param_shapes())


def unflatten(flat):
    out, o = {}, 0
    for name, sh in param_shapes():
        n = int(np.prod(sh))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(sh)
        o += n
    return out


def init_params(seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = []
    for name, sh in param_shapes():
        if name.endswith(".w") or ".w" in name:
            fan_in = int(np.prod(sh[1:]))
            flat.append(rng.standard_normal(sh).ravel() * np.sqrt(2.0 / fan_in))
        else:
            flat.append(np.zeros(int(np.prod(sh))))
    return np.concatenate(flat)


def conv1d(x, w, b, rnd=_id):
    """x [Cin, T], w [Cout, Cin, 5], zero padding 2 -> [Cout, T]."""
    T = x.shape[1]
    xp = rnd(np.pad(x, ((0, 0), (2, 2))))
    w = rnd(w)
    y = np.zeros((w.shape[0], T))
    for k in range(KW):
        y += w[:, :, k] @ xp[:, k:k + T]
    return y + b[:, None]


def forward(flat, feats, head_type, rnd=None):
    """feats [256, T] -> (output [N_t], cache)."""
    rnd = rnd or _id
    p = unflatten(flat)
    cache = {"x0": np.asarray(feats, np.float64), "rnd": rnd}
    h = cache["x0"]
    for l in range(4):
        z = conv1d(h, p[f"conv{l}.w"], p[f"conv{l}.b"], rnd)
        cache[f"z{l}"] = z
        h = gelu(z)
        cache[f"h{l}"] = h
    e = h.mean(axis=1)
    cache["e"] = e
    t = head_type
    a1 = rnd(p[f"h{t}.w1"]) @ rnd(e) + p[f"h{t}.b1"]
    g1 = gelu(a1)
    a2 = rnd(p[f"h{t}.w2"]) @ rnd(g1) + p[f"h{t}.b2"]
    g2 = gelu(a2)
    out = rnd(p[f"h{t}.w3"]) @ rnd(g2) + p[f"h{t}.b3"]
    cache.update(a1=a1, g1=g1, a2=a2, g2=g2)
    return out, cache


def backward(flat, cache, head_type, d_out):
    """Gradient of <d_out, output> with respect to the flat parameters (the operand
    rounding of the forward applies to every product here too)."""
    r = cache["rnd"]
    p = unflatten(flat)
    g = {name: np.zeros(sh) for name, sh in param_shapes()}
    t = head_type
    d_out = np.asarray(d_out, np.float64)
    g[f"h{t}.w3"] = np.outer(r(d_out), r(cache["g2"]))
    g[f"h{t}.b3"] = d_out.copy()
    da2 = (r(p[f"h{t}.w3"]).T @ r(d_out)) * gelu_grad(cache["a2"])
    g[f"h{t}.w2"] = np.outer(r(da2), r(cache["g1"]))
    g[f"h{t}.b2"] = da2
    da1 = (r(p[f"h{t}.w2"]).T @ r(da2)) * gelu_grad(cache["a1"])
    g[f"h{t}.w1"] = np.outer(r(da1), r(cache["e"]))
    g[f"h{t}.b1"] = da1
    de = r(p[f"h{t}.w1"]).T @ r(da1)
    T = cache["x0"].shape[1]
    dh = np.repeat(de[:, None] / T, T, axis=1)
    for l in range(3, -1, -1):
        dz = dh * gelu_grad(cache[f"z{l}"])
        x = cache["x0"] if l == 0 else cache[f"h{l - 1}"]
        xp = r(np.pad(x, ((0, 0), (2, 2))))
        w = r(p[f"conv{l}.w"])
        g[f"conv{l}.b"] = dz.sum(axis=1)
        dzr = r(dz)
        for k in range(KW):
            g[f"conv{l}.w"][:, :, k] = dzr @ xp[:, k:k + T].T
        dxp = np.zeros_like(xp)
        for k in range(KW):
            dxp[:, k:k + T] += w[:, :, k].T @ dzr
        dh = dxp[:, 2:2 + T]
    return np.concatenate([g[name].ravel() for name, _ in param_shapes()])
