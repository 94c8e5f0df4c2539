"""Multi-resolution STFT magnitude loss and its gradient in float64 (oracle; test
infrastructure only, see ``oracle/__init__``).

The paper only says that the rendered output is used "to calculate a loss and
perform the gradient descent to match the target mix" (Sec. 4, Example usage).
Reading used here, per output row and per resolution M in {512, 1024, 2048} with
hop M/4, periodic Hann window w[n] = 0.5 - 0.5 cos(2 pi n / M), frames at
f*hop for f = 0..F-1, F = 1 + (L - M) // hop (no centre padding), and per channel:
  L_sc  = || |Y| - |T| ||_F / || |T| ||_F
  L_mag = mean | ln(|Y| + 1e-7) - ln(|T| + 1e-7) |
over the one-sided bins k = 0..M/2.  The row loss is the mean of (L_sc + L_mag)
over the 3 resolutions and 2 channels; the total is the sum over output rows.
"""
import numpy as np

RESOLUTIONS = (512, 1024, 2048)
MAG_EPS = 1e-7


def hann_periodic(M):
    return 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(M) / M)


def frames(x, M):
    hop = M // 4
    L = x.shape[-1]
    F = 1 + (L - M) // hop
    idx = np.arange(F)[:, None] * hop + np.arange(M)[None, :]
    return x[idx], F


def spec(x, M):
    """One-sided DFT of windowed frames: [F, M/2+1] complex."""
    fr, _ = frames(np.asarray(x, dtype=np.float64), M)
    return np.fft.rfft(fr * hann_periodic(M)[None, :], axis=-1)


def row_loss(y, t, resolutions=RESOLUTIONS):
    total = 0.0
    for M in resolutions:
        for c in range(2):
            Y, T = np.abs(spec(y[c], M)), np.abs(spec(t[c], M))
            sc = np.linalg.norm(Y - T) / np.linalg.norm(T)
            mag = np.mean(np.abs(np.log(Y + MAG_EPS) - np.log(T + MAG_EPS)))
            total += sc + mag
    return total / (2 * len(resolutions))


def mrstft(Y, T, resolutions=RESOLUTIONS):
    """Sum over output rows of ``row_loss``; Y, T: [rows, 2, L]."""
    return sum(row_loss(Y[j], T[j], resolutions) for j in range(Y.shape[0]))


def row_grad(y, t, resolutions=RESOLUTIONS):
    """dLoss/dy for one row: chain through |Y|, the one-sided DFT, the window and
    the overlap-add of the frames."""
    y = np.asarray(y, dtype=np.float64)
    L = y.shape[-1]
    g = np.zeros((2, L))
    w_res = 1.0 / (2 * len(resolutions))
    for M in resolutions:
        hop = M // 4
        win = hann_periodic(M)
        for c in range(2):
            Yc = spec(y[c], M)
            A, B = np.abs(Yc), np.abs(spec(t[c], M))
            F = A.shape[0]
            nd, nt = np.linalg.norm(A - B), np.linalg.norm(B)
            dA = np.zeros_like(A)
            if nd > 0:
                dA += (A - B) / (nd * nt)
            dA += np.sign(np.log(A + MAG_EPS) - np.log(B + MAG_EPS)) / ((A + MAG_EPS) * A.size)
            dA *= w_res
            with np.errstate(invalid="ignore", divide="ignore"):
                G = np.where(A > 0, dA * Yc / np.where(A > 0, A, 1.0), 0.0)
            # x_bar[n] = Re sum_{k=0}^{M/2} G_k exp(+2 pi j k n / M)
            full = np.zeros((F, M), dtype=np.complex128)
            full[:, :M // 2 + 1] = G
            xbar = np.real(np.fft.ifft(full, axis=-1)) * M
            xbar *= win[None, :]
            for f in range(F):
                g[c, f * hop:f * hop + M] += xbar[f]
    return g


def mrstft_grad(Y, T, resolutions=RESOLUTIONS):
    return np.stack([row_grad(Y[j], T[j], resolutions) for j in range(Y.shape[0])])
