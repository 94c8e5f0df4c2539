"""Parameter fitting by gradient descent: Adam on unconstrained parameters (FP64 oracle;
test infrastructure only, see ``oracle/__init__``).

The paper fits every processor's parameters of a large graph by gradient descent to
match a target mix (Abstract; Sec. 4 "Example usage") without naming the optimiser or
how constrained parameters are handled.  Reading used here: Adam (Kingma & Ba, the
published algorithm with bias correction) on unconstrained theta; the processors take
physical parameters p = map(theta), element-wise:

  IDENT     p = theta                              (gains, bands, thresholds, ...)
  ALPHA     p = 0.9 + 0.0999 * sigmoid(theta)      (compressor coefficient in (0.9, 0.9999))
  SOFTPLUS  p = softplus(theta)                    (knee half-width W > 0)
  RATIO     p = 1 + softplus(theta)                (ratio R > 1)
  NEGSP     p = -softplus(theta)                   (per-frame decay, < 0)
  ATTACK    p = 0.5 + 0.4999 * sigmoid(theta)      (attack coefficient in (0.5, 0.9999))
  ZRE, ZIM  p = theta                              (a delay tap's Re z and Im z, a pair)

dLoss/dtheta = dLoss/dp * dp/dtheta.

Multitap delay (Sec. 3, the sentences after Eq. 15): the paper normalises the
surrogate's z-gradients and pulls z towards the unit circle, without constants.
Reading (``delay_z_grad``): per (channel, tap) the 2-vector (dL/dRe z, dL/dIm z) is
scaled to unit L2 norm (a zero vector stays zero), then the gradient of the penalty
LAMBDA_Z (|z| - 1)^2, LAMBDA_Z = 1e-2, is added; Adam takes that as the pair's
gradient.  The penalty enters the update only, not the reported loss.
"""
import numpy as np

IDENT, ALPHA, SOFTPLUS, RATIO, NEGSP, ATTACK, ZRE, ZIM = range(8)
LAMBDA_Z = 1e-2


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def to_param(theta, code):
    theta = np.asarray(theta, dtype=np.float64)
    code = np.broadcast_to(code, theta.shape)
    out = theta.copy()
    out = np.where(code == ALPHA, 0.9 + 0.0999 * sigmoid(theta), out)
    out = np.where(code == SOFTPLUS, softplus(theta), out)
    out = np.where(code == RATIO, 1.0 + softplus(theta), out)
    out = np.where(code == NEGSP, -softplus(theta), out)
    out = np.where(code == ATTACK, 0.5 + 0.4999 * sigmoid(theta), out)
    return out


def dparam_dtheta(theta, code):
    theta = np.asarray(theta, dtype=np.float64)
    code = np.broadcast_to(code, theta.shape)
    s = sigmoid(theta)
    d = np.ones_like(theta)
    d = np.where(code == ALPHA, 0.0999 * s * (1.0 - s), d)
    d = np.where((code == SOFTPLUS) | (code == RATIO), s, d)   # softplus' = sigmoid
    d = np.where(code == NEGSP, -s, d)
    d = np.where(code == ATTACK, 0.4999 * s * (1.0 - s), d)
    return d


def to_theta(param, code):
    """Inverse of ``to_param`` (for starting a fit from physical parameters)."""
    p = np.asarray(param, dtype=np.float64)
    code = np.broadcast_to(code, p.shape)
    out = p.copy()
    with np.errstate(divide="ignore", invalid="ignore"):
        a = (p - 0.9) / 0.0999
        out = np.where(code == ALPHA, np.log(a) - np.log1p(-a), out)
        out = np.where(code == SOFTPLUS, p + np.log(-np.expm1(-p)), out)
        out = np.where(code == RATIO, (p - 1) + np.log(-np.expm1(-(p - 1))), out)
        out = np.where(code == NEGSP, -p + np.log(-np.expm1(p)), out)
        b = (p - 0.5) / 0.4999
        out = np.where(code == ATTACK, np.log(b) - np.log1p(-b), out)
    return out


def z_penalty(zr, zi, lam=LAMBDA_Z):
    """The unit-circle regulariser lam (|z| - 1)^2 of a delay tap."""
    return lam * (np.hypot(zr, zi) - 1.0) ** 2


def delay_z_grad(theta, grad_theta, code, lam=LAMBDA_Z):
    """The delay taps' update direction: every (ZRE, ZIM) column pair of grad_theta
    scaled to unit length, plus the gradient of z_penalty at theta's (Re z, Im z); other
    columns unchanged.  Rows are the last axis's column layout ``code``."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.array(grad_theta, dtype=np.float64, copy=True)
    code = np.asarray(code)
    for j in np.flatnonzero(code == ZRE):
        assert code[j + 1] == ZIM
        gr, gi = g[..., j], g[..., j + 1]
        n = np.hypot(gr, gi)
        safe = np.where(n > 0, n, 1.0)
        gr, gi = np.where(n > 0, gr / safe, 0.0), np.where(n > 0, gi / safe, 0.0)
        zr, zi = theta[..., j], theta[..., j + 1]
        r = np.hypot(zr, zi)
        k = np.where(r > 0, 2.0 * lam * (r - 1.0) / np.where(r > 0, r, 1.0), 0.0)
        g[..., j], g[..., j + 1] = gr + k * zr, gi + k * zi
    return g


def adam_step(theta, m, v, grad_theta, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (theta, m, v)."""
    g = np.asarray(grad_theta, dtype=np.float64)
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def param_codes(t, cols):
    """Map code of every column of P[t] (type ids as in synth.types)."""
    codes = np.full(cols, IDENT, dtype=np.int8)
    if t in (6, 9, 12):              # compressor / noisegate / sidechain [alpha, T, W, R]
        codes[:] = [ALPHA, IDENT, SOFTPLUS, RATIO]
    if t == 13:                      # attack/release compressor [alpha_a, alpha_r, T, W, R]
        codes[:] = [ATTACK, ALPHA, IDENT, SOFTPLUS, RATIO]
    if t == 8 and cols == 50:        # reverb (12 bands): H_delta columns are decays
        c = np.full(50, IDENT, dtype=np.int8)
        c[:48] = np.tile(np.repeat([IDENT, NEGSP], 12), 2)
        codes = c
    elif t == 8:                     # reverb, per-bin layout [mid, side] x [H0 (K), H_delta (K)]
        K = cols // 4
        codes = np.tile(np.repeat(np.array([IDENT, NEGSP], dtype=np.int8), K), 2)
    if t == 7:                       # delay: per (channel, tap) [Re z, Im z, 20 log-magnitudes]
        codes = np.tile(np.array([ZRE, ZIM] + [IDENT] * 20, dtype=np.int8), cols // 22)
    return codes
