"""Differentiable processors and their analytic adjoints in float64 (oracle; test
infrastructure only, see ``oracle/__init__``).

Every processor maps a stereo input u[2, L] and one parameter row p to y[2, L]
(Sec. 3: processors take and produce stereo signals, C = 2).  Signals are zero
outside [0, L) and outputs are truncated to L.  Every ``*_bwd`` takes the output
adjoint ybar = dLoss/dy and returns (ubar, pbar) = (dLoss/du, dLoss/dp).

Readings of points the paper leaves open (each is stated where used):
  * EQ (Eq. 4): the index range printed for n has N+2 points; this oracle uses an odd
    N and n in [-H, H], H = (N-1)/2, with K = (N+1)/2 log-magnitudes mirrored so the
    filter is real and even; the Hann window is 0.5(1 + cos(2 pi n/(N+1))), which is
    zero at n = +-(N+1)/2, the printed bounds.  The convolution of Eq. 5 is centred
    (zero phase).  The 8 band gains in dB map to the K log-magnitudes by linear
    interpolation in log2 frequency between log-spaced band centres
    f_b = 20 * 1000^((b+0.5)/8) Hz, constant beyond the end centres.
  * Compressor (Eq. 8-12): the mid signal is u_l + u_r (a sum, as in the text); the
    one-pole recursion of Eq. 8 runs exactly with g[-1] = 0 (Eq. 9 with an FIR as
    long as the signal); G_u = ln(g + eps) with eps = 1e-7; T and W are in natural-log
    energy units.
"""
import numpy as np
import scipy.signal

LN10 = np.log(10.0)
COMP_EPS = 1e-7
EQ_BANDS = 8


def _f64(x):
    return np.asarray(x, dtype=np.float64)


# ---------------------------------------------------------------- gain / panning (Eq. 2)
def gain_fwd(u, p):
    """y_c = exp(p_c) u_c, p in R^2 (log scale, one per channel)."""
    u, p = _f64(u), _f64(p)
    return np.exp(p)[:, None] * u


def gain_bwd(u, p, ybar):
    u, p, ybar = _f64(u), _f64(p), _f64(ybar)
    a = np.exp(p)
    ubar = a[:, None] * ybar
    pbar = a * np.sum(ybar * u, axis=1)
    return ubar, pbar


# ---------------------------------------------------------------- stereo imager (Eq. 3a/3b)
def imager_fwd(u, p):
    """mid = l + r, side = exp(p_s)(l - r), then l = (mid+side)/2, r = (mid-side)/2."""
    u, p = _f64(u), _f64(p)
    mid = u[0] + u[1]
    side = np.exp(p[0]) * (u[0] - u[1])
    return np.stack([(mid + side) / 2, (mid - side) / 2])


def gain_bwd_abs(u, p, ybar):
    """Sum of the magnitudes of the terms of ``gain_bwd``'s parameter gradient (how far
    a finite-precision evaluation of that sum can be trusted)."""
    u, p, ybar = _f64(u), _f64(p), _f64(ybar)
    return np.exp(p) * np.sum(np.abs(ybar * u), axis=1)


def imager_bwd_abs(u, p, ybar):
    """Sum of the magnitudes of the terms of ``imager_bwd``'s parameter gradient."""
    u, p, ybar = _f64(u), _f64(p), _f64(ybar)
    sidebar = (ybar[0] - ybar[1]) / 2
    return np.array([np.exp(p[0]) * np.sum(np.abs(sidebar * (u[0] - u[1])))])


def imager_bwd(u, p, ybar):
    u, p, ybar = _f64(u), _f64(p), _f64(ybar)
    a = np.exp(p[0])
    midbar = (ybar[0] + ybar[1]) / 2
    sidebar = (ybar[0] - ybar[1]) / 2
    ubar = np.stack([midbar + a * sidebar, midbar - a * sidebar])
    pbar = np.array([a * np.sum(sidebar * (u[0] - u[1]))])
    return ubar, pbar


# ---------------------------------------------------------------- zero-phase FIR EQ (Eq. 4-5)
def eq_band_centres(n_bands=EQ_BANDS):
    return 20.0 * 1000.0 ** ((np.arange(n_bands) + 0.5) / n_bands)


def eq_band_matrix(N, fs=44100, n_bands=EQ_BANDS):
    """B (K x n_bands): dB of bin k = sum_b B[k, b] band_dB[b]; bin k sits at k fs / N."""
    K = (N + 1) // 2
    c = eq_band_centres(n_bands)
    lc = np.log2(c)
    B = np.zeros((K, n_bands))
    for k in range(K):
        f = k * fs / N
        if f <= c[0]:
            B[k, 0] = 1.0
        elif f >= c[-1]:
            B[k, -1] = 1.0
        else:
            b = int(np.searchsorted(c, f, side="right")) - 1
            w = (np.log2(f) - lc[b]) / (lc[b + 1] - lc[b])
            B[k, b] = 1.0 - w
            B[k, b + 1] = w
    return B


def eq_logmag(bands_db, N, fs=44100):
    """p_e[k] (natural-log magnitude) from band gains in dB."""
    return eq_band_matrix(N, fs, len(bands_db)) @ _f64(bands_db) * LN10 / 20.0


def hann_sym(N):
    """v[n] = 0.5 (1 + cos(2 pi n / (N+1))), n in [-H, H]."""
    H = (N - 1) // 2
    n = np.arange(-H, H + 1)
    return 0.5 * (1.0 + np.cos(2 * np.pi * n / (N + 1)))


def zerophase_taps(logmag, N):
    """Eq. 4: h[n] = v[n] (1/N) sum_k exp(p[k]) w_N^{kn}, magnitudes mirrored
    (A_{N-k} = A_k) so that h is real and even.  Returns h[-H..H] as length N."""
    H = (N - 1) // 2
    K = (N + 1) // 2
    A = np.exp(_f64(logmag))
    assert A.shape[0] == K
    n = np.arange(-H, H + 1)
    k = np.arange(1, K)
    h0 = (A[0] + 2.0 * np.cos(2 * np.pi * np.outer(n, k) / N) @ A[1:]) / N
    return hann_sym(N) * h0


def zerophase_taps_bwd(logmag, N, hbar):
    """Adjoint of ``zerophase_taps``: dLoss/dp[k] from dLoss/dh[n]."""
    H = (N - 1) // 2
    K = (N + 1) // 2
    A = np.exp(_f64(logmag))
    n = np.arange(-H, H + 1)
    h0bar = hann_sym(N) * _f64(hbar)
    coef = np.full(K, 2.0 / N)
    coef[0] = 1.0 / N
    Abar = coef * (np.cos(2 * np.pi * np.outer(np.arange(K), n) / N) @ h0bar)
    return A * Abar


def eq_taps_from_bands(bands_db, N, fs=44100):
    return zerophase_taps(eq_logmag(bands_db, N, fs), N)


def fir_centred(u, h):
    """Eq. 5, centred: y[t] = sum_{m=-H}^{H} h[m] u[t-m], u = 0 outside [0, L)."""
    H = (len(h) - 1) // 2
    L = u.shape[-1]
    return scipy.signal.fftconvolve(u, h[None, :], axes=-1)[..., H:H + L]


def fir_centred_adjoint(ybar, h):
    """ubar[t] = sum_m h[m] ybar[t+m] (transpose of ``fir_centred``)."""
    return fir_centred(ybar, h[::-1])


def fir_centred_taps_grad(u, ybar, H):
    """dLoss/dh[m] = sum_x sum_t ybar_x[t] u_x[t-m], m in [-H, H] (zero for |m| >= L:
    no sample pair is that far apart)."""
    L = u.shape[-1]
    # correlation via a library FFT convolution: c[j] = sum_t ybar[t] u[t - (j - L + 1)]
    c = scipy.signal.fftconvolve(ybar, u[:, ::-1], axes=-1).sum(axis=0)
    lag = np.arange(-H, H + 1)
    out = np.zeros(2 * H + 1)
    ok = np.abs(lag) <= L - 1
    out[ok] = c[lag[ok] + L - 1]
    return out


def eq_fwd(u, p, N, fs=44100):
    h = eq_taps_from_bands(p, N, fs)
    return fir_centred(_f64(u), h)


def eq_bwd(u, p, ybar, N, fs=44100):
    u, ybar = _f64(u), _f64(ybar)
    logmag = eq_logmag(p, N, fs)
    h = zerophase_taps(logmag, N)
    ubar = fir_centred_adjoint(ybar, h)
    hbar = fir_centred_taps_grad(u, ybar, (N - 1) // 2)
    lbar = zerophase_taps_bwd(logmag, N, hbar)
    pbar = eq_band_matrix(N, fs, len(p)).T @ lbar * LN10 / 20.0
    return ubar, pbar


# The paper's own EQ parameter (Sec. 3 "Equalizer"): p_e holds the K = (N+1)/2
# log-magnitudes themselves (N = 2047 -> 1024 values), no band interpolation.
def eq_fwd_logmag(u, p, N):
    return fir_centred(_f64(u), zerophase_taps(p, N))


def eq_bwd_logmag(u, p, ybar, N):
    u, ybar = _f64(u), _f64(ybar)
    h = zerophase_taps(p, N)
    ubar = fir_centred_adjoint(ybar, h)
    hbar = fir_centred_taps_grad(u, ybar, (N - 1) // 2)
    return ubar, zerophase_taps_bwd(p, N, hbar)


# ---------------------------------------------------------------- compressor (Eq. 8-12)
def envelope(x, alpha):
    """Eq. 8 with one coefficient: g[n] = alpha g[n-1] + (1-alpha) x[n], g[-1] = 0.
    Run as the exact one-pole IIR (a library linear filter)."""
    return scipy.signal.lfilter([1.0 - alpha], [1.0, -alpha], x)


def envelope_reverse(a, alpha):
    """lambda[n] = a[n] + alpha lambda[n+1], lambda[L] = 0 (adjoint recursion)."""
    return scipy.signal.lfilter([1.0], [1.0, -alpha], a[::-1])[::-1]


def knee(Gu, T, W, R):
    """Eq. 10-11: quadratic-knee static curve and its partials
    (dGy/dGu, dGy/dT, dGy/dW, dGy/dR)."""
    above = Gu >= T + W
    mid = (Gu >= T - W) & ~above
    Gy = Gu.copy()
    dGu = np.ones_like(Gu)
    dT = np.zeros_like(Gu)
    dW = np.zeros_like(Gu)
    dR = np.zeros_like(Gu)
    # above: T + (Gu - T)/R
    Gy[above] = T + (Gu[above] - T) / R
    dGu[above] = 1.0 / R
    dT[above] = 1.0 - 1.0 / R
    dR[above] = -(Gu[above] - T) / R ** 2
    # mid: Gu + (1/R - 1) (Gu - T + W)^2 / (4W)
    d = Gu[mid] - T + W
    c = 1.0 / R - 1.0
    Gy[mid] = Gu[mid] + c * d * d / (4 * W)
    dGu[mid] = 1.0 + c * d / (2 * W)
    dT[mid] = -c * d / (2 * W)
    dW[mid] = c * (d / (2 * W) - d * d / (4 * W * W))
    dR[mid] = -d * d / (4 * W * R ** 2)
    return Gy, dGu, dT, dW, dR


def gate_curve(Gu, T, W, R):
    """Eq. 13 (noisegate): G_y = G_u above T + W; G_u + (1 - R)(G_u - T - W)^2 / (4W)
    inside the knee; T + R (G_u - T) below T - W; with the partials
    (dGy/dGu, dGy/dT, dGy/dW, dGy/dR)."""
    above = Gu >= T + W
    mid = (Gu >= T - W) & ~above
    below = ~(above | mid)
    Gy = Gu.copy()
    dGu = np.ones_like(Gu)
    dT = np.zeros_like(Gu)
    dW = np.zeros_like(Gu)
    dR = np.zeros_like(Gu)
    d = Gu[mid] - T - W
    c = 1.0 - R
    Gy[mid] = Gu[mid] + c * d * d / (4 * W)
    dGu[mid] = 1.0 + c * d / (2 * W)
    dT[mid] = -c * d / (2 * W)
    dW[mid] = c * (-d / (2 * W) - d * d / (4 * W * W))
    dR[mid] = -d * d / (4 * W)
    Gy[below] = T + R * (Gu[below] - T)
    dGu[below] = R
    dT[below] = 1.0 - R
    dR[below] = Gu[below] - T
    return Gy, dGu, dT, dW, dR


def compressor_fwd(u, p, eps=COMP_EPS, return_env=False, curve=knee, key=None):
    """Eq. 8-12 (curve = knee); the noisegate is the same with curve = gate_curve.  With
    ``key`` (a sidechain input) the envelope of Eq. 8 follows the key's mid signal and
    the gain of Eq. 12 applies to u."""
    u = _f64(u)
    alpha, T, W, R = (float(v) for v in _f64(p))
    src = u if key is None else _f64(key)
    um = src[0] + src[1]
    g = envelope(um * um, alpha)
    Gu = np.log(g + eps)
    Gy = curve(Gu, T, W, R)[0]
    y = np.exp(Gy - Gu)[None, :] * u
    return (y, g) if return_env else y


def compressor_bwd(u, p, ybar, eps=COMP_EPS, curve=knee, key=None):
    """Adjoint of ``compressor_fwd``: (ubar, pbar), or (ubar, keybar, pbar) with a key."""
    u, ybar = _f64(u), _f64(ybar)
    alpha, T, W, R = (float(v) for v in _f64(p))
    src = u if key is None else _f64(key)
    um = src[0] + src[1]
    x = um * um
    g = envelope(x, alpha)
    Gu = np.log(g + eps)
    Gy, dGu, dT, dW, dR = curve(Gu, T, W, R)
    k = np.exp(Gy - Gu)
    kbar = np.sum(ybar * u, axis=0)
    Gybar = kbar * k
    gbar = Gybar * (dGu - 1.0) / (g + eps)
    lam = envelope_reverse(gbar, alpha)
    xbar = (1.0 - alpha) * lam
    srcbar = (2.0 * um * xbar)[None, :] * np.ones((2, 1))
    gprev = np.concatenate([[0.0], g[:-1]])
    pbar = np.array([np.sum(lam * (gprev - x)), np.sum(Gybar * dT),
                     np.sum(Gybar * dW), np.sum(Gybar * dR)])
    if key is None:
        return k[None, :] * ybar + srcbar, pbar
    return k[None, :] * ybar, srcbar, pbar


# ---------------------------------------------------------------- attack/release ballistics (Sec. 3, Eq. 8)
# Eq. 8 with the coefficient the paper describes before restricting it: alpha[n] is the
# attack constant while the envelope rises (x[n] > g[n-1]) and the release constant while
# it falls, g[n] = alpha[n] g[n-1] + (1 - alpha[n]) x[n], g[-1] = 0.  The rest is the
# compressor of Eq. 9-12.  Parameter row [alpha_attack, alpha_release, T, W, R].  The
# branch is a comparison, so the derivative treats it as fixed (ties have measure zero).
def envelope_ar(x, aa, ar):
    """(g, attack mask) of the attack/release recursion, run sample by sample."""
    x = _f64(x)
    g = np.empty_like(x)
    att = np.empty(x.shape[0], dtype=bool)
    prev = 0.0
    for n in range(x.shape[0]):
        att[n] = x[n] > prev
        a = aa if att[n] else ar
        prev = a * prev + (1.0 - a) * x[n]
        g[n] = prev
    return g, att


def ballistic_fwd(u, p, eps=COMP_EPS):
    u = _f64(u)
    aa, ar, T, W, R = (float(v) for v in _f64(p))
    um = u[0] + u[1]
    g, _ = envelope_ar(um * um, aa, ar)
    Gu = np.log(g + eps)
    Gy = knee(Gu, T, W, R)[0]
    return np.exp(Gy - Gu)[None, :] * u


def ballistic_bwd(u, p, ybar, eps=COMP_EPS):
    u, ybar = _f64(u), _f64(ybar)
    aa, ar, T, W, R = (float(v) for v in _f64(p))
    um = u[0] + u[1]
    x = um * um
    g, att = envelope_ar(x, aa, ar)
    alpha = np.where(att, aa, ar)
    Gu = np.log(g + eps)
    Gy, dGu, dT, dW, dR = knee(Gu, T, W, R)
    k = np.exp(Gy - Gu)
    Gybar = np.sum(ybar * u, axis=0) * k
    gbar = Gybar * (dGu - 1.0) / (g + eps)
    # lambda[n] = gbar[n] + alpha[n+1] lambda[n+1] (the coefficient of step n+1)
    lam = np.empty_like(gbar)
    acc = 0.0
    for n in range(gbar.shape[0] - 1, -1, -1):
        acc = gbar[n] + (alpha[n + 1] * acc if n + 1 < gbar.shape[0] else 0.0)
        lam[n] = acc
    xbar = (1.0 - alpha) * lam
    ubar = k[None, :] * ybar + (2.0 * um * xbar)[None, :]
    gprev = np.concatenate([[0.0], g[:-1]])
    da = lam * (gprev - x)
    pbar = np.array([np.sum(da[att]), np.sum(da[~att]), np.sum(Gybar * dT), np.sum(Gybar * dW),
                     np.sum(Gybar * dR)])
    return ubar, pbar


# ---------------------------------------------------------------- MIMO processors (Sec. 2 Definitions, Eq. 1a/1b)
# The paper's nodes take M inputs and give N outputs, each edge carrying its (output,
# input) port pair.  Its Sec. 3 processors are all single-input single-output; these
# three multi-port processors of a mixing console exercise the general form:
#   * split (1 in, 2 out): mid and side as separate stereo rows, y0 = (m, m) with
#     m = (l + r)/2, y1 = (s, s) with s = (l - r)/2;
#   * merge (2 in, 1 out): back to left/right, y = (u0_l + u1_l, u0_r - u1_r), so that
#     merge(split(u)) = u;
#   * sidechain compressor (2 in: main, key; 1 out): the compressor of Eq. 8-12 with
#     the envelope computed from the key input and the gain applied to the main input.
def split_fwd(u):
    u = _f64(u)
    m = (u[0] + u[1]) / 2
    s = (u[0] - u[1]) / 2
    return [np.stack([m, m]), np.stack([s, s])]


def split_bwd(u, ybars):
    """ybars: the adjoints of both outputs; returns [ubar]."""
    a = np.sum(_f64(ybars[0]), axis=0) / 2
    b = np.sum(_f64(ybars[1]), axis=0) / 2
    return [np.stack([a + b, a - b])]


def merge_fwd(us):
    u0, u1 = _f64(us[0]), _f64(us[1])
    return np.stack([u0[0] + u1[0], u0[1] - u1[1]])


def merge_bwd(us, ybar):
    ybar = _f64(ybar)
    return [ybar.copy(), np.stack([ybar[0], -ybar[1]])]


def sidechain_fwd(us, p, eps=COMP_EPS):
    return compressor_fwd(us[0], p, eps, key=us[1])


def sidechain_bwd(us, p, ybar, eps=COMP_EPS):
    """Returns ([ubar_main, ubar_key], pbar)."""
    ub, kb, pb = compressor_bwd(us[0], p, ybar, eps, key=us[1])
    return [ub, kb], pb


# ---------------------------------------------------------------- noisegate (Eq. 13)
def noisegate_fwd(u, p, eps=COMP_EPS):
    return compressor_fwd(u, p, eps, curve=gate_curve)


def noisegate_bwd(u, p, ybar, eps=COMP_EPS):
    return compressor_bwd(u, p, ybar, eps, curve=gate_curve)


# ---------------------------------------------------------------- mix / output
def identity_fwd(u, p=None):
    return _f64(u).copy()


def identity_bwd(u, p, ybar):
    return _f64(ybar).copy(), np.zeros(0)


# ---------------------------------------------------------------- multitap delay (Eq. 14-15)
# Readings: each channel has M taps, each a delay d_m and a 39-tap zero-phase FIR
# c_m built like the EQ from 20 log-magnitudes.  Two layouts:
#   * compact (default): M = 4 taps, each anywhere in [0, N_d), N_d = 32768
#     (>= 500 ms at 44.1 kHz);
#   * the paper's setting: a 2 s effect with at most one delay in every 100 ms
#     (M = 20): tap m lives in its own slot [m S, m S + S), S = fs / 10 = 4410
#     samples, and its surrogate transform spans the slot (N_d = S).
# The delay used by the forward pass is d_m = m S + (round(N_d (-arg z_m) / 2 pi)
# mod N_d) (S = 0 in the compact layout), which makes Eq. 15 exact at |z| = 1 with
# integer phase.  The forward pass uses the exact integer delays (straight-through);
# the z-gradient is the gradient of the surrogate of Eq. 15 placed at the slot,
# s_m[n] = Re{(1/N_d) sum_k z^k w^{k (n - m S)}}, n in [m S, m S + N_d).
# Parameter row: [channel][tap][re, im, 20 log-magnitudes] = 2 x M x 22
# (176 compact, 880 paper).
DELAY_NFFT = 32768
DELAY_TAPS = 4
DELAY_FIR = 39
DELAY_K = 20
DELAY_PAPER_TAPS = 20


def delay_paper_hp(fs=44100):
    """Layout of the paper's multitap delay: 20 taps per channel in 100 ms slots."""
    return dict(delay_taps=DELAY_PAPER_TAPS, delay_nfft=fs // 10, delay_slot=fs // 10)


def delay_split(p, taps=DELAY_TAPS):
    q = _f64(p).reshape(2, taps, 2 + DELAY_K)
    z = q[..., 0] + 1j * q[..., 1]
    return z, q[..., 2:]


def delay_samples(z, nfft=DELAY_NFFT, slot=0):
    """d_m = m S + (round(N_d (-arg z_m) / 2 pi) mod N_d), m along the last axis."""
    d = np.mod(np.rint(nfft * (-np.angle(z)) / (2 * np.pi)).astype(np.int64), nfft)
    return d + slot * np.arange(np.shape(z)[-1])


def delay_fir(p, nfft=DELAY_NFFT, taps=DELAY_TAPS, slot=0):
    """Per channel the sparse FIR h_x[n] = sum_m c_m[n - d_m] as (offset, taps):
    h_x is stored from n = offset."""
    z, lm = delay_split(p, taps)
    d = delay_samples(z, nfft, slot)
    H = (DELAY_FIR - 1) // 2
    out = []
    for x in range(2):
        lo = int(d[x].min()) - H
        hi = int(d[x].max()) + H
        h = np.zeros(hi - lo + 1)
        for m in range(taps):
            c = zerophase_taps(lm[x, m], DELAY_FIR)
            s = int(d[x, m]) - H - lo
            h[s:s + DELAY_FIR] += c
        out.append((lo, h))
    return out


def _fir_at(u, h, lo):
    """y[t] = sum_i h[i] u[t - (lo + i)] (taps starting at delay lo), u = 0 outside
    [0, L), truncated to [0, L)."""
    L = u.shape[-1]
    full = scipy.signal.fftconvolve(u, h)             # full[q] = sum_i h[i] u[q - i]
    q = np.arange(L) - lo
    ok = (q >= 0) & (q < full.shape[0])
    y = np.zeros(L)
    y[ok] = full[q[ok]]
    return y


def delay_fwd(u, p, nfft=DELAY_NFFT, taps=DELAY_TAPS, slot=0):
    """Eq. 14 with the exact integer delays: y_x = sum_m c_{x,m} * delta[n - d_{x,m}] * u_x."""
    u = _f64(u)
    return np.stack([_fir_at(u[x], h, lo) for x, (lo, h) in enumerate(delay_fir(p, nfft, taps, slot))])


def _corr_lags(u, ybar, lo, hi):
    """r[n] = sum_t ybar[t] u[t - n] for n in [lo, hi]."""
    L = u.shape[-1]
    c = scipy.signal.fftconvolve(ybar, u[::-1])       # c[j] = sum_t ybar[t] u[t - (j - L + 1)]
    n = np.arange(lo, hi + 1)
    j = n + L - 1
    ok = (j >= 0) & (j < c.shape[0])
    r = np.zeros(n.shape[0])
    r[ok] = c[j[ok]]
    return r


def delay_surrogate_dz(g, z, nfft=DELAY_NFFT):
    """d/d(re, im) of sum_n g[n] s[n] with s[n] = Re{(1/N) sum_k z^k w^{kn}}, w = e^{2 pi j/N}:
    Q = sum_k k z^{k-1} ifft(g)[k]; d/dre = Re Q, d/dim = -Im Q."""
    G = np.fft.ifft(g)
    k = np.arange(nfft)
    zk = np.exp((k - 1) * np.log(complex(z))) if z != 0 else (k == 1).astype(complex)
    Q = np.sum(k * zk * G)
    return np.real(Q), -np.imag(Q)


def delay_bwd(u, p, ybar, nfft=DELAY_NFFT, taps=DELAY_TAPS, slot=0):
    u, ybar = _f64(u), _f64(ybar)
    z, lm = delay_split(p, taps)
    d = delay_samples(z, nfft, slot)
    H = (DELAY_FIR - 1) // 2
    firs = delay_fir(p, nfft, taps, slot)
    ubar = np.stack([_fir_at(ybar[x], h[::-1], -(lo + h.shape[0] - 1)) for x, (lo, h) in enumerate(firs)])
    pbar = np.zeros((2, taps, 2 + DELAY_K))
    reach = (taps - 1) * slot + nfft                    # surrogates cover n in [0, reach)
    for x in range(2):
        r = _corr_lags(u[x], ybar[x], -H, reach - 1 + H)  # r[n], n in [-H, reach + H)
        for m in range(taps):
            c = zerophase_taps(lm[x, m], DELAY_FIR)
            # taps: dL/dc[j] = r[d + j], j in [-H, H]
            cbar = r[d[x, m] + np.arange(-H, H + 1) + H]
            pbar[x, m, 2:] = zerophase_taps_bwd(lm[x, m], DELAY_FIR, cbar)
            # surrogate at the slot: g[n] = dL/ds_m[m S + n] = sum_j c[j] r[m S + n + j], n in [0, N_d)
            g = np.zeros(nfft)
            base = m * slot
            for jj, cj in enumerate(c):
                g += cj * r[base + jj:base + jj + nfft]
            pbar[x, m, 0], pbar[x, m, 1] = delay_surrogate_dz(g, z[x, m], nfft)
    return ubar, pbar.reshape(-1)


def delay_fwd_surrogate(u, p, nfft=DELAY_NFFT, taps=DELAY_TAPS, slot=0):
    """Forward through the surrogate of Eq. 15 (for checking the z-gradient by finite
    differences): y_x = sum_m s_m * c_m * u_x with s_m[n] = Re{IDFT(z^k)}[n - m S]."""
    u = _f64(u)
    z, lm = delay_split(p, taps)
    H = (DELAY_FIR - 1) // 2
    k = np.arange(nfft)
    y = np.zeros_like(u)
    for x in range(2):
        for m in range(taps):
            s = np.real(np.fft.ifft(np.exp(k * np.log(complex(z[x, m])))))
            c = zerophase_taps(lm[x, m], DELAY_FIR)
            y[x] += _fir_at(u[x], np.convolve(s, c), m * slot - H)
    return y


# ---------------------------------------------------------------- filtered-noise reverb (Eq. 6-7)
# Readings (the paper gives the model, not these constants): two noise buffers (mid,
# side) of 2 s = 88200 samples, U(-1, 1), are inputs shared by every reverb node (the
# random numbers the method draws are passed in); STFT with FFT 1024, hop 256,
# periodic Hann, centred frames (frame m = 1..F covers [(m-1) hop - N/2, (m-1) hop + N/2),
# the signal zero outside [0, 88200)), F = 1 + 88200 // 256; masks
# M_x[k, m] = exp(H0_x[k] + (m-1) Hd_x[k]) with H0, Hd interpolated from 12
# log-spaced bands like the EQ (natural-log magnitudes); ISTFT by windowed
# overlap-add divided by the window envelope sum w^2 (bounded below by centring); h_l =
# (h_m + h_s)/2, h_r = (h_m - h_s)/2 (the imager's convention); y = e^{q_dry} u +
# e^{q_wet} (h * u), causal, truncated to L.
# Parameter row (50): [mid, side] x [H0 (12), Hd (12)], then q_dry, q_wet.
# The paper's own setting (rv_mode "paper"): FFT 384, hop 192, the masks' log-magnitudes
# are the parameters themselves, 192 per filter for bins 0..191 (the one-sided spectrum
# has 193 bins: the Nyquist bin 192 is dropped, mask 0), and the output is the wet
# convolution alone, y = h * u.  Parameter row (768): [mid, side] x [H0 (192), Hd (192)].
RV_LEN = 88200
RV_NFFT = 1024
RV_HOP = 256
RV_BANDS = 12
RV_PAPER = dict(rv_nfft=384, rv_hop=192, rv_mode="paper")


def rv_hp(hp=None):
    d = dict(rv_len=RV_LEN, rv_nfft=RV_NFFT, rv_hop=RV_HOP, fs=44100, rv_mode="bands")
    if hp:
        d.update({k: v for k, v in hp.items() if k in d})
    return d


def rv_cols(hp=None):
    """Parameter columns of one reverb row."""
    h = rv_hp(hp)
    return 4 * (h["rv_nfft"] // 2) if h["rv_mode"] == "paper" else 50


def rv_band_matrix(nfft, fs=44100, n_bands=RV_BANDS):
    """Bins 0..nfft/2 at k fs / nfft; the same log2-interpolation rule as the EQ."""
    c = 20.0 * 1000.0 ** ((np.arange(n_bands) + 0.5) / n_bands)
    lc = np.log2(c)
    B = np.zeros((nfft // 2 + 1, n_bands))
    for k in range(nfft // 2 + 1):
        f = k * fs / nfft
        if f <= c[0]:
            B[k, 0] = 1.0
        elif f >= c[-1]:
            B[k, -1] = 1.0
        else:
            b = int(np.searchsorted(c, f, side="right")) - 1
            w = (np.log2(f) - lc[b]) / (lc[b + 1] - lc[b])
            B[k, b], B[k, b + 1] = 1.0 - w, w
    return B


def rv_window(n):
    return 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n) / n)


def rv_frames(length, nfft, hop):
    return 1 + length // hop


def _rv_padded_len(length, nfft, hop):
    return (rv_frames(length, nfft, hop) - 1) * hop + nfft


def rv_stft(x, nfft, hop):
    """[F, nfft/2+1] one-sided spectra of centred frames (frame m covers
    [m hop - nfft/2, m hop + nfft/2)), zero outside the signal."""
    F = rv_frames(x.shape[0], nfft, hop)
    pad = np.zeros(_rv_padded_len(x.shape[0], nfft, hop))
    pad[nfft // 2:nfft // 2 + x.shape[0]] = x
    idx = np.arange(F)[:, None] * hop + np.arange(nfft)[None, :]
    return np.fft.rfft(pad[idx] * rv_window(nfft)[None, :], axis=-1)


def rv_ola_norm(length, nfft, hop):
    """Window envelope sum_m w^2 at every sample of [0, length)."""
    F = rv_frames(length, nfft, hop)
    D = np.zeros(_rv_padded_len(length, nfft, hop))
    w2 = rv_window(nfft) ** 2
    for m in range(F):
        D[m * hop:m * hop + nfft] += w2
    return D[nfft // 2:nfft // 2 + length]


def rv_istft(S, length, nfft, hop):
    """Windowed overlap-add of irfft frames divided by the window envelope."""
    F = S.shape[0]
    fr = np.fft.irfft(S, nfft, axis=-1) * rv_window(nfft)[None, :]
    out = np.zeros(_rv_padded_len(length, nfft, hop))
    for m in range(F):
        out[m * hop:m * hop + nfft] += fr[m]
    D = rv_ola_norm(length, nfft, hop)
    h = np.zeros(length)
    ok = D > 1e-8
    h[ok] = out[nfft // 2:nfft // 2 + length][ok] / D[ok]
    return h


def rv_log_filters(p, nfft, fs=44100, mode="bands"):
    """Per channel x (mid, side) the per-bin log-magnitudes (H0_x[k], Hd_x[k]) of Eq. 7
    over the nfft/2+1 one-sided bins; in the paper's mode the Nyquist bin is None."""
    q = _f64(p)
    out = []
    if mode == "paper":
        K = nfft // 2
        for x in range(2):
            out.append((q[x * 2 * K:x * 2 * K + K], q[x * 2 * K + K:x * 2 * K + 2 * K]))
        return out
    B = rv_band_matrix(nfft, fs)
    for x in range(2):
        out.append((B @ q[x * 24:x * 24 + 12], B @ q[x * 24 + 12:x * 24 + 24]))
    return out


def rv_masks(p, nfft, F, fs=44100, mode="bands"):
    """M_x[m, k] = exp(H0_x[k] + m Hd_x[k]) (Eq. 7, m the 0-based frame), [F, nfft/2+1]."""
    out = []
    for H0, Hd in rv_log_filters(p, nfft, fs, mode):
        M = np.zeros((F, nfft // 2 + 1))
        K = H0.shape[0]
        M[:, :K] = np.exp(H0[None, :] + np.arange(F)[:, None] * Hd[None, :])
        out.append(M)
    return out


def rv_ir(p, noise, hp=None):
    """Stereo IR [2, length] of one reverb node from its parameters and the noise."""
    hp = rv_hp(hp)
    n, hop, length = hp["rv_nfft"], hp["rv_hop"], hp["rv_len"]
    F = rv_frames(length, n, hop)
    Ms = rv_masks(p, n, F, hp["fs"], hp["rv_mode"])
    hm = rv_istft(rv_stft(_f64(noise[0][:length]), n, hop) * Ms[0], length, n, hop)
    hs = rv_istft(rv_stft(_f64(noise[1][:length]), n, hop) * Ms[1], length, n, hop)
    return np.stack([(hm + hs) / 2, (hm - hs) / 2])


def _causal(u, h):
    L = u.shape[-1]
    return scipy.signal.fftconvolve(u, h)[:L]


def reverb_fwd(u, p, noise, hp=None):
    h_ = rv_hp(hp)
    u, q = _f64(u), _f64(p)
    h = rv_ir(q, noise, hp)
    wet = np.stack([_causal(u[x], h[x]) for x in range(2)])
    if h_["rv_mode"] == "paper":
        return wet
    return np.exp(q[48]) * u + np.exp(q[49]) * wet


def reverb_bwd(u, p, ybar, noise, hp=None):
    hp = rv_hp(hp)
    paper = hp["rv_mode"] == "paper"
    u, q, ybar = _f64(u), _f64(p), _f64(ybar)
    n, hop, length = hp["rv_nfft"], hp["rv_hop"], hp["rv_len"]
    F = rv_frames(length, n, hop)
    h = rv_ir(q, noise, hp)
    a_dry, a_wet = (0.0, 1.0) if paper else (np.exp(q[48]), np.exp(q[49]))
    L = u.shape[-1]
    # input adjoint: dry + correlation with the IR
    ubar = a_dry * ybar + a_wet * np.stack([scipy.signal.fftconvolve(ybar[x][::-1], h[x])[:L][::-1]
                                            for x in range(2)])
    # r_x[n] = sum_t ybar[t] u[t - n], n in [0, length)
    r = np.stack([scipy.signal.fftconvolve(ybar[x], u[x][::-1])[L - 1:L - 1 + length] for x in range(2)])
    if r.shape[1] < length:
        r = np.pad(r, ((0, 0), (0, length - r.shape[1])))
    pbar = np.zeros(rv_cols(hp))
    if not paper:
        pbar[48] = a_dry * np.sum(ybar * u)
        pbar[49] = a_wet * np.sum(h * r)
    hbar = a_wet * r                                       # dL/dh_l, dL/dh_r
    hbar_ms = [(hbar[0] + hbar[1]) / 2, (hbar[0] - hbar[1]) / 2]
    D = rv_ola_norm(length, n, hop)
    Ms = rv_masks(q, n, F, hp["fs"], hp["rv_mode"])
    w = rv_window(n)
    ck = np.full(n // 2 + 1, 2.0)
    ck[0] = ck[-1] = 1.0
    for x in range(2):
        g = np.zeros(length)
        ok = D > 1e-8
        g[ok] = hbar_ms[x][ok] / D[ok]
        gp = np.zeros(_rv_padded_len(length, n, hop))
        gp[n // 2:n // 2 + length] = g
        idx = np.arange(F)[:, None] * hop + np.arange(n)[None, :]
        xbar = gp[idx] * w[None, :]                          # dL/d(irfft frame)
        Gb = ck[None, :] / n * np.fft.rfft(xbar, axis=-1)    # dL/dRe H + j dL/dIm H
        Ux = rv_stft(_f64(noise[x][:length]), n, hop)
        Mbar = np.real(Gb) * np.real(Ux) + np.imag(Gb) * np.imag(Ux)
        MM = Ms[x] * Mbar
        dH0 = MM.sum(axis=0)
        dHd = (np.arange(F)[:, None] * MM).sum(axis=0)
        if paper:
            K = n // 2
            pbar[x * 2 * K:x * 2 * K + K] = dH0[:K]
            pbar[x * 2 * K + K:x * 2 * K + 2 * K] = dHd[:K]
        else:
            B = rv_band_matrix(n, hp["fs"])
            pbar[x * 24:x * 24 + 12] = B.T @ dH0
            pbar[x * 24 + 12:x * 24 + 24] = B.T @ dHd
    return ubar, pbar
