"""Gradient-descent fit of every processor parameter of a plan to a target mix (the
paper's example application, Sec. 4): render, MRSTFT loss, loss gradient, backprop and
a fused Adam step per type, all through the C-ABI library on one stream.  The render,
loss and backprop of a step can be replayed as one captured CUDA graph.

Unconstrained variables theta map to the processors' parameters column by column
(grafx_adam_step codes): compressor [alpha, T, W, R] -> [alpha map, identity, softplus,
1 + softplus]; reverb decay columns -> -softplus; everything else identity.
"""
import ctypes

from . import PARAM_COLS, T_COMP, T_DELAY, T_REVERB, _check, _ptr, _stream_of, lib

MAP_IDENT, MAP_ALPHA, MAP_SOFTPLUS, MAP_RATIO, MAP_NEGSP = range(5)


def param_codes(t):
    """Per-column map codes of parameter type t (a list of PARAM_COLS[t] ints)."""
    cols = PARAM_COLS[t]
    if t == T_COMP:
        return [MAP_ALPHA, MAP_IDENT, MAP_SOFTPLUS, MAP_RATIO]
    if t == T_REVERB:
        # [mid/side][H0 x 12, H_delta x 12], then wet and dry gains
        return ([MAP_IDENT] * 12 + [MAP_NEGSP] * 12) * 2 + [MAP_IDENT, MAP_IDENT]
    return [MAP_IDENT] * cols


def neutral_params(plan, torch, device):
    """Nearly transparent physical parameters for every type the plan holds: 0 dB gains,
    flat EQ, centred image, compressor with ratio 1.001 at a 0 dB threshold, delays of
    44 samples (1 ms) through four 0.25 taps, reverb dry only (wet gain e^-30)."""
    import math
    P = {}
    for t, cols in PARAM_COLS.items():
        rows = plan.info.n_type_rows[t]
        if not rows:
            continue
        p = torch.zeros((rows, cols), dtype=torch.float32, device=device)
        if t == T_COMP:
            p[:, 0], p[:, 1], p[:, 2], p[:, 3] = 0.99, 0.0, 3.0 * math.log(10.0) / 10.0, 1.001
        if t == T_DELAY:
            q = p.view(rows, 2, 4, 22)
            ang = -2.0 * math.pi * 44 / 32768
            q[..., 0], q[..., 1], q[..., 2:] = math.cos(ang), math.sin(ang), math.log(0.25)
        if t == T_REVERB:
            p[:, 12:24] = -0.05
            p[:, 36:48] = -0.05
            p[:, 49] = -30.0
        P[t] = p
    return P


class Fit:
    """Adam on theta for every parameter type of ``plan`` (workspace bound, reverb noise
    bound if needed).  ``params``: device float32 physical parameters per type (updated in
    place every step); ``theta0`` (optional) the unconstrained start, else the inverse
    map of ``params``."""

    def __init__(self, plan, sources, target, params, lr=1e-2, betas=(0.9, 0.999), eps=1e-8,
                 use_graph=True, stream=None, theta0=None):
        import torch
        self.torch = torch
        dev = sources.device
        self.plan, self.src, self.tgt = plan, sources, target
        self.stream = stream or torch.cuda.Stream(dev)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        self.st = _stream_of(self.stream)
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.P = params
        plan.bind_params(self.P)
        self.codes = {t: torch.tensor(param_codes(t), dtype=torch.int8, device=dev) for t in self.P}
        self.theta, self.m, self.v, self.g = {}, {}, {}, {}
        with torch.cuda.stream(self.stream):
            for t, p in self.P.items():
                self.theta[t] = torch.empty_like(p)
                if theta0 is not None and t in theta0:
                    self.theta[t].copy_(theta0[t])
                else:
                    _check(lib().grafx_params_to_theta(_ptr(p), _ptr(self.codes[t]), p.shape[1], p.numel(),
                                                       _ptr(self.theta[t]), self.st))
                self.m[t] = torch.zeros_like(p)
                self.v[t] = torch.zeros_like(p)
                self.g[t] = torch.zeros_like(p)
            self.out = torch.empty(plan.info.out_elems, dtype=torch.float32, device=dev)
            self.d_out = torch.empty_like(self.out)
            self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        if theta0 is not None:
            self._apply_map()
        self.t = 0
        self.graph = None
        if use_graph:
            self.stream.synchronize()
            self.graph = plan.capture_step(self.src, self.out, self.tgt, self.loss, self.d_out, self.g, None,
                                           self.st)

    def _apply_map(self):
        # param = map(theta) via a zero-learning-rate Adam step on zero gradients
        for t, p in self.P.items():
            with self.torch.cuda.stream(self.stream):
                z, m0, v0 = self.torch.zeros_like(p), self.torch.zeros_like(p), self.torch.zeros_like(p)
            _check(lib().grafx_adam_step(_ptr(self.theta[t]), _ptr(m0), _ptr(v0), _ptr(z), _ptr(p),
                                         _ptr(self.codes[t]), p.shape[1], p.numel(), 1, ctypes.c_float(0.0),
                                         ctypes.c_float(self.b1), ctypes.c_float(self.b2),
                                         ctypes.c_float(self.eps), self.st))
            self.stream.synchronize()

    def step(self):
        """One fit step (loss of the current parameters, then the Adam update)."""
        self.t += 1
        if self.graph is not None:
            self.graph.launch(self.st)
        else:
            self.plan.render_raw(self.src, self.out, self.st)
            self.plan.loss_raw(self.out, self.tgt, self.loss, self.st)
            self.plan.loss_backward_raw(self.out, self.tgt, self.d_out, self.st)
            self.plan.backprop_raw(self.src, self.d_out, self.g, None, self.st)
        for t, p in self.P.items():
            _check(lib().grafx_adam_step(_ptr(self.theta[t]), _ptr(self.m[t]), _ptr(self.v[t]), _ptr(self.g[t]),
                                         _ptr(p), _ptr(self.codes[t]), p.shape[1], p.numel(), self.t,
                                         ctypes.c_float(self.lr), ctypes.c_float(self.b1), ctypes.c_float(self.b2),
                                         ctypes.c_float(self.eps), self.st))

    def current_loss(self):
        """Loss of the parameters before the last step (synchronises the stream)."""
        self.stream.synchronize()
        return float(self.loss.item())

    def evaluate(self):
        """Loss of the current parameters (one render + loss, synchronises)."""
        self.plan.render_raw(self.src, self.out, self.st)
        self.plan.loss_raw(self.out, self.tgt, self.loss, self.st)
        self.stream.synchronize()
        return float(self.loss.item())
