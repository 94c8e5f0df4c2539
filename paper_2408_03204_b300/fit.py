"""Gradient-descent fit of every processor parameter of a plan to a target mix (the
paper's example application, Sec. 4): render, MRSTFT loss, loss gradient, backprop and
a fused Adam step per type, all through the C-ABI library on one stream.  A whole step
(Adam included, its step counter on the device) can be replayed as one CUDA graph.

Unconstrained variables theta map to the processors' parameters column by column
(grafx_adam_step codes): compressor and noisegate [alpha, T, W, R] -> [alpha map,
identity, softplus, 1 + softplus]; reverb decay columns -> -softplus; a delay tap's
(Re z, Im z) is updated with its gradient normalised and a unit-circle penalty added
(Sec. 3 "Multitap delay"); everything else identity.
"""
import ctypes

from . import PARAM_COLS, T_BALLISTIC, T_COMP, T_DELAY, T_GATE, T_REVERB, T_SIDECHAIN, _check, _ptr, _stream_of, lib

MAP_IDENT, MAP_ALPHA, MAP_SOFTPLUS, MAP_RATIO, MAP_NEGSP, MAP_ATTACK, MAP_ZRE, MAP_ZIM = range(8)


def param_codes(t, cols=None):
    """Per-column map codes of parameter type t (a list of cols ints; cols defaults to
    the compact layout's width PARAM_COLS[t])."""
    cols = PARAM_COLS[t] if cols is None else cols
    if t in (T_COMP, T_GATE, T_SIDECHAIN):
        return [MAP_ALPHA, MAP_IDENT, MAP_SOFTPLUS, MAP_RATIO]
    if t == T_BALLISTIC:
        return [MAP_ATTACK, MAP_ALPHA, MAP_IDENT, MAP_SOFTPLUS, MAP_RATIO]
    if t == T_REVERB and cols == 50:
        # [mid/side][H0 x 12, H_delta x 12], then wet and dry gains
        return ([MAP_IDENT] * 12 + [MAP_NEGSP] * 12) * 2 + [MAP_IDENT, MAP_IDENT]
    if t == T_REVERB:
        # per-bin layout: [mid/side][H0 x K, H_delta x K]
        K = cols // 4
        return ([MAP_IDENT] * K + [MAP_NEGSP] * K) * 2
    if t == T_DELAY:
        # per (channel, tap): [Re z, Im z, 20 log-magnitudes]; z normalised and regularised
        return ([MAP_ZRE, MAP_ZIM] + [MAP_IDENT] * 20) * (cols // 22)
    return [MAP_IDENT] * cols


def neutral_params(plan, torch, device):
    """Nearly transparent physical parameters for every type the plan holds: 0 dB gains,
    flat EQ, centred image, compressor and noisegate with ratio 1.001, delays of
    44 samples (1 ms) into each slot through taps of 1/(taps per channel), reverb dry
    only (wet gain e^-30; the paper's wet-only reverb gets a quiet -36 dB, 0.5 s tail)."""
    import math
    P = {}
    for t, cols in plan.param_cols.items():
        rows = plan.info.n_type_rows[t]
        if not rows:
            continue
        p = torch.zeros((rows, cols), dtype=torch.float32, device=device)
        if t == T_BALLISTIC:
            p[:, 0], p[:, 1], p[:, 2], p[:, 3], p[:, 4] = 0.95, 0.999, 0.0, 3.0 * math.log(10.0) / 10.0, 1.001
        if t in (T_COMP, T_GATE, T_SIDECHAIN):  # ratio 1.001: (nearly) no compression / expansion
            p[:, 0], p[:, 1], p[:, 2], p[:, 3] = 0.99, 0.0, 3.0 * math.log(10.0) / 10.0, 1.001
        if t == T_DELAY:
            taps = cols // 44
            q = p.view(rows, 2, taps, 22)
            ang = -2.0 * math.pi * 44 / (32768 if taps == 4 else plan.sample_rate // 10)
            q[..., 0], q[..., 1], q[..., 2:] = math.cos(ang), math.sin(ang), math.log(1.0 / taps)
        if t == T_REVERB and cols == 50:
            p[:, 12:24] = -0.05
            p[:, 36:48] = -0.05
            p[:, 49] = -30.0
        elif t == T_REVERB:
            K = cols // 4
            q = p.view(rows, 2, 2, K)
            q[:, :, 0] = -36.0 * math.log(10.0) / 20.0
            q[:, :, 1] = -3.0 * math.log(10.0) * 192 / (0.5 * plan.sample_rate)
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
        self.codes = {t: torch.tensor(param_codes(t, self.P[t].shape[1]), dtype=torch.int8, device=dev)
                      for t in self.P}
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
        with torch.cuda.stream(self.stream):
            self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.t = 0
        self.graph = None
        if use_graph:
            # the whole step (render, loss, loss gradient, backprop, step counter, Adam of
            # every type) as one CUDA graph replayed with a single launch
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._body()
            self.stream.synchronize()

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

    def _body(self):
        st = _stream_of(self.torch.cuda.current_stream(self.src.device))
        self.plan.render_raw(self.src, self.out, st)
        self.plan.loss_raw(self.out, self.tgt, self.loss, st)
        self.plan.loss_backward_raw(self.out, self.tgt, self.d_out, st)
        self.plan.backprop_raw(self.src, self.d_out, self.g, None, st)
        self.step_dev.add_(1)
        for t, p in self.P.items():
            _check(lib().grafx_adam_step_dev(_ptr(self.theta[t]), _ptr(self.m[t]), _ptr(self.v[t]), _ptr(self.g[t]),
                                             _ptr(p), _ptr(self.codes[t]), p.shape[1], p.numel(), _ptr(self.step_dev),
                                             ctypes.c_float(self.lr), ctypes.c_float(self.b1),
                                             ctypes.c_float(self.b2), ctypes.c_float(self.eps), st))

    def step(self):
        """One fit step (loss of the current parameters, then the Adam update), queued on
        the fit's stream."""
        self.t += 1
        with self.torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._body()

    def save(self, path):
        """Write the fit's state (theta, Adam moments and step of every type) to `path`."""
        from .state import save_state
        self.stream.synchronize()
        tensors = {}
        for t in self.P:
            tensors[f"theta.{t}"], tensors[f"m.{t}"], tensors[f"v.{t}"] = self.theta[t], self.m[t], self.v[t]
        tensors["step"] = self.step_dev
        save_state(path, tensors, {"kind": "fit", "t": self.t, "lr": self.lr, "betas": [self.b1, self.b2],
                                   "eps": self.eps, "types": sorted(int(t) for t in self.P)})

    def load(self, path):
        """Resume from a file written by save() for the same plan: theta, moments and step
        are restored and the parameters set to map(theta)."""
        from .state import load_state
        tensors, meta = load_state(path, self.src.device)
        if meta.get("kind") != "fit" or sorted(meta["types"]) != sorted(int(t) for t in self.P):
            raise ValueError(f"{path}: not a fit state for these parameter types")
        with self.torch.cuda.stream(self.stream):
            for t in self.P:
                for name, dst in (("theta", self.theta[t]), ("m", self.m[t]), ("v", self.v[t])):
                    src = tensors[f"{name}.{t}"]
                    if src.shape != dst.shape:
                        raise ValueError(f"{path}: {name}.{t} has shape {tuple(src.shape)}, want {tuple(dst.shape)}")
                    dst.copy_(src)
            self.step_dev.copy_(tensors["step"])
        self.t = int(meta["t"])
        self._apply_map()

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


def main():
    """Fit of a random console with every processor type (reverb included) to a target
    rendered from hidden parameters; prints one JSON line with the time per step, the
    total time and the loss curve summary.

        python -m paper_2408_03204_b300.fit --nodes 200 --length 262144 --steps 1000
    """
    import argparse
    import json

    import numpy as np
    import torch

    import synth
    from . import Graph, Plan

    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=200)
    ap.add_argument("--length", type=int, default=2 ** 18)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--checkpoint-steps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=4)
    args = ap.parse_args()
    g = synth.console_all_types(args.seed, args.nodes)
    L = args.length
    dev = torch.device("cuda")
    plan = Plan([Graph.from_lists(g.types, g.edges)], [L], checkpoint_steps=args.checkpoint_steps)
    ws_plain = Plan([Graph.from_lists(g.types, g.edges)], [L]).info.ws_bytes
    plan.bind_workspace(dev)
    noise = torch.tensor(synth.reverb_noise(), device=dev).contiguous()
    plan.bind_reverb_noise(noise)
    P = (L + 3) // 4 * 4
    src = torch.tensor(synth.sources(args.seed, g.count(synth.I), L, pitch=P).reshape(-1), device=dev)
    hidden = {t: torch.tensor(a, device=dev).contiguous() for t, a in synth.random_params(g, 100 + args.seed).items()}
    target = torch.empty(plan.info.out_elems, device=dev)
    plan.bind_params(hidden)
    plan.render_raw(src, target, _stream_of(torch.cuda.current_stream(dev)))
    f = Fit(plan, src, target, neutral_params(plan, torch, dev), lr=args.lr)
    hist = torch.zeros(args.steps, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(f.stream):
        e0.record(f.stream)
        for i in range(args.steps):
            f.step()
            hist[i:i + 1].copy_(f.loss)
        e1.record(f.stream)
    f.stream.synchronize()
    plan.sync_status(f.st)
    h = hist.cpu().numpy()
    ms = e0.elapsed_time(e1)
    print(json.dumps(dict(nodes=g.n_nodes, types="".join(synth.TYPE_LETTERS[t] for t in sorted(set(g.types))), length=L,
                          steps=args.steps, lr=args.lr, checkpoint_steps=args.checkpoint_steps,
                          ws_bytes=int(plan.info.ws_bytes), ws_bytes_without_checkpointing=int(ws_plain),
                          ms_per_step=ms / args.steps, total_s=ms / 1e3, loss_first=float(h[0]),
                          loss_at=[float(h[min(k, args.steps - 1)]) for k in (10, 100, 200, 500, 999)],
                          loss_final=float(h[-1]), loss_min=float(np.min(h)), gpu=torch.cuda.get_device_name())))


if __name__ == "__main__":
    main()
