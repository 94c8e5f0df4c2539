"""Learned warm start for the parameter fit (grafx_ws_* kernels): a network that maps
the log-mel of a node's input (rendered with neutral parameters) and the cross-spectral
band gain of that input against the target mix to the node's unconstrained parameters
theta.  The paper motivates such a trained
estimator (Sec. 1) and leaves it open; this is the library's own.

Everything numeric runs in the library's kernels: renders and node inputs, log-mel
features, the network forward/backward (BF16 tensor-core products, FP32 accumulation),
the masked MSE and the Adam update.  torch provides device memory, streams, random
initial weights and the index bookkeeping of minibatches.

    python -m paper_2408_03204_b300.warmstart --train-graphs 512 --test-graphs 8
trains on random consoles and prints one JSON line comparing the fit from the
predicted start (inference + 200 Adam steps) with 1000 Adam steps from neutral.
"""
import argparse
import json
import math
import time

import numpy as np

from . import (PARAM_COLS, T_COMP, T_DELAY, T_EQ, T_GAIN, T_IMAGER, T_IN, T_OUT, T_MIX, T_REVERB, WS_HEAD_OUT,
               WS_HEAD_TYPES, WS_OUTMAX, Graph, Plan, WarmStartNet, _check, _ptr, _stream_of, lib)
from . import fit as gfit

HEAD_OF = {t: i for i, t in enumerate(WS_HEAD_TYPES)}
# processor type -> head (-1: no head) and head -> output count, as lookup arrays
_HEAD_LUT = np.full(16, -1, np.int32)
_HEAD_LUT[list(HEAD_OF)] = list(HEAD_OF.values())
_HEAD_NOUT = np.asarray(WS_HEAD_OUT, np.int32)


def param_shapes():
    """(name, shape) of every weight tensor in the flat order of the kernels."""
    s = []
    cin = (256, 128, 128, 128)
    for l in range(4):
        s += [(f"conv{l}.w", (128, cin[l], 5)), (f"conv{l}.b", (128,))]
    for t, n in zip(WS_HEAD_TYPES, WS_HEAD_OUT):
        s += [(f"h{t}.w1", (288, 128)), (f"h{t}.b1", (288,)), (f"h{t}.w2", (288, 288)), (f"h{t}.b2", (288,)),
              (f"h{t}.w3", (n, 288)), (f"h{t}.b3", (n,))]
    return s


def init_weights(torch, device, seed=0):
    """He-normal weights, zero biases; the first layer is scaled by 1/8 because log-mel
    inputs have magnitudes of about 6."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for name, sh in param_shapes():
        n = int(np.prod(sh))
        if ".w" in name:
            fan_in = int(np.prod(sh[1:]))
            w = torch.randn(n, generator=g) * math.sqrt(2.0 / fan_in)
            if name == "conv0.w":
                w *= 0.125
            parts.append(w)
        else:
            parts.append(torch.zeros(n))
    return torch.cat(parts).to(device=device, dtype=torch.float32).contiguous()


class GraphBatch:
    """A plan over a batch of graphs plus host bookkeeping of its processor nodes:
    union id, type, row within the type's parameter table, output row of its graph."""

    def __init__(self, graph_lists, L, eq_taps=1023, schedule="beam"):
        self.graph_lists = graph_lists
        self.L = L
        self.plan = Plan([Graph.from_lists(t, e) for t, e in graph_lists], [L] * len(graph_lists),
                         eq_taps=eq_taps, schedule=schedule)
        ids, types, rows, outrow, graph_of = [], [], [], [], []
        cnt = {t: 0 for t in PARAM_COLS}
        base, n_out = 0, 0
        for gi, (tys, _) in enumerate(graph_lists):
            first_out = n_out
            for v, t in enumerate(tys):
                if t in HEAD_OF:  # types without a head (noisegate) keep their start
                    ids.append(base + v)
                    types.append(t)
                    rows.append(cnt[t])
                    outrow.append(first_out)
                    graph_of.append(gi)
                    cnt[t] += 1
            n_out += sum(1 for t in tys if t == T_OUT)
            base += len(tys)
        # samples sorted by head, then union id
        order = sorted(range(len(ids)), key=lambda i: (HEAD_OF[types[i]], ids[i]))
        self.ids = [ids[i] for i in order]
        self.types = [types[i] for i in order]
        self.rows = [rows[i] for i in order]
        self.outrow = [outrow[i] for i in order]
        self.graph_of = [graph_of[i] for i in order]
        self.head_count = [sum(1 for t in self.types if t == ht) for ht in WS_HEAD_TYPES]
        self.n_out_rows = n_out


class WarmStart:
    """Network weights, Adam state, target standardisation and the feature pipeline."""

    def __init__(self, max_batch=2048, max_rows=4096, max_len=2 ** 16, device="cuda", seed=0, lr=1e-3):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.net = WarmStartNet(max_batch, max_rows, max_len, device=device)
        self.max_batch, self.max_rows = max_batch, max_rows
        self.W = init_weights(torch, self.device, seed)
        assert self.W.numel() == self.net.n_params
        self.m = torch.zeros_like(self.W)
        self.v = torch.zeros_like(self.W)
        self.dW = torch.zeros_like(self.W)
        self.code = torch.zeros(1, dtype=torch.int8, device=self.device)
        self.step_no = 0
        self.lr = lr
        # per head-column standardisation of theta (fitted on the training targets)
        self.mu = torch.zeros(len(WS_HEAD_TYPES), WS_OUTMAX, device=self.device)
        self.sd = torch.ones(len(WS_HEAD_TYPES), WS_OUTMAX, device=self.device)
        # the caller's current stream: torch bookkeeping and library calls stay ordered
        self.stream = torch.cuda.current_stream(self.device)
        self.st = _stream_of(self.stream)

    # ---------------------------------------------------------------- state
    def save(self, path):
        """Weights, Adam moments and step, target standardisation (resumable training)."""
        from .state import save_state
        self.stream.synchronize()
        save_state(path, {"W": self.W, "m": self.m, "v": self.v, "mu": self.mu, "sd": self.sd},
                   {"kind": "warmstart", "step": self.step_no, "lr": self.lr, "n_params": int(self.W.numel())})

    def load(self, path):
        from .state import load_state
        tensors, meta = load_state(path, self.device)
        if meta.get("kind") != "warmstart" or meta.get("n_params") != int(self.W.numel()):
            raise ValueError(f"{path}: not a warm-start state of this network")
        for name in ("W", "m", "v", "mu", "sd"):
            getattr(self, name).copy_(tensors[name])
        self.step_no = int(meta["step"])
        self.lr = float(meta["lr"])

    # ---------------------------------------------------------------- features
    def features(self, batch, sources, target, neutral, out=None):
        """feats [n, 256, 32] for the batch's processor nodes (sorted by head): the log-mel
        of the node's input under ``neutral`` parameters, and the cross-spectral band gain
        of that input against the target mix of the node's graph (grafx_ws_xgain).
        Written into ``out`` (a contiguous [n, 256, 32] view) when given."""
        torch = self.torch
        plan, L = batch.plan, batch.L
        P = (L + 3) // 4 * 4
        n = len(batch.ids)
        feats = out if out is not None else torch.empty((n, 256, 32), dtype=torch.float32, device=self.device)
        rmap = torch.tensor(batch.outrow, dtype=torch.int32, device=self.device)
        step = max(1, self.max_rows // 2)        # the cross gain keeps two frame rows per sample
        with torch.cuda.stream(self.stream):
            plan.bind_params(neutral)
            out = torch.empty(plan.info.out_elems, dtype=torch.float32, device=self.device)
            plan.render_raw(sources, out, self.st)
            for a in range(0, n, step):
                b = min(n, a + step)
                u = torch.empty((b - a, 2, P), dtype=torch.float32, device=self.device)
                plan.node_inputs_raw(sources, out, batch.ids[a:b], u, P, self.st)
                self.net.logmel_raw(u, b - a, 2 * P, P, L, None, b - a, 0, feats[a:], self.st)
                self.net.xgain_raw(u, b - a, 2 * P, target, batch.n_out_rows, 2 * P, rmap[a:b], P, L, 128,
                                   feats[a:], self.st)
        return feats

    def theta_targets(self, batch, hidden):
        """[n, 176] theta of the hidden physical parameters, rows sorted like the samples."""
        torch = self.torch
        tgt = torch.zeros((len(batch.ids), WS_OUTMAX), dtype=torch.float32, device=self.device)
        with torch.cuda.stream(self.stream):
            for t in WS_HEAD_TYPES:
                if t not in hidden:
                    continue
                p = hidden[t]
                codes = torch.tensor(gfit.param_codes(t), dtype=torch.int8, device=self.device)
                th = torch.empty_like(p)
                _check(lib().grafx_params_to_theta(_ptr(p), _ptr(codes), p.shape[1], p.numel(), _ptr(th), self.st))
                sel = [i for i, tt in enumerate(batch.types) if tt == t]
                if sel:
                    rows = torch.tensor([batch.rows[i] for i in sel], device=self.device)
                    tgt[sel[0]:sel[-1] + 1, :p.shape[1]] = th.index_select(0, rows)
        return tgt

    # ---------------------------------------------------------------- network
    def fit_standardisation(self, targets, types):
        torch = self.torch
        types = torch.as_tensor(types, device=self.device)
        for h, t in enumerate(WS_HEAD_TYPES):
            m = types == t
            if int(m.sum()) > 1:
                x = targets[m]
                self.mu[h] = x.mean(0)
                self.sd[h] = x.std(0).clamp_min(1e-3)

    def _standardise(self, x, heads, n_out, back):
        """(x - mu) / sd (back = False) or mu + sd x (back = True) per row's head, columns
        past the head's width 0, in the library's kernel (grafx_ws_standardise)."""
        y = self.torch.empty_like(x)
        _check(lib().grafx_ws_standardise(_ptr(x), _ptr(heads), _ptr(n_out), _ptr(self.mu), _ptr(self.sd),
                                          x.shape[0], x.shape[1], int(back), _ptr(y), self.st))
        return y

    def _head_rows(self, types):
        """Per sample its head and output count on the device (one upload), and the host
        counts per head; types is a sequence or array of processor types."""
        h = _HEAD_LUT[np.asarray(types, dtype=np.int64)]
        both = self.torch.from_numpy(np.stack([h, _HEAD_NOUT[h]])).to(self.device)
        return both[0], both[1], np.bincount(h, minlength=len(WS_HEAD_TYPES)).tolist()

    def train_step(self, feats, targets, types):
        """One Adam step on a minibatch (feats [B,256,32], targets theta [B,176], types
        sorted by head).  Returns the device loss tensor."""
        torch = self.torch
        B = feats.shape[0]
        heads, n_out, hc = self._head_rows(types)
        with torch.cuda.stream(self.stream):
            y = self._standardise(targets.contiguous(), heads, n_out, back=False)
            out = torch.empty((B, WS_OUTMAX), dtype=torch.float32, device=self.device)
            d = torch.empty_like(out)
            loss = torch.empty(1, dtype=torch.float32, device=self.device)
            self.net.forward_raw(self.W, feats, hc, out, self.st)
            WarmStartNet.mse_raw(out, y, n_out, loss, d, self.st)
            self.net.backward_raw(self.W, feats, hc, d, self.dW, self.st)
            self.step_no += 1
            _check(lib().grafx_adam_step(_ptr(self.W), _ptr(self.m), _ptr(self.v), _ptr(self.dW), _ptr(self.W),
                                         _ptr(self.code), 1, self.W.numel(), self.step_no, float(self.lr), 0.9,
                                         0.999, 1e-8, self.st))
        return loss

    def predict(self, feats, types):
        """theta [n, 176] (un-standardised) for samples sorted by head."""
        torch = self.torch
        heads, n_out, _ = self._head_rows(types)
        outs = []
        with torch.cuda.stream(self.stream):
            for a in range(0, feats.shape[0], self.max_batch):
                b = min(feats.shape[0], a + self.max_batch)
                hcs = np.bincount(_HEAD_LUT[np.asarray(types[a:b], dtype=np.int64)],
                                  minlength=len(WS_HEAD_TYPES)).tolist()
                out = torch.empty((b - a, WS_OUTMAX), dtype=torch.float32, device=self.device)
                self.net.forward_raw(self.W, feats[a:b], hcs, out, self.st)
                outs.append(out)
            out = torch.cat(outs)
            theta = self._standardise(out, heads, n_out, back=True)
        return theta

    def theta_tables(self, batch, theta):
        """Scatter per-sample theta back into per-type [rows, cols] tables of the plan."""
        torch = self.torch
        tabs = {}
        with torch.cuda.stream(self.stream):
            for t in WS_HEAD_TYPES:
                rows = batch.plan.info.n_type_rows[t]
                if not rows:
                    continue
                sel = [i for i, tt in enumerate(batch.types) if tt == t]
                tab = torch.zeros((rows, PARAM_COLS[t]), dtype=torch.float32, device=self.device)
                idx = torch.tensor([batch.rows[i] for i in sel], device=self.device)
                tab.index_copy_(0, idx, theta[sel[0]:sel[-1] + 1, :PARAM_COLS[t]])
                tabs[t] = tab
        return tabs


# -------------------------------------------------------------------- synthetic data
def random_graph_lists(rng, n, lo=32, hi=200, kinds=(T_GAIN, T_EQ, T_COMP, T_IMAGER, T_DELAY)):
    import synth
    out = []
    for _ in range(n):
        g = synth.random_console(rng, budget_lo=lo, budget_hi=hi, kinds=kinds)
        out.append((list(g.types), list(g.edges)))
    return out


def _sources_task(a):
    """Pool worker: one graph's seeded source tracks, flat float32."""
    import synth
    seed, K, L, P = a
    return synth.sources(seed, K, L, pitch=P).reshape(-1)


def make_batch(ws, graph_lists, L, seed, hidden_seed, pool=None):
    """Plan, sources, hidden parameters, target mix and neutral parameters of a batch
    (sources drawn by ``pool``, a multiprocessing pool, when given)."""
    import synth
    torch = ws.torch
    batch = GraphBatch(graph_lists, L)
    plan = batch.plan
    plan.bind_workspace(ws.device)
    P = (L + 3) // 4 * 4
    tasks = [(seed + k, sum(1 for t in tys if t == T_IN), L, P) for k, (tys, _) in enumerate(graph_lists)]
    src = np.concatenate(pool.map(_sources_task, tasks) if pool is not None else [_sources_task(a) for a in tasks])
    src = torch.tensor(src, device=ws.device)
    hidden = {}
    for k, (tys, eds) in enumerate(graph_lists):
        g = synth.Graph(list(tys), list(eds))
        for t, a in synth.random_params(g, hidden_seed + k).items():
            hidden.setdefault(t, []).append(a)
    hidden = {t: torch.tensor(np.concatenate(v), device=ws.device).contiguous() for t, v in hidden.items()}
    target = torch.empty(plan.info.out_elems, dtype=torch.float32, device=ws.device)
    with torch.cuda.stream(ws.stream):
        plan.bind_params(hidden)
        plan.render_raw(src, target, ws.st)
    neutral = gfit.neutral_params(plan, torch, ws.device)
    ws.stream.synchronize()
    return batch, src, hidden, target, neutral


def train(ws, n_graphs, L, graphs_per_batch=16, epochs=4, minibatch=512, seed=5, log=None, lo=32, hi=200, pool=None,
          hold_frac=0.1):
    """Generate n_graphs random consoles, build their features and theta targets, fit the
    standardisation and train.  The last hold_frac of the graphs are held out (their
    samples are not trained on) for the per-head evaluation in ``ws.held_out``.  Returns
    (losses per step, data seconds, train seconds, training samples)."""
    torch = ws.torch
    rng = np.random.Generator(np.random.PCG64(seed))
    gls = random_graph_lists(rng, n_graphs, lo, hi)
    per_graph = [sum(1 for t in tys if t in HEAD_OF) for tys, _ in gls]
    n_all = sum(per_graph)
    feats = torch.empty((n_all, 256, 32), dtype=torch.float32, device=ws.device)
    targets = torch.empty((n_all, WS_OUTMAX), dtype=torch.float32, device=ws.device)
    types = []
    t0 = time.time()
    off = 0
    for b0 in range(0, n_graphs, graphs_per_batch):
        gl = gls[b0:b0 + graphs_per_batch]
        batch, src, hidden, target, neutral = make_batch(ws, gl, L, seed * 100000 + b0 * 37, seed * 7919 + b0, pool)
        n = len(batch.ids)
        # samples of one batch are sorted by head; kept in that order (graph order is lost
        # within a batch but not across batches)
        ws.features(batch, src, target, neutral, out=feats[off:off + n])
        targets[off:off + n] = ws.theta_targets(batch, hidden)
        types += batch.types
        off += n
        ws.stream.synchronize()
        del batch, src, hidden, target, neutral
    assert off == n_all
    t_data = time.time() - t0
    # held out: the samples of the last graphs (whole batches, so whole graphs)
    n_hold_graphs = int(n_graphs * hold_frac)
    first_hold_batch = ((n_graphs - n_hold_graphs) // graphs_per_batch) * graphs_per_batch
    n_train = sum(per_graph[:first_hold_batch])
    types_all = torch.as_tensor(types, device=ws.device)
    hold_set = (feats[n_train:], targets[n_train:], types_all[n_train:])
    feats, targets = feats[:n_train], targets[:n_train]
    types = types[:n_train]
    ws.fit_standardisation(targets, types)
    head_of = torch.as_tensor([HEAD_OF.get(t, 0) for t in range(9)], device=ws.device)
    # minibatch order and head sort on the host (no device round trip per step)
    types_np = np.asarray(types, dtype=np.int64)
    head_np = np.maximum(_HEAD_LUT[types_np], 0).astype(np.int64)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = feats.shape[0]
    losses = []
    t1 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).numpy()
        for a in range(0, n - minibatch + 1, minibatch):
            idx = perm[a:a + minibatch]
            idx = idx[np.argsort(head_np[idx] * n + idx)]
            idx_d = torch.from_numpy(idx).to(ws.device)
            loss = ws.train_step(feats.index_select(0, idx_d), targets.index_select(0, idx_d), types_np[idx])
            losses.append(loss)
        if log:
            ws.stream.synchronize()
            log(f"epoch {ep}: loss {float(torch.stack(losses[-10:]).mean()):.4f}")
    ws.stream.synchronize()
    t_train = time.time() - t1
    ws.held_out = evaluate_heads(ws, *hold_set, head_of) if hold_set[0].shape[0] else {}
    return [float(x) for x in torch.cat(losses).cpu()], t_data, t_train, n


def evaluate_heads(ws, feats, targets, types_t, head_of):
    """Per head: mean over held-out samples of the standardised squared error averaged
    over the head's outputs (1.0 = predicting the training mean), and the sample count."""
    torch = ws.torch
    order = torch.argsort(head_of[types_t] * feats.shape[0] + torch.arange(feats.shape[0], device=ws.device))
    feats, targets, types_t = feats.index_select(0, order), targets.index_select(0, order), types_t[order]
    tl = types_t.tolist()
    theta = ws.predict(feats, tl)
    heads = head_of[types_t]
    err = ((theta - targets) / ws.sd[heads]) ** 2
    out = {}
    for h, t in enumerate(WS_HEAD_TYPES):
        m = types_t == t
        if int(m.sum()):
            k = WS_HEAD_OUT[h]
            out["gsecdr"[h]] = (float(err[m][:, :k].mean()), int(m.sum()))
    return out


def evaluate(ws, graph_lists, L, seed, plain_steps=1000, warm_steps=200, lr=1e-2, pool=None):
    """Per test graph: loss curve of plain Adam from neutral and of Adam from the
    predicted start; wall times (CUDA events) of the inference and of the steps."""
    torch = ws.torch
    res = []
    for k, gl in enumerate(graph_lists):
        batch, src, hidden, target, neutral = make_batch(ws, [gl], L, seed + 1000 * k, seed + 7 * k + 1, pool)
        # plain fit from neutral (its own stream; the captured step needs one)
        P0 = {t: p.clone() for t, p in neutral.items()}
        f = gfit.Fit(batch.plan, src, target, P0, lr=lr)
        hist = torch.zeros(plain_steps, device=ws.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f.stream.wait_stream(ws.stream)
        with torch.cuda.stream(f.stream):
            e0.record(f.stream)
            for i in range(plain_steps):
                f.step()
                hist[i:i + 1].copy_(f.loss)
            e1.record(f.stream)
        f.stream.synchronize()
        plain = hist.cpu().numpy()
        t_plain = e0.elapsed_time(e1) / 1e3
        # warm start: neutral render, node inputs, features and network, then Adam
        e2, e3, e4, e5 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e2.record(ws.stream)
        feats = ws.features(batch, src, target, neutral)
        theta = ws.predict(feats, batch.types)
        th0 = ws.theta_tables(batch, theta)
        e3.record(ws.stream)
        P1 = {t: p.clone() for t, p in neutral.items()}
        f2 = gfit.Fit(batch.plan, src, target, P1, lr=lr, theta0=th0)
        hist2 = torch.zeros(warm_steps, device=ws.device)
        f2.stream.wait_stream(ws.stream)
        with torch.cuda.stream(f2.stream):
            e5.record(f2.stream)
            for i in range(warm_steps):
                f2.step()
                hist2[i:i + 1].copy_(f2.loss)
            e4.record(f2.stream)
        f2.stream.synchronize()
        ws.stream.synchronize()
        warm = hist2.cpu().numpy()
        t_inf = e2.elapsed_time(e3) / 1e3
        t_warm_steps = e5.elapsed_time(e4) / 1e3
        final = float(plain[-1])
        reach = np.nonzero(warm <= final)[0]
        step_time = t_warm_steps / warm_steps
        t_reach = t_inf + (int(reach[0]) + 1) * step_time if reach.size else None
        res.append(dict(nodes=len(gl[0]), plain_final=final, plain_first=float(plain[0]), warm_first=float(warm[0]),
                        warm_final=float(warm[-1]), warm_best=float(warm.min()), t_plain=t_plain, t_inference=t_inf,
                        t_warm_steps=t_warm_steps, steps_to_plain_final=int(reach[0]) + 1 if reach.size else None,
                        t_warm_to_plain_final=t_reach,
                        speedup=(t_plain / t_reach) if t_reach else None))
        del f, f2, batch
    return res


def train_bench(steps, minibatch=512, warmup=5):
    """Time training steps (forward, MSE, backward, Adam) on random log-mel-like features
    of one minibatch; prints one JSON line (ms per step, TFLOP/s of the products)."""
    import torch
    ws = WarmStart(max_batch=max(minibatch, 2048), max_rows=64, max_len=2 ** 16)
    g = torch.Generator(device="cpu").manual_seed(1)
    feats = (-6.0 + 3.0 * torch.randn(minibatch, 256, 32, generator=g)).to(ws.device).contiguous()
    types = sorted((WS_HEAD_TYPES[i] for i in torch.randint(0, 5, (minibatch,), generator=g).tolist()),
                   key=lambda t: HEAD_OF[t])
    tgt = torch.randn(minibatch, WS_OUTMAX, generator=g).to(ws.device)
    for _ in range(warmup):
        ws.train_step(feats, tgt, types)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ws.stream)
    for _ in range(steps):
        loss = ws.train_step(feats, tgt, types)
    e1.record(ws.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rows = minibatch * 32
    conv = sum(2 * rows * k * 128 for k in (1280, 640, 640, 640))
    flops = conv + 2 * conv - 2 * rows * 1280 * 128          # forward, weight grads, input grads (l > 0)
    heads = 2 * minibatch * (128 * 288 + 288 * 288 + 288 * 60) * 3
    print(json.dumps(dict(minibatch=minibatch, steps=steps, ms_per_step=ms, loss=float(loss),
                          gemm_tflops=(flops + heads) / ms / 1e9, gpu=torch.cuda.get_device_name())))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-graphs", type=int, default=256)
    ap.add_argument("--test-graphs", type=int, default=4)
    ap.add_argument("--length", type=int, default=2 ** 16)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--minibatch", type=int, default=512)
    ap.add_argument("--plain-steps", type=int, default=1000)
    ap.add_argument("--warm-steps", type=int, default=200)
    ap.add_argument("--budget-lo", type=int, default=32)
    ap.add_argument("--budget-hi", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--graphs-per-batch", type=int, default=16)
    ap.add_argument("--workers", type=int, default=0, help="source-generating processes (default: host cores)")
    ap.add_argument("--out", default=None, help="also write the JSON record to this file")
    ap.add_argument("--train-bench", type=int, default=0,
                    help="only time this many training steps on random features (no data, no fit)")
    args = ap.parse_args()
    import multiprocessing as mp
    import os
    import torch
    if args.train_bench:
        return train_bench(args.train_bench, args.minibatch)
    workers = args.workers or min(len(os.sched_getaffinity(0)), 32)
    pool = mp.get_context("spawn").Pool(workers) if workers > 1 else None
    ws = WarmStart(max_batch=max(2048, args.minibatch), max_rows=1024, max_len=args.length, lr=args.lr)
    losses, t_data, t_train, n = train(ws, args.train_graphs, args.length, graphs_per_batch=args.graphs_per_batch,
                                       epochs=args.epochs, minibatch=args.minibatch,
                                       log=lambda s: print(s, flush=True), lo=args.budget_lo, hi=args.budget_hi,
                                       pool=pool)
    rng = np.random.Generator(np.random.PCG64(555))
    tests = random_graph_lists(rng, args.test_graphs, args.budget_lo, args.budget_hi)
    res = evaluate(ws, tests, args.length, 9000, args.plain_steps, args.warm_steps, pool=pool)
    if pool is not None:
        pool.close()
    sp = [r["speedup"] for r in res if r["speedup"]]
    # over every test graph, a graph whose warm fit never reaches the plain final loss
    # within the warm steps counting as no speedup (0)
    sp_all = [r["speedup"] or 0.0 for r in res]
    rec = dict(train_graphs=args.train_graphs, train_samples=n, length=args.length, test_graphs=len(res),
               plain_steps=args.plain_steps, warm_steps=args.warm_steps, data_s=round(t_data, 2),
               train_s=round(t_train, 2), train_steps=len(losses), loss_first=losses[0],
               loss_last=float(np.mean(losses[-20:])), held_out_mse_per_head=ws.held_out,
               median_speedup_reached=float(np.median(sp)) if sp else None,
               median_speedup_all=float(np.median(sp_all)) if sp_all else None,
               reached=len(sp), tests=res, gpu=torch.cuda.get_device_name())
    print(json.dumps(rec))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
