"""Tile-size autotuner for a plan: times the candidate EQ block-FFT sizes and
compressor chunk sizes on the actual graph batch (render + backprop through the C-ABI,
CUDA events, median of a few runs) and keeps the fastest.  Results are cached per
(graph structure, lengths, EQ taps) in a JSON file.

Only timing happens here; every candidate runs the library's own kernels.
"""
import hashlib
import json
import os

from . import T_COMP, Plan, _stream

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "grafx_autotune.json")


def _key(graph_lists, lengths, eq_taps):
    h = hashlib.sha1()
    h.update(json.dumps([graph_lists, list(lengths), eq_taps]).encode())
    return h.hexdigest()


def candidates(eq_taps):
    H = (eq_taps - 1) // 2
    ffts = [m for m in (1024, 2048, 4096, 8192) if ((m - 2 * H) & ~3) >= max(256, m // 4, 2 * H)]
    return [{"eq_fft": m, "comp_chunk": cc} for m in ffts for cc in (1024, 2048, 4096)]


def _neutral_params(plan, torch, device):
    P = {}
    for t, cols in plan.param_cols.items():
        rows = plan.info.n_type_rows[t]
        if rows:
            p = torch.zeros((rows, cols), dtype=torch.float32, device=device)
            if t == T_COMP:
                p[:, 0], p[:, 2], p[:, 3] = 0.99, 0.69, 2.0
            P[t] = p
    return P


def time_plan(plan, torch, device, reps=3):
    plan.bind_workspace(device)
    P = _neutral_params(plan, torch, device)
    plan.bind_params(P)
    src = torch.zeros(plan.info.src_elems, device=device)
    out = torch.empty(plan.info.out_elems, device=device)
    d_out = torch.ones_like(out)
    dP = {t: torch.empty_like(p) for t, p in P.items()}
    st = _stream(torch, device)
    stream = torch.cuda.current_stream(device)
    times = []
    for r in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.render_raw(src, out, st)
        plan.backprop_raw(src, d_out, dP, None, st)
        b.record(stream)
        torch.cuda.synchronize(device)
        if r:
            times.append(a.elapsed_time(b))
    plan.sync_status(st)
    return sorted(times)[len(times) // 2]


def autotune(graphs, lengths, graph_lists=None, eq_taps=1023, cache=DEFAULT_CACHE, device="cuda", **plan_kw):
    """Best {eq_fft, comp_chunk} for this batch; ``graphs`` are library Graphs,
    ``graph_lists`` their (types, edges) for the cache key."""
    import torch
    key = _key(graph_lists, lengths, eq_taps) if graph_lists is not None else None
    store = {}
    if key and cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
        if key in store:
            return store[key]["best"]
    results = []
    for cand in candidates(eq_taps):
        plan = Plan(graphs, lengths, eq_taps=eq_taps, **dict(plan_kw, **cand))
        results.append((time_plan(plan, torch, torch.device(device)), cand))
        del plan
    ms, best = min(results, key=lambda x: x[0])
    if key and cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        store[key] = {"best": best, "ms": ms, "all": [{"ms": m, **c} for m, c in results]}
        with open(cache, "w") as f:
            json.dump(store, f, indent=1)
    return best
