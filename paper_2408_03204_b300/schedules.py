"""Schedule-method comparison (the paper's Sec. 4 speed benchmark, on synthetic consoles):
for each graph, the number of schedule steps (processor calls) of one-by-one, greedy,
beam-32 and optimal (optimal only for graphs small enough for the exact search) and the
GPU time of a render and of a render + backprop under each schedule.

    python -m paper_2408_03204_b300.schedules --graphs 16 --length 131072
"""
import argparse
import json

import numpy as np

from . import Graph, Plan, _stream

METHODS = ("one_by_one", "greedy", "beam", "optimal")
OPTIMAL_MAX_PROC = 28  # processing nodes the exact search accepts


def consoles(n, seed=42):
    """Random mixing consoles (tracks with processor chains, nested subgroups): half of
    them small enough for the exact optimal search, half of 32-128 nodes."""
    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    small = [synth.random_console(rng, budget_lo=12, budget_hi=26, depth_lo=1, depth_hi=2) for _ in range(n // 2)]
    large = [synth.random_console(rng, budget_lo=32, budget_hi=128) for _ in range(n - n // 2)]
    return small + large


def time_method(g, L, method, reps, torch):
    """(steps, fwd ms, fwd+bwd ms) of graph g with a schedule method."""
    import synth
    plan = Plan([Graph.from_lists(g.types, g.edges)], [L], schedule=method)
    plan.bind_workspace("cuda")
    P = {t: torch.tensor(v, device="cuda").contiguous() for t, v in synth.random_params(g, 7).items()}
    plan.bind_params(P)
    Pp = (L + 3) // 4 * 4
    src = torch.tensor(synth.sources(3, g.count(synth.I), L, pitch=Pp).reshape(-1), device="cuda")
    out = torch.empty(plan.info.out_elems, device="cuda")
    d_out = torch.ones_like(out)
    dP = {t: torch.empty_like(p) for t, p in P.items()}
    st = _stream(torch, out.device)
    for _ in range(2):
        plan.render_raw(src, out, st)
        plan.backprop_raw(src, d_out, dP, None, st)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(reps):
        plan.render_raw(src, out, st)
    ev[1].record()
    for _ in range(reps):
        plan.render_raw(src, out, st)
        plan.backprop_raw(src, d_out, dP, None, st)
    ev[2].record()
    torch.cuda.synchronize()
    plan.sync_status(st)
    return plan.info.n_steps, ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=16)
    ap.add_argument("--length", type=int, default=2 ** 17)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=42)
    args = ap.parse_args()
    import torch
    import synth
    rows = []
    for g in consoles(args.graphs, args.seed):
        n_proc = sum(1 for t in g.types if t not in (synth.I, synth.O))
        r = {"nodes": g.n_nodes, "processing_nodes": n_proc}
        for m in METHODS:
            if m == "optimal" and n_proc > OPTIMAL_MAX_PROC:
                continue
            steps, fwd, both = time_method(g, args.length, m, args.reps, torch)
            r[m] = {"steps": steps, "fwd_ms": fwd, "fwd_bwd_ms": both}
        rows.append(r)
    summary = {}
    for m in METHODS:
        have = [r[m] for r in rows if m in r]
        if have:
            summary[m] = {"graphs": len(have), "mean_steps": float(np.mean([h["steps"] for h in have])),
                          "mean_fwd_ms": float(np.mean([h["fwd_ms"] for h in have])),
                          "mean_fwd_bwd_ms": float(np.mean([h["fwd_bwd_ms"] for h in have]))}
    print(json.dumps({"length": args.length, "graphs": len(rows), "summary": summary, "per_graph": rows,
                      "gpu": torch.cuda.get_device_name()}))


if __name__ == "__main__":
    main()
