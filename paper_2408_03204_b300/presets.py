"""Throughput of the paper's processor settings (Sec. 3) next to the compact ones: render +
backprop through the C-ABI, timed with CUDA events on the plan's stream.

Cases (2^17 stereo samples unless --length):
  * console: the nested 64-track console (chains g-e-c-s-g), EQ of 1023 taps by 8 bands
    (compact) or of 2047 taps by its 1024 log-magnitudes (paper);
  * delay bank: 64 independent i -> d -> o chains, 4 taps anywhere in 32768 samples
    (compact) or 20 taps per channel in 100 ms slots (paper);
  * reverb bank: 64 independent i -> r -> o chains, STFT 1024/256 with 12 bands and
    dry/wet (compact) or 384/192 with 192 log-magnitudes per filter, wet only (paper);
  * multi-port nodes: a mid/side console (64 tracks split -> gain on mid and on side ->
    merge, mixed) and a bank of 64 sidechain compressors keyed by a second source;
  * 64 compressors with attack/release ballistics next to 64 single-coefficient ones.

    python -m paper_2408_03204_b300.presets --reps 10
"""
import argparse
import json

import numpy as np

from . import Graph, Plan, _stream


def bank(t, n=64):
    """n independent chains input -> t -> output."""
    import synth
    g = synth.Graph()
    for _ in range(n):
        i = g.add(synth.I)
        v = g.add(t)
        o = g.add(synth.O)
        g.connect(i, v)
        g.connect(v, o)
    return g


def mid_side_console(n=64):
    """n tracks i -> split -> (mid: gain, side: gain) -> merge, all merged into one output."""
    import synth
    g = synth.Graph()
    mix = None
    outs = []
    for _ in range(n):
        i = g.add(synth.I)
        sp = g.add(synth.P)
        gm, gs = g.add(synth.G), g.add(synth.G)
        mg = g.add(synth.J)
        g.connect(i, sp)
        g.connect(sp, gm, 0, 0)
        g.connect(sp, gs, 1, 0)
        g.connect(gm, mg, 0, 0)
        g.connect(gs, mg, 0, 1)
        outs.append(mg)
    mix = g.add(synth.M)
    for v in outs:
        g.connect(v, mix)
    o = g.add(synth.O)
    g.connect(mix, o)
    return g


def sidechain_bank(n=64):
    """n chains main input -> sidechain compressor -> output, keyed by their own second input."""
    import synth
    g = synth.Graph()
    for _ in range(n):
        i, key = g.add(synth.I), g.add(synth.I)
        k = g.add(synth.K)
        o = g.add(synth.O)
        g.connect(i, k, 0, 0)
        g.connect(key, k, 0, 1)
        g.connect(k, o)
    return g


def time_case(g, L, preset, reps, torch):
    """(ms per render + backprop, processed node-samples per step, workspace GB)."""
    import synth
    plan = Plan([Graph.from_lists(g.types, g.edges, g.ports)], [L], preset=preset)
    plan.bind_workspace("cuda")
    P = {t: torch.tensor(v, device="cuda").contiguous() for t, v in synth.random_params(g, 7, preset=preset).items()}
    plan.bind_params(P)
    if g.count(synth.R):
        noise = torch.tensor(synth.reverb_noise(), device="cuda").contiguous()
        plan.bind_reverb_noise(noise)
    Pp = (L + 3) // 4 * 4
    src = torch.tensor(synth.sources(3, g.count(synth.I), L, pitch=Pp).reshape(-1), device="cuda")
    out = torch.empty(plan.info.out_elems, device="cuda")
    d_out = torch.randn(plan.info.out_elems, device="cuda")
    dP = {t: torch.empty_like(p) for t, p in P.items()}
    st = _stream(torch, out.device)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        plan.render_raw(src, out, st)
        plan.backprop_raw(src, d_out, dP, None, st)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        plan.render_raw(src, out, st)
        plan.backprop_raw(src, d_out, dP, None, st)
    b.record(stream)
    torch.cuda.synchronize()
    plan.sync_status(st)
    return a.elapsed_time(b) / reps, int(plan.info.node_samples), plan.info.ws_bytes / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--length", type=int, default=2 ** 17)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--case", choices=["console", "delay", "reverb", "mid", "sidechain", "ballistic", "compressor"],
                    default=None,
                    help="one case only")
    ap.add_argument("--preset", choices=["compact", "paper"], default=None, help="one preset only")
    args = ap.parse_args()
    import torch
    import synth
    cases = {"console": synth.console_cfg2(), "delay bank": bank(synth.D), "reverb bank": bank(synth.R),
             "mid/side console": mid_side_console(), "sidechain bank": sidechain_bank(),
             "ballistic bank": bank(synth.A), "compressor bank": bank(synth.C)}
    rows = []
    for name, g in cases.items():
        if args.case and not name.startswith(args.case):
            continue
        for preset in ("compact", "paper"):
            if args.preset and preset != args.preset:
                continue
            if name in ("mid/side console", "sidechain bank", "ballistic bank", "compressor bank") and preset == "paper":
                continue   # no processor with a paper layout in these graphs
            ms, ns, ws = time_case(g, args.length, preset, args.reps, torch)
            rows.append({"case": name, "preset": preset, "ms_fwd_bwd": ms, "node_samples_per_s": ns / (ms / 1e3),
                         "workspace_gb": ws})
    print(json.dumps({"length": args.length, "reps": args.reps, "gpu": torch.cuda.get_device_name(), "rows": rows}))


if __name__ == "__main__":
    main()
