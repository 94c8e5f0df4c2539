#!/usr/bin/env python
"""Forward+backward render throughput of a nested 64-track mixing console.

Workload (one "step" = one pass of the whole hot path over one synthetic batch):
64 stereo tracks i -> g -> e(1023 taps) -> c -> s -> g, nested into 4 subgroup
levels of mix nodes with fan-in U{2..8}, one master output; 2^17 samples at
44.1 kHz; render, multi-resolution STFT loss (512/1024/2048, hop 1/4) against a
target rendered from hidden parameters, the loss gradient, and the backward pass
through every processor to every parameter.  Metric: processed node-samples per
second (non-input nodes x samples, forward+backward).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun every rank renders its own replica
(the single-graph path does not shard; graphs are independent units), the
barrier + max-over-ranks time gives the whole-job rate.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_FULL = 2 ** 17
EQ_TAPS = 1023
METRIC = "fwd+bwd graph-render node-samples/s"
UNIT = "node-samples/s"
CONFIG = {"workload": "nested 64-track console, chain g-e(1023)-c-s-g, 4 subgroup levels, "
                      "2^17 stereo samples, fwd+bwd with multi-resolution STFT loss",
          "tracks": 64, "subgroup_levels": 4, "samples": L_FULL, "eq_taps": EQ_TAPS,
          "sample_rate": 44100, "schedule": "beam-32",
          "l2": "working set (U + adjoint rows, ~850 MB) larger than L2; no flush"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--samples", type=int, default=L_FULL, help="signal length (smaller only for profiling captures)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the plan's default tiles (keeps the launch list short for profiling captures)")
    return ap.parse_args()


def workload():
    import synth
    g = synth.console_cfg2()
    return g


def algorithmic_bytes(g, string, steps_nodes, L):
    """Per schedule step: forward bytes 8*(indeg+1) per node-sample; backward bytes
    8*outdeg (consumer adjoints) + 8*indeg (re-gathered input, only for processors
    whose adjoint needs it) + 8 (input-adjoint write).  Output nodes alias dL/dY."""
    n = g.n_nodes
    indeg = [0] * n
    outdeg = [0] * n
    for s, d in g.edges:
        indeg[d] += 1
        outdeg[s] += 1
    fwd, bwd = {}, {}
    for k in range(1, len(string)):
        t = string[k]
        fb = bb = 0
        for v in steps_nodes[k]:
            fb += 8 * (indeg[v] + 1) * L
            if t == 1:  # output: its adjoint row is d_out itself
                continue
            needs_u = t not in (1, 2)
            bb += (8 * outdeg[v] + (8 * indeg[v] if needs_u else 0) + 8) * L
        fwd[k], bwd[k] = fb, bb
    return fwd, bwd


class _Nvml:
    """The three NVML queries the sampler needs, through ctypes on libnvidia-ml."""

    def __init__(self, index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")

    def _clock(self, fn):
        v = self.ct.c_uint()
        if fn(self.h, self.ct.c_int(1), self.ct.byref(v)) != 0:  # NVML_CLOCK_SM = 1
            raise RuntimeError("clock query failed")
        return v.value

    def sm(self):
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def max_sm(self):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self):
        v = self.ct.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(self.h, self.ct.byref(v)) != 0:
            raise RuntimeError("reasons query failed")
        return v.value


class ClockSampler:
    """SM clock and throttle reasons sampled through NVML every ~2 ms in a thread
    (the timed region can be far shorter than nvidia-smi's sampling period)."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, index):
        import threading
        self.sm, self.reasons, self.smax, self.err = [], set(), None, None
        self.on = False
        try:
            self.nv = _Nvml(index)
            self.smax = float(self.nv.max_sm())
        except Exception as e:  # no NVML: report it
            self.nv, self.err = None, str(e)
        self.stop_flag = False
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()

    def _run(self):
        while not self.stop_flag and self.nv is not None:
            if self.on:
                try:
                    self.sm.append(float(self.nv.sm()))
                    r = self.nv.reasons()
                    for nm, bit in self.REASONS.items():
                        if r & bit:
                            self.reasons.add(nm)
                except Exception as e:
                    self.err = str(e)
            time.sleep(0.002)

    def start(self):
        self.on = True

    def stop(self):
        self.on = False
        self.stop_flag = True
        self.t.join(timeout=5)
        if self.nv is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": f"NVML unavailable: {self.err}"}
        sm = sorted(self.sm)
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": self.smax, "reasons": sorted(self.reasons), "samples": len(sm),
                "source": "NVML during the timed region"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def traffic_for(kernel_key):
    """ncu DRAM bytes per launch recorded in profiles/dram_traffic.json, if the kernel's
    sources (its .cu file and the headers it includes) have not changed since (sha1)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel_key)
    if not d:
        return None
    if "sources" not in d:
        return None
    return d["bytes_per_launch"] if sources_sha1(d["sources"]) == d["sha1"] else None


def sources_sha1(names):
    h = hashlib.sha1()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2408_03204_b300", "csrc", n), "rb").read())
    return h.hexdigest()


def cpu_baseline(L=L_FULL, steps=1):
    """The FP64 oracle as it stands: one fwd+bwd step (render, loss, loss gradient,
    backward) of the same console at full length, on this host."""
    import numpy as np
    import synth
    from oracle import render as orr, loss as ol
    g = workload()
    src = synth.sources(2, g.count(synth.I), L)
    P = synth.random_params(g, 2)
    Ph = synth.random_params(g, 102)
    hp = dict(eq_taps=EQ_TAPS)
    tgt = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, Ph, hp))
    t0 = time.time()
    for _ in range(steps):
        Y = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P, hp))
        ol.mrstft(Y, tgt)
        dY = ol.mrstft_grad(Y, tgt)
        orr.backward(g.types, g.edges, src, P, dY, hp)
    dt = time.time() - t0
    ns = sum(1 for t in g.types if t != synth.I) * L * steps
    return {"value": ns / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} fwd+bwd step(s) of the same console at {L} samples "
                      f"({dt:.1f} s; numpy/scipy FP64, single-threaded)"}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the whole job ends with it (no-op on one rank)."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank_step, world, steps, ms_total):
    """Whole-job throughput: every rank processes its own replica's units each step."""
    return units_per_rank_step * world * steps / (ms_total / 1e3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    L = 2 ** 13
    cpu_baseline(L=2 ** 11, steps=1)                 # untimed warm-up (imports, caches)
    cb = cpu_baseline(L=L, steps=max(1, args.steps))
    val = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, sample_samples=L),
            "cpu_baseline": dict(cb, value=val),
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import synth
    from paper_2408_03204_b300 import build
    build.build()
    import paper_2408_03204_b300 as gx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    g = workload()
    L = args.samples
    graphs = [gx.Graph.from_lists(g.types, g.edges)]
    tiles = {}
    if not args.no_autotune:
        # tile sizes timed on this GPU for this graph (outside the timed region)
        from paper_2408_03204_b300 import autotune as gat
        tiles = gat.autotune(graphs, [L], eq_taps=EQ_TAPS, cache=None, device=str(dev))
    plan = gx.Plan(graphs, [L], eq_taps=EQ_TAPS, **tiles)
    plan.bind_workspace(dev)
    info = plan.info
    exp = plan.export()
    string = exp["type_string"]
    sp = exp["step_ptr"]
    inv = [0] * g.n_nodes
    for v, nv in enumerate(exp["sigma"]):
        inv[nv] = v
    steps_nodes = [[inv[x] for x in range(sp[k], sp[k + 1])] for k in range(len(string))]
    fwd_b, bwd_b = algorithmic_bytes(g, string, steps_nodes, L)

    src_h = synth.sources(2 + rank, g.count(synth.I), L).reshape(-1)
    P_h = synth.random_params(g, 2)
    Ph_h = synth.random_params(g, 102)
    src = torch.tensor(src_h, device=dev)
    P = {t: torch.tensor(v, device=dev) for t, v in P_h.items()}
    Ph = {t: torch.tensor(v, device=dev) for t, v in Ph_h.items()}
    stream = torch.cuda.current_stream(dev)
    st = gx._stream(torch, dev)
    out = torch.empty(info.out_elems, device=dev)
    tgt = torch.empty_like(out)
    plan.bind_params(Ph)
    plan.render_raw(src, tgt, st)            # target from hidden parameters (input generation)
    plan.bind_params(P)
    loss = torch.empty(1, device=dev)
    d_out = torch.empty_like(out)
    dP = {t: torch.empty_like(p) for t, p in P.items()}
    N = len(string) - 1

    def step(evs=None):
        i = 0
        for k in range(1, N + 1):
            plan.render_steps_raw(src, out, k, k + 1, st)
            if evs is not None:
                evs[i].record(stream); i += 1
        plan.loss_raw(out, tgt, loss, st)
        plan.loss_backward_raw(out, tgt, d_out, st)
        if evs is not None:
            evs[i].record(stream); i += 1
        for k in range(N, 0, -1):
            plan.backprop_steps_raw(src, d_out, dP, None, k, k + 1, st)
            if evs is not None:
                evs[i].record(stream); i += 1

    def launches_per_step():
        n = 0
        for k in range(1, N + 1):
            plan.render_steps_raw(src, out, k, k + 1, st)
            n += plan.last_launches()
        plan.loss_raw(out, tgt, loss, st)
        n += plan.last_launches()
        plan.loss_backward_raw(out, tgt, d_out, st)
        n += plan.last_launches()
        for k in range(N, 0, -1):
            plan.backprop_steps_raw(src, d_out, dP, None, k, k + 1, st)
            n += plan.last_launches()
        return n

    n_launch = launches_per_step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    plan.sync_status(st)

    # ---- the timed region: the whole step (render, loss, loss gradient, backprop) as
    # the library's captured CUDA graph (grafx_step_graph_*), replayed on a side stream
    side = torch.cuda.Stream(dev)
    ss = gx._stream_of(side)
    torch.cuda.synchronize(dev)
    graph = plan.capture_step(src, out, tgt, loss, d_out, dP, None, ss)
    for _ in range(max(3, args.warmup)):
        graph.launch(ss)
    torch.cuda.synchronize(dev)
    plan.sync_status(ss)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    t_start.record(side)
    for _ in range(args.steps):
        graph.launch(ss)
    t_end.record(side)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    plan.sync_status(ss)
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
    ms_step = ms_total / args.steps
    node_samples = int(info.node_samples)
    value = job_rate(node_samples, world, args.steps, ms_total)

    # ---- diagnostics outside the timed region: per schedule-step durations of the same
    # step launched step by step (fwd k = 1..N, loss, bwd k = N..1)
    n_ev = N + 1 + N
    diag = max(5, args.steps // 2)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(diag)]
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(diag)]
    torch.cuda.synchronize(dev)
    for it in range(diag):
        e0[it].record(stream)
        step(evs[it])
    torch.cuda.synchronize(dev)
    labels = [f"fwd:{synth.TYPE_LETTERS[string[k]]}{k}" for k in range(1, N + 1)] + ["loss"] + \
             [f"bwd:{synth.TYPE_LETTERS[string[k]]}{k}" for k in range(N, 0, -1)]
    dur = np.zeros(n_ev)
    for it in range(diag):
        prev = e0[it]
        for j in range(n_ev):
            dur[j] += prev.elapsed_time(evs[it][j])
            prev = evs[it][j]
    dur /= diag
    algo = [fwd_b[k] for k in range(1, N + 1)] + [0] + [bwd_b[k] for k in range(N, 0, -1)]
    j = int(np.argmax(dur))
    kernel_key = labels[j]
    # the dominant step alone, launched back to back on its stream (its kernels only)
    k_step = (N - (j - N - 1)) if j > N else (j + 1)
    reps = 20
    ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ka.record(stream)
    for _ in range(reps):
        if j > N:
            plan.backprop_steps_raw(src, d_out, dP, None, k_step, k_step + 1, st)
        elif j == N:
            plan.loss_raw(out, tgt, loss, st)
            plan.loss_backward_raw(out, tgt, d_out, st)
        else:
            plan.render_steps_raw(src, out, k_step, k_step + 1, st)
    kb.record(stream)
    torch.cuda.synchronize(dev)
    ms_kernel = ka.elapsed_time(kb) / reps
    peak, peak_kind = peaks()
    achieved = algo[j] / (ms_kernel / 1e3) / 1e9
    step_bytes = sum(algo)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_for(kernel_key), "kernel": kernel_key,
                "peak_source": peak_kind, "ms_per_launch": ms_kernel,
                "algorithmic_bytes_per_launch": algo[j],
                "step": {"algorithmic_bytes": step_bytes, "achieved": step_bytes / (ms_step / 1e3) / 1e9,
                         "frac": step_bytes / (ms_step / 1e3) / 1e9 / peak},
                "eager_breakdown_ms": {lab: round(float(d), 4) for lab, d in zip(labels, dur)},
                "eager_ms_per_step": float(dur.sum())}
    plan.sync_status(st)

    # end to end through the C-ABI with host buffers: H2D of the step's inputs from pinned
    # memory, the captured step, D2H of the loss and every parameter gradient
    src_pin = torch.tensor(src_h).pin_memory()
    tgt_pin = tgt.cpu().pin_memory()
    P_pin = {t: v.cpu().pin_memory() for t, v in P.items()}
    loss_pin = torch.empty(1).pin_memory()
    dP_pin = {t: torch.empty(v.shape).pin_memory() for t, v in P.items()}
    h2d = src_pin.numel() * 4 + tgt_pin.numel() * 4 + sum(v.numel() * 4 for v in P_pin.values())
    d2h = 4 + sum(v.numel() * 4 for v in dP_pin.values())

    # Double-buffered: every step copies its own sources and target from pinned memory,
    # on a copy stream into the buffer the previous-but-one step read, while the step
    # before it computes; the parameters (a few KB) are copied on the compute stream just
    # before their step, and the loss and gradients come back after it.
    src2, tgt2 = torch.empty_like(src), torch.empty_like(tgt)
    graph2 = plan.capture_step(src2, out, tgt2, loss, d_out, dP, None, ss)
    bufs = [(src, tgt, graph), (src2, tgt2, graph2)]
    cstream = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        s_, t_, _ = bufs[k]
        with torch.cuda.stream(cstream):
            cstream.wait_event(ev_used[k])      # the step that last read this buffer is done
            s_.copy_(src_pin, non_blocking=True)
            t_.copy_(tgt_pin, non_blocking=True)
            ev_in[k].record(cstream)

    def e2e_steps(n):
        copy_in(0)
        for i in range(n):
            k = i % 2
            if i + 1 < n:
                copy_in((i + 1) % 2)
            with torch.cuda.stream(side):
                side.wait_event(ev_in[k])
                for t in P:
                    P[t].copy_(P_pin[t], non_blocking=True)
                bufs[k][2].launch(ss)
                ev_used[k].record(side)
                loss_pin.copy_(loss, non_blocking=True)
                for t in dP:
                    dP_pin[t].copy_(dP[t], non_blocking=True)

    e2e_steps(2)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    a.record(side)
    cstream.wait_event(a)
    e2e_steps(args.e2e_steps)
    b.record(side)
    torch.cuda.synchronize(dev)
    ms_e2e = max_over_ranks(a.elapsed_time(b), dist, dev)
    e2e = {"value": job_rate(node_samples, world, args.e2e_steps, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e / args.e2e_steps,
           "loss": float(loss_pin.item())}

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()

    if rank == 0:
        cfg = dict(CONFIG, samples=L)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(cfg, nodes=int(info.n_nodes), processed_node_samples=node_samples,
                               schedule_steps=N, parallelism=f"replicas{world}",
                               tiles={"eq_fft": int(info.eq_fft), "comp_chunk": int(info.comp_chunk),
                                      "chosen_by": "defaults" if args.no_autotune else "autotune"}),
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "clocks": clocks,
                "gpu_launches": graph.launches() * args.steps,
                "timed": "captured CUDA graph of the whole step (grafx_step_graph), "
                         f"{graph.launches()} kernels per step, {n_launch} when launched step by step"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
