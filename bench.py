#!/usr/bin/env python
"""Forward+backward render throughput of a batch of 128 random mixing consoles.

Workload (one "step" = one pass of the whole hot path over one synthetic batch): 128
random mixing consoles of uneven size (node budget U{16..256}, subgroup depth U{1..4},
tracks with chains of 1-5 processors drawn from gain/pan, zero-phase FIR EQ with 1023
taps, compressor, stereo imager and 4-tap multitap delay), each with its own signal
length L ~ U[2^15, 2^18] stereo samples at 44.1 kHz, rendered as one disjoint union
(Sec. 2 "Batched processing": one launch per kernel and schedule step over every
graph's nodes); the multi-resolution STFT loss (512/1024/2048, hop 1/4) of every
console's output against a target rendered from hidden parameters; the loss gradient;
and the backward pass to every parameter.  Metric: processed node-samples (non-input
nodes x samples) per second, forward+backward.  A secondary measurement times the
nested 64-track console (402 nodes, 2^17 samples).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun the batch's graphs are partitioned over
the ranks by cost (nodes x samples, `paper_2408_03204_b300.shard`); every rank plans
and renders its own graphs with no collective on the data path; the barrier +
max-over-ranks time gives the whole-job rate.
"""
import argparse
import hashlib
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EQ_TAPS = 1023
METRIC = "fwd+bwd graph-render node-samples/s"
UNIT = "node-samples/s"
SRC_SEED, PARAM_SEED, HIDDEN_SEED = 300, 3000, 9000
CONFIGS = {
    "batch128": {"workload": "128 random mixing consoles (node budget U{16..256}, subgroup depth U{1..4}, "
                             "chains of 1-5 of gain/pan, EQ(1023 taps), compressor, imager, 4-tap delay), "
                             "ragged L ~ U[2^15, 2^18] stereo samples, one disjoint-union plan, fwd+bwd with "
                             "multi-resolution STFT loss",
                 "graphs": 128, "eq_taps": EQ_TAPS, "sample_rate": 44100, "schedule": "beam-32",
                 "l2": "working set (signal and adjoint rows, ~40 GB) larger than L2; no flush"},
    "console64": {"workload": "nested 64-track console, chain g-e(1023)-c-s-g, 4 subgroup levels, "
                              "2^17 stereo samples, fwd+bwd with multi-resolution STFT loss",
                  "tracks": 64, "subgroup_levels": 4, "samples": 2 ** 17, "eq_taps": EQ_TAPS,
                  "sample_rate": 44100, "schedule": "beam-32",
                  "l2": "working set (U + adjoint rows, ~850 MB) larger than L2; no flush"},
}
# the compact multitap delay's layout (4 taps per channel, N_d = 32768 lags, lag
# partitions of B = 4096 with 8192-point spectra) for its algorithmic FLOP count
DL_TAPS, DL_FIR, DL_ND, DL_B, DL_M, DL_P = 4, 39, 32768, 4096, 8192, 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch128", choices=sorted(CONFIGS))
    ap.add_argument("--graphs", type=int, default=128,
                    help="first N graphs of the batch (fewer only for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--samples", type=int, default=2 ** 17, help="console64 signal length (profiling only)")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="graphs per oracle step (default: one per host core, at most 16)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the plan's default tiles (keeps the launch list short for profiling captures)")
    return ap.parse_args()


def workload(name, n_graphs=128, samples=2 ** 17):
    """(graphs, lengths, source seeds) of a workload."""
    import synth
    if name == "console64":
        return [synth.console_cfg2()], [samples], [2]
    graphs, lengths = synth.batch_cfg3()
    n = max(1, min(n_graphs, len(graphs)))
    return graphs[:n], lengths[:n], [SRC_SEED + k for k in range(n)]


def params_for(name, graphs, seed):
    import synth
    return synth.union_params(graphs, {"param": 2 if name == "console64" else PARAM_SEED,
                                       "hidden": 102 if name == "console64" else HIDDEN_SEED}[seed])


# ----------------------------------------------------------------------------- inputs
def _src_task(a):
    """Worker: graph k's sources into the shared buffer at its offset."""
    from multiprocessing import shared_memory
    import numpy as np
    import synth
    name, total, off, seed, K, L, pitch = a
    shm = shared_memory.SharedMemory(name=name)
    try:
        buf = np.ndarray((total,), np.float32, buffer=shm.buf)
        s = synth.sources(seed, K, L, pitch=pitch)
        buf[off:off + s.size] = s.reshape(-1)
    finally:
        shm.close()
    return 0


def sources_for(graphs, lengths, seeds, workers):
    """Flat float32 sources of the batch, graph-major [K_g][2][pitch_g], generated by a
    spawn pool of host processes (the shared seeded generator, one graph per task)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    import synth
    offs, total = [], 0
    for g, L in zip(graphs, lengths):
        offs.append(total)
        total += g.count(synth.I) * 2 * ((L + 3) // 4 * 4)
    if len(graphs) == 1 or workers <= 1:
        out = np.zeros(total, np.float32)
        for g, L, s, o in zip(graphs, lengths, seeds, offs):
            x = synth.sources(s, g.count(synth.I), L, pitch=(L + 3) // 4 * 4).reshape(-1)
            out[o:o + x.size] = x
        return out
    shm = shared_memory.SharedMemory(create=True, size=total * 4)
    try:
        tasks = [(shm.name, total, o, s, g.count(synth.I), L, (L + 3) // 4 * 4)
                 for g, L, s, o in zip(graphs, lengths, seeds, offs)]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_src_task, tasks, chunksize=1)
        return np.ndarray((total,), np.float32, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()


# ----------------------------------------------------------------------------- roofline
def graph_degrees(graphs):
    """Union node ids (graph-major, original order) -> (type, indeg, outdeg, L)."""
    nodes = []
    for g, L in graphs:
        base = len(nodes)
        indeg = [0] * g.n_nodes
        outdeg = [0] * g.n_nodes
        for s, d in g.edges:
            indeg[d] += 1
            outdeg[s] += 1
        nodes.extend((t, indeg[v], outdeg[v], L) for v, t in enumerate(g.types))
        assert len(nodes) == base + g.n_nodes
    return nodes


def delay_flops(L):
    """Algorithmic FP32 flops of one compact multitap delay node on L samples (both
    channels), forward and backward, for the FFT-partitioned algorithm of Eq. 14-15:
    the sparse FIR (T taps x 39 multiply-adds per output sample and channel) forward
    and transposed; 8192-point transforms (5 M log2 M flops each) of the u windows
    holding signal (nb + 1) and of the nb ybar blocks; the lag accumulation (P
    partitions x nb blocks x (M/2 + 1) bins x 2 channels x 8 flops); P inverse
    transforms; the surrogate z-gradient (per channel, tap and each of N_d lags: the
    39-tap correlation, 78 flops, and the closed form of phi with its product, 50)."""
    nb = (L + DL_B - 1) // DL_B
    fft = 5.0 * DL_M * math.log2(DL_M)
    fir = 2 * L * DL_TAPS * DL_FIR * 2.0
    bwd = fir + (2 * nb + 1) * fft + DL_P * nb * (DL_M // 2 + 1) * 2 * 8.0 + DL_P * fft \
        + 2 * DL_TAPS * DL_ND * (2 * DL_FIR + 50.0)
    return fir, bwd


def step_costs(nodes, string, step_nodes):
    """Per schedule step (k = 1..N): algorithmic bytes forward and backward (8 B per
    node-sample per row read or written: forward 8 (indeg + 1); backward 8 outdeg + 8
    indeg (re-gathered input, only for processors whose adjoint needs it) + 8; output
    nodes alias dL/dY) and algorithmic FP32 flops of the ALU-bound delay steps."""
    fwd_b, bwd_b, fwd_f, bwd_f = {}, {}, {}, {}
    for k in range(1, len(string)):
        t = string[k]
        fb = bb = ff = bf = 0
        for v in step_nodes[k]:
            tv, ind, outd, L = nodes[v]
            fb += 8 * (ind + 1) * L
            if t == 7:
                f, b = delay_flops(L)
                ff += f
                bf += b
            if t == 1:
                continue
            needs_u = t not in (1, 2)
            bb += (8 * outd + (8 * ind if needs_u else 0) + 8) * L
        fwd_b[k], bwd_b[k], fwd_f[k], bwd_f[k] = fb, bb, ff, bf
    return fwd_b, bwd_b, fwd_f, bwd_f


def peaks(n_sm):
    """HBM GB/s and the FP32 (non-tensor) FMA peak in TFLOP/s: n_sm x 128 FP32 lanes x
    2 flops x the maximum SM clock."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        mhz = float(d.get("sm_max_mhz", 2032.0))
        return float(d["hbm_gbs"]), "measured", n_sm * 128 * 2 * mhz * 1e6 / 1e12
    return 6400.0, "fallback", n_sm * 128 * 2 * 2032e6 / 1e12


def traffic_for(kernel_key):
    """ncu DRAM bytes per launch recorded in profiles/dram_traffic.json, if the kernel's
    sources (its .cu file and the headers it includes) have not changed since (sha1)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel_key)
    if not d or "sources" not in d:
        return None
    return d["bytes_per_launch"] if sources_sha1(d["sources"]) == d["sha1"] else None


def sources_sha1(names):
    h = hashlib.sha1()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2408_03204_b300", "csrc", n), "rb").read())
    return h.hexdigest()


# ----------------------------------------------------------------------------- clocks
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


# ----------------------------------------------------------------------------- oracle baseline
def _oracle_task(a):
    """Worker: one graph of the batch through the FP64 oracle as it stands: the target
    from the hidden parameters (untimed), then one timed fwd+bwd step (render, loss,
    loss gradient, backward).  Returns (node-samples, wall start, wall end)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    name, k, n_graphs, samples, barrier = a
    import synth
    from oracle import render as orr, loss as ol
    graphs, lengths, seeds = workload(name, n_graphs, samples)
    g, L = graphs[k], lengths[k]
    src = synth.sources(seeds[k], g.count(synth.I), L)
    P = params_for(name, graphs, "param")
    Ph = params_for(name, graphs, "hidden")
    row0 = {t: sum(h.count(t) for h in graphs[:k]) for t in P}
    Pk = {t: P[t][row0[t]:row0[t] + g.count(t)] for t in P if g.count(t)}
    Phk = {t: Ph[t][row0[t]:row0[t] + g.count(t)] for t in Ph if g.count(t)}
    hp = dict(eq_taps=EQ_TAPS)
    tgt = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, Phk, hp))
    if barrier is not None:
        barrier.wait()
    t0 = time.time()
    Y = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, Pk, hp))
    ol.mrstft(Y, tgt)
    dY = ol.mrstft_grad(Y, tgt)
    orr.backward(g.types, g.edges, src, Pk, dY, hp)
    t1 = time.time()
    return sum(1 for t in g.types if t != synth.I) * L, t0, t1


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_round(name, ks, n_graphs, samples, workers):
    """One timed oracle step over the graphs ks, one spawn process per graph, all
    started together behind a barrier: (node-samples, seconds of the round)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    if workers <= 1 or len(ks) == 1:
        res = [_oracle_task((name, k, n_graphs, samples, None)) for k in ks]
        return sum(r[0] for r in res), sum(r[2] - r[1] for r in res)
    with ctx.Manager() as man:
        bar = man.Barrier(len(ks))
        with ctx.Pool(len(ks)) as pool:
            res = pool.map(_oracle_task, [(name, k, n_graphs, samples, bar) for k in ks], chunksize=1)
    return sum(r[0] for r in res), max(r[2] for r in res) - min(r[1] for r in res)


def sample_graphs(n_graphs, per_step, step):
    """Graphs of oracle step `step`: per_step graphs spread evenly over the batch,
    shifted by one each step."""
    stride = max(1, n_graphs // per_step)
    return sorted({(step + i * stride) % n_graphs for i in range(per_step)})


def cpu_baseline(name, n_graphs, samples, per_step=0):
    """The FP64 oracle (numpy/scipy, as it stands) on this host's cores: one process per
    core, each a whole graph of the batch at full length."""
    cores = host_cores()
    per = per_step or min(cores, 16)
    if name == "console64":
        per = 1
    ks = sample_graphs(n_graphs, per, 0) if name != "console64" else [0]
    ns, dt = oracle_round(name, ks, n_graphs, samples, per)
    return {"value": ns / dt, "unit": UNIT, "cores": min(per, cores), "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{len(ks)} graph(s) of the workload at full length ({ns / 1e6:.1f} M node-samples), "
                      f"one spawn process per graph, one fwd+bwd step each, started together: {dt:.1f} s "
                      f"(numpy/scipy FP64)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name, n = args.workload, args.graphs
    cores = host_cores()
    per = 1 if name == "console64" else (args.ref_sample or min(cores, 16))
    # warm-up: imports and caches, on the smallest graph at its own length
    graphs, lengths, _ = workload(name, n, args.samples)
    small = min(range(len(graphs)), key=lambda k: graphs[k].n_nodes * lengths[k])
    oracle_round(name, [small], n, args.samples, 1)
    ns_tot = dt_tot = 0.0
    steps = 0
    t_start = time.time()
    while steps < max(1, args.steps):
        ks = sample_graphs(len(graphs), per, steps) if name != "console64" else [0]
        ns, dt = oracle_round(name, ks, n, args.samples, per)
        ns_tot += ns
        dt_tot += dt
        steps += 1
        if time.time() - t_start > 150:      # bounded: the run ends within a few minutes
            break
    val = ns_tot / dt_tot
    cb = {"value": val, "unit": UNIT, "cores": min(per, cores), "host_cores": os.cpu_count(), "kind": "oracle",
          "sample": f"{steps} step(s), each {per} graph(s) of the workload at full length, one spawn process "
                    f"per graph started together ({ns_tot / 1e6:.1f} M node-samples in {dt_tot:.1f} s; "
                    f"numpy/scipy FP64)"}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "steps_requested": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "strong" if name == "batch128" else "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(CONFIGS[name], same_config=True),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- multi-rank
def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the whole job ends with it (no-op on one rank)."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank_step, world, steps, ms_total):
    """Whole-job throughput when every rank processes the same number of units per step."""
    return units_per_rank_step * world * steps / (ms_total / 1e3)


def sum_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    tt = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tt.item())


# ----------------------------------------------------------------------------- GPU arm
def measure(gx, torch, np, graphs, lengths, src_h, P_h, Ph_h, dev, steps, warmup, autotune, dist=None,
            e2e_steps=0):
    """Plan, bind, time the captured fwd+bwd step; per-step diagnostics; optional e2e."""
    import synth
    glist = [gx.Graph.from_lists(g.types, g.edges) for g in graphs]
    tiles = {}
    if autotune:
        from paper_2408_03204_b300 import autotune as gat
        tiles = gat.autotune(glist, lengths, eq_taps=EQ_TAPS, cache=None, device=str(dev))
    plan = gx.Plan(glist, lengths, eq_taps=EQ_TAPS, **tiles)
    plan.bind_workspace(dev)
    info = plan.info
    exp = plan.export()
    string = exp["type_string"]
    sp = exp["step_ptr"]
    inv = [0] * info.n_nodes
    for v, nv in enumerate(exp["sigma"]):
        inv[nv] = v
    step_nodes = [[inv[x] for x in range(sp[k], sp[k + 1])] for k in range(len(string))]
    nodes = graph_degrees(list(zip(graphs, lengths)))
    fwd_b, bwd_b, fwd_f, bwd_f = step_costs(nodes, string, step_nodes)

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
    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize(dev)
    plan.sync_status(st)

    # ---- the timed region: the whole step (render, loss, loss gradient, backprop) as
    # the library's captured CUDA graph (grafx_step_graph_*), replayed on a side stream
    side = torch.cuda.Stream(dev)
    ss = gx._stream_of(side)
    torch.cuda.synchronize(dev)
    graph = plan.capture_step(src, out, tgt, loss, d_out, dP, None, ss)
    for _ in range(max(3, warmup)):
        graph.launch(ss)
    torch.cuda.synchronize(dev)
    plan.sync_status(ss)
    sampler = ClockSampler(dev.index or 0)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    t_start.record(side)
    for _ in range(steps):
        graph.launch(ss)
    t_end.record(side)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    plan.sync_status(ss)
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
    res = {"ms_total": ms_total, "ms_step": ms_total / steps, "node_samples": int(info.node_samples),
           "clocks": clocks, "launches": graph.launches(), "launches_eager": n_launch, "n_steps": N,
           "nodes": int(info.n_nodes), "tiles": {"eq_fft": int(info.eq_fft), "comp_chunk": int(info.comp_chunk),
                                                 "chosen_by": "autotune" if autotune else "defaults"},
           "ws_gb": info.ws_bytes / 1e9}

    # ---- diagnostics outside the timed region: per schedule-step durations of the same
    # step launched step by step (fwd k = 1..N, loss, bwd k = N..1)
    n_ev = N + 1 + N
    diag = 3 if N > 20 else 10
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
    flops = [fwd_f[k] for k in range(1, N + 1)] + [0] + [bwd_f[k] for k in range(N, 0, -1)]
    j = int(np.argmax(dur))
    kernel_key = labels[j]
    # the dominant step alone, launched back to back on its stream (its kernels only)
    k_step = (N - (j - N - 1)) if j > N else (j + 1)
    reps = max(3, min(20, int(200.0 / max(dur[j], 1e-3))))
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
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm, peak_kind, fp32 = peaks(n_sm)
    if flops[j] > 0:          # the multitap delay: above the FP32 ridge (see delay_flops)
        achieved = flops[j] / (ms_kernel / 1e3) / 1e12
        rl = {"bound": "alu", "achieved": achieved, "peak": fp32, "unit": "TFLOP/s", "frac": achieved / fp32,
              "algorithmic_flops_per_launch": flops[j], "algorithmic_bytes_per_launch": algo[j],
              "peak_source": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flops x max SM clock (of {peak_kind} "
                             "MEASURED_PEAKS sm_max_mhz)",
              "hbm_frac": algo[j] / (ms_kernel / 1e3) / 1e9 / hbm}
    else:
        achieved = algo[j] / (ms_kernel / 1e3) / 1e9
        rl = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
              "algorithmic_bytes_per_launch": algo[j], "peak_source": peak_kind}
    step_bytes = sum(algo)
    rl.update({"traffic": traffic_for(kernel_key), "kernel": kernel_key, "ms_per_launch": ms_kernel,
               "step": {"algorithmic_bytes": step_bytes,
                        "achieved_gbs": step_bytes / (res["ms_step"] / 1e3) / 1e9,
                        "hbm_frac": step_bytes / (res["ms_step"] / 1e3) / 1e9 / hbm},
               "eager_ms_per_step": float(dur.sum())})
    # per processor type and direction: eager ms and the fraction of its own roofline
    per = {}
    for lab, d, b, f in zip(labels, dur, algo, flops):
        key = lab.split(":")[0] + ":" + "".join(ch for ch in lab.split(":")[-1] if ch.isalpha())
        e = per.setdefault(key, [0.0, 0, 0.0])
        e[0] += float(d)
        e[1] += b
        e[2] += f
    rl["by_type"] = {k: {"ms": round(v[0], 3),
                         **({"alu_frac": round(v[2] / (v[0] / 1e3) / 1e12 / fp32, 3)} if v[2] else {}),
                         "hbm_frac": round(v[1] / (v[0] / 1e3) / 1e9 / hbm, 3) if v[1] else None}
                     for k, v in sorted(per.items(), key=lambda kv: -kv[1][0])}
    res["roofline"] = rl
    plan.sync_status(st)

    if e2e_steps:
        res["e2e"] = e2e(torch, plan, src_h, src, tgt, P, loss, d_out, dP, graph, side, ss, dev, dist,
                         e2e_steps)
    del graph
    return res


def e2e(torch, plan, src_h, src, tgt, P, loss, d_out, dP, graph, side, ss, dev, dist, n):
    """End to end through the C-ABI with host buffers: every step copies its sources and
    target from pinned memory on a copy stream (double-buffered against the previous
    step's compute), copies the parameters before its step, replays the captured step and
    copies the loss and every parameter gradient back."""
    src_pin = torch.from_numpy(src_h).pin_memory()
    tgt_pin = tgt.cpu().pin_memory()
    P_pin = {t: v.cpu().pin_memory() for t, v in P.items()}
    loss_pin = torch.empty(1).pin_memory()
    dP_pin = {t: torch.empty(v.shape).pin_memory() for t, v in P.items()}
    h2d = src_pin.numel() * 4 + tgt_pin.numel() * 4 + sum(v.numel() * 4 for v in P_pin.values())
    d2h = 4 + sum(v.numel() * 4 for v in dP_pin.values())
    src2, tgt2 = torch.empty_like(src), torch.empty_like(tgt)
    out = graph._keep[1]                    # both graphs run on one stream: one output buffer
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

    def steps(m):
        copy_in(0)
        for i in range(m):
            k = i % 2
            if i + 1 < m:
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

    steps(2)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    a.record(side)
    cstream.wait_event(a)
    steps(n)
    b.record(side)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(a.elapsed_time(b), dist, dev)
    del graph2
    return {"ms_total": ms, "steps": n, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms / n, "loss": float(loss_pin.item())}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    graphs, lengths, seeds = workload(name, args.graphs, args.samples)
    all_graphs = len(graphs)
    # this rank's graphs: the batch partitioned by cost; one graph is replicated
    from paper_2408_03204_b300 import shard
    if name == "console64" or world == 1:
        mine = list(range(len(graphs)))
        seeds = [s + (rank if name == "console64" else 0) for s in seeds]
    else:
        mine = shard.partition([g.n_nodes * L for g, L in zip(graphs, lengths)], world)[rank]
    g_r = [graphs[k] for k in mine]
    l_r = [lengths[k] for k in mine]
    s_r = [seeds[k] for k in mine]
    # host inputs before the first GPU call (spawn pool of source generators)
    src_h = sources_for(g_r, l_r, s_r, min(host_cores(), 16))
    P_all = params_for(name, graphs, "param")
    Ph_all = params_for(name, graphs, "hidden")
    P_h, Ph_h = shard.rows_of(graphs, mine, P_all), shard.rows_of(graphs, mine, Ph_all)

    import torch
    from paper_2408_03204_b300 import build
    build.build()
    import paper_2408_03204_b300 as gx
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    r = measure(gx, torch, np, g_r, l_r, src_h, P_h, Ph_h, dev, args.steps, args.warmup,
                not args.no_autotune, dist, e2e_steps=args.e2e_steps)
    units = sum_over_ranks(r["node_samples"], dist, dev)        # node-samples of one whole-job step
    value = units * args.steps / (r["ms_total"] / 1e3)
    e = r.get("e2e")
    e2e_line = None if e is None else {
        "value": units * e["steps"] / (e["ms_total"] / 1e3), "unit": UNIT,
        "h2d_bytes_per_step": e["h2d_bytes_per_step"], "d2h_bytes_per_step": e["d2h_bytes_per_step"],
        "ms_per_step": e["ms_per_step"], "loss": e["loss"]}

    secondary = None
    if name == "batch128" and not args.no_secondary:
        g2, l2, s2 = workload("console64", samples=2 ** 17)
        s2 = [s + rank for s in s2]
        r2 = measure(gx, torch, np, g2, l2, sources_for(g2, l2, s2, 1), params_for("console64", g2, "param"),
                     params_for("console64", g2, "hidden"), dev, max(10, args.steps), args.warmup,
                     not args.no_autotune, dist)
        u2 = sum_over_ranks(r2["node_samples"], dist, dev)
        secondary = {"workload": CONFIGS["console64"]["workload"], "value": u2 * max(10, args.steps) /
                     (r2["ms_total"] / 1e3), "unit": UNIT, "ms_per_step": r2["ms_step"],
                     "launches_per_step": r2["launches"], "roofline": {k: r2["roofline"][k] for k in (
                         "bound", "achieved", "peak", "unit", "frac", "kernel", "ms_per_launch", "step")},
                     "clocks": r2["clocks"]}

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(name, args.graphs, args.samples)

    if rank == 0:
        cfg = dict(CONFIGS[name], nodes=r["nodes"], graphs_total=all_graphs,
                   processed_node_samples=int(units), schedule_steps=r["n_steps"],
                   parallelism=f"graphs sharded over {world} rank(s) by cost, no collective"
                   if name == "batch128" else f"replicas{world}",
                   tiles=r["tiles"], workspace_gb_rank0=round(r["ws_gb"], 2))
        if name == "console64":
            cfg["samples"] = args.samples
        # the batch is fixed and its graphs are split over the ranks: strong scaling;
        # the single console is replicated per rank: weak
        scaling = "strong" if name == "batch128" else "weak"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_step"], "higher_is_better": True, "scaling": scaling,
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "roofline": r["roofline"], "cpu_baseline": cb, "e2e": e2e_line, "clocks": r["clocks"],
                "gpu_launches": r["launches"] * args.steps,
                "timed": "captured CUDA graph of the whole step (grafx_step_graph), "
                         f"{r['launches']} kernels per step, {r['launches_eager']} when launched step by step",
                "secondary": secondary}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
