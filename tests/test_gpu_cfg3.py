"""The batched workload at full size (128 random consoles, uneven L up to 2^18, one
plan, one launch sequence per schedule step): sampled graphs of the batch against the
FP64 oracle, forward and backward: the two cheapest, the one with the longest signal,
the one with the most nodes and the deepest one.  Only the sampled graphs get synthetic
sources from the shared generator; the other graphs get seeded noise made on the device
(their renders are independent of the sampled ones: the batch is a disjoint union)."""
import numpy as np
import pytest

import synth
from gpu_common import GRAD_TOL, assert_grad_close, assert_out_close, union_params
from oracle import render as orr

pytestmark = pytest.mark.gpu


def _depth(g):
    """Nodes on the longest input -> output path."""
    preds = {}
    for s_, d_ in g.edges:
        preds.setdefault(d_, []).append(s_)
    done = {}

    def f(v):
        if v not in done:
            done[v] = 1 + max((f(u) for u in preds.get(v, [])), default=0)
        return done[v]
    return max(f(v) for v in range(g.n_nodes))


def test_cfg3_full_batch_sampled_graphs_match_oracle():
    import torch
    import paper_2408_03204_b300 as gx
    graphs, lengths = synth.batch_cfg3()
    assert len(graphs) == 128
    pitches = [(L + 3) // 4 * 4 for L in lengths]
    plan = gx.Plan([gx.Graph.from_lists(g.types, g.edges) for g in graphs], lengths)
    plan.bind_workspace("cuda")
    P = union_params(graphs, 3000)
    Pd = {t: torch.tensor(v, device="cuda").contiguous() for t, v in P.items()}
    plan.bind_params(Pd)
    # source rows: graph-major, [K_g][2][pitch_g]
    offs, o = [], 0
    for g, p in zip(graphs, pitches):
        offs.append(o)
        o += g.count(synth.I) * 2 * p
    assert o == plan.info.src_elems
    gen = torch.Generator(device="cuda").manual_seed(3)
    src = (0.05 * torch.randn(o, device="cuda", generator=gen)).contiguous()
    cost = [g.n_nodes * L for g, L in zip(graphs, lengths)]
    # the two cheapest graphs, the longest signal, the most nodes and the deepest graph
    # (longest input -> output path: the largest work lists and scan chunk counts)
    sampled = sorted(range(len(graphs)), key=lambda k: cost[k])[:2]
    for key in (lambda k: lengths[k], lambda k: graphs[k].n_nodes, lambda k: _depth(graphs[k])):
        k = max(range(len(graphs)), key=key)
        if k not in sampled:
            sampled.append(k)
    per = {}
    for k in sampled:
        g, L, p = graphs[k], lengths[k], pitches[k]
        s = synth.sources(300 + k, g.count(synth.I), L, pitch=p)
        per[k] = s
        src[offs[k]:offs[k] + s.size] = torch.from_numpy(s.reshape(-1)).cuda()
    out = torch.empty(plan.info.out_elems, device="cuda")
    st = gx._stream(torch, out.device)
    plan.render_raw(src, out, st)
    rng = np.random.Generator(np.random.PCG64(33))
    d_out = torch.tensor(rng.standard_normal(plan.info.out_elems).astype(np.float32), device="cuda")
    dP = {t: torch.full_like(v, float("nan")) for t, v in Pd.items()}
    plan.backprop_raw(src, d_out, dP, None, st)
    plan.sync_status(st)
    assert torch.isfinite(out).all()
    out_h, d_h = out.cpu().numpy(), d_out.cpu().numpy()
    dP_h = {t: v.cpu().numpy() for t, v in dP.items()}
    # per-graph output rows and parameter rows
    out_off, oo = [], 0
    for g, p in zip(graphs, pitches):
        out_off.append(oo)
        oo += g.count(synth.O) * 2 * p
    row0 = {t: np.cumsum([0] + [g.count(t) for g in graphs]) for t in P}
    for k in sampled:
        g, L, p = graphs[k], lengths[k], pitches[k]
        n_o = g.count(synth.O)
        Pk = {t: P[t][row0[t][k]:row0[t][k + 1]] for t in P if g.count(t)}
        Y = orr.render_one_by_one(g.types, g.edges, per[k][:, :, :L], Pk)
        want = orr.outputs_of(g.types, Y)
        got = out_h[out_off[k]:out_off[k] + n_o * 2 * p].reshape(n_o, 2, p)
        assert_out_close(got[:, :, :L], want)
        assert not got[:, :, L:].any()
        dY = d_h[out_off[k]:out_off[k] + n_o * 2 * p].reshape(n_o, 2, p)[:, :, :L].astype(np.float64)
        wP, _ = orr.backward(g.types, g.edges, per[k][:, :, :L], Pk, dY)
        for t in wP:
            assert_grad_close(dP_h[t][row0[t][k]:row0[t][k + 1]], wP[t], GRAD_TOL, what=f"graph {k} type {t}")
