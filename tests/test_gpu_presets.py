"""GPU parity of the processors in the paper's own settings (Sec. 3) against the FP64
oracle: the 2047-tap EQ parameterised by its 1024 log-magnitudes, the multitap delay
with 20 taps per channel in 100 ms slots (880 parameters) and the reverb with FFT 384 /
hop 192, 192 per-bin log-magnitudes per filter and wet output (768 parameters); and
source-level batching (Sec. 2 "Batched processing"): B source sets through one graph
with shared parameters, checked copy by copy against the oracle, with the parameter
gradients summed over the copies.
Tolerances as in the other parity tests: outputs 1e-5 at full scale, gradients 1e-3
relative with a floor of 1e-2 of the tensor's largest entry."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import (DeviceRun, assert_grad_close, assert_out_close, flat_sources, split_rows,
                              union_params, per_graph_params)

pytestmark = pytest.mark.gpu

I, O, M, G, S, E, C, D, R, N = range(10)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def paper_hp():
    hp = orr.paper_hp()
    hp["reverb_noise"] = synth.reverb_noise().astype(np.float64)
    return hp


def single_node_graph(t, fan_in=2):
    g = synth.Graph()
    ins = [g.add(I) for _ in range(fan_in)]
    v = g.add(t)
    o = g.add(O)
    for i in ins:
        g.connect(i, v)
    g.connect(v, o)
    return g


def run_paper(graphs, lengths, seed):
    src_flat, src_per = flat_sources(graphs, lengths, [seed + k for k in range(len(graphs))])
    P = union_params(graphs, seed, preset="paper")
    run = DeviceRun(graphs, lengths, P, src_flat, preset="paper")
    for t, a in P.items():
        assert run.plan.param_cols[t] == a.shape[1] == synth.PAPER_PARAM_COLS[t]
    out = run.render().cpu().numpy()
    hp = paper_hp()
    for g, L, src, p, got in zip(graphs, lengths, src_per, per_graph_params(graphs, P),
                                 split_rows(out, graphs, lengths)):
        want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src[:, :, :L], p, hp))
        assert_out_close(got, want)
    return run, P, src_per


def backward_check(run, g, L, P, src, seed, split=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src[:, :, :L], P, W[:, :, :L], paper_hp())
    for t in P:
        if split and t in split:
            split[t](dP[t], wP[t])
        else:
            assert_grad_close(dP[t], wP[t], what=f"type {t}")
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


@pytest.mark.parametrize("L", [5003, 30001])
def test_paper_eq_2047_taps_logmag(L):
    g = single_node_graph(E)
    run, P, src = run_paper([g], [L], seed=61)
    assert run.plan.info.eq_fft == 8192
    backward_check(run, g, L, P, src[0], L + 5)


def _delay_split(got, want):
    q = got.reshape(-1, 2, 20, 22)
    wq = want.reshape(-1, 2, 20, 22)
    assert_grad_close(q[..., :2], wq[..., :2], what="delay z (surrogate)")
    assert_grad_close(q[..., 2:], wq[..., 2:], what="delay FIR log-magnitudes")


@pytest.mark.parametrize("L", [20000, 100003])
def test_paper_delay_20_taps_in_slots(L):
    """Taps past the signal's end (L = 20000 reaches 4 of the 20 slots) contribute
    nothing; L = 100003 covers every slot of the 2 s effect with a ragged tail."""
    g = single_node_graph(D)
    run, P, src = run_paper([g], [L], seed=71)
    backward_check(run, g, L, P, src[0], L + 7, split={D: _delay_split})


@pytest.mark.parametrize("L", [6001, 30001])
def test_paper_reverb_384_192(L):
    g = single_node_graph(R)
    run, P, src = run_paper([g], [L], seed=81)
    backward_check(run, g, L, P, src[0], L + 9)


def test_paper_settings_random_graphs():
    from tests.helpers import random_dag
    rng = np.random.Generator(np.random.PCG64(91))
    for k in range(2):
        g = random_dag(rng, n_inputs=2, n_mid=8, n_outputs=1, kinds=(M, G, S, E, C, D, R, N))
        L = int(rng.integers(9000, 14000))
        run, P, src = run_paper([g], [L], seed=400 + k)
        backward_check(run, g, L, P, src[0], 500 + k)


@pytest.mark.parametrize("preset", ["compact", "paper"])
def test_source_batch(preset):
    import torch
    import paper_2408_03204_b300 as gx
    from tests.helpers import random_dag
    rng = np.random.Generator(np.random.PCG64(33))
    g = random_dag(rng, n_inputs=2, n_mid=7, n_outputs=2, kinds=(M, G, S, E, C, D, R, N))
    B, L = 3, 7001
    Pd = (L + 3) // 4 * 4
    K, O_ = g.count(I), g.count(O)
    srcs = [synth.sources(700 + b, K, L, pitch=Pd) for b in range(B)]
    P = synth.random_params(g, 17, preset=preset)
    plan = gx.Plan([gx.Graph.from_lists(g.types, g.edges)], [L], preset=preset, source_batch=B)
    plan.bind_workspace("cuda")
    Pt = {t: torch.tensor(v, device="cuda").contiguous() for t, v in P.items()}
    plan.bind_params(Pt)
    noise = torch.tensor(synth.reverb_noise(), device="cuda").contiguous()
    plan.bind_reverb_noise(noise)
    src = torch.tensor(np.stack(srcs).reshape(-1), device="cuda")
    assert src.numel() == plan.info.src_elems
    out = torch.empty(plan.info.out_elems, device="cuda")
    st = gx._stream(torch, out.device)
    plan.render_raw(src, out, st)
    W = rng.standard_normal((B, O_, 2, Pd)).astype(np.float32)
    W[..., L:] = 0
    dP = {t: torch.full_like(p, float("nan")) for t, p in Pt.items()}
    dS = torch.full_like(src, float("nan"))
    plan.backprop_raw(src, torch.tensor(W.reshape(-1), device="cuda"), dP, dS, st)
    plan.sync_status()
    got = out.cpu().numpy().reshape(B, O_, 2, Pd)
    dSg = dS.cpu().numpy().reshape(B, K, 2, Pd)
    hp = paper_hp() if preset == "paper" else dict(eq_taps=1023, reverb_noise=synth.reverb_noise().astype(np.float64))
    want_P = {t: np.zeros(v.shape) for t, v in P.items()}
    for b in range(B):
        Y = orr.render_one_by_one(g.types, g.edges, srcs[b][:, :, :L], P, hp)
        assert_out_close(got[b, :, :, :L], orr.outputs_of(g.types, Y))
        wP, wS = orr.backward(g.types, g.edges, srcs[b][:, :, :L], P, W[b, :, :, :L], hp)
        assert_grad_close(dSg[b, :, :, :L], wS, what=f"sources of copy {b}")
        for t in want_P:
            want_P[t] += wP[t]
    for t in P:
        assert_grad_close(dP[t].cpu().numpy(), want_P[t], what=f"type {t} summed over copies")
    # a partial backward range is refused with a source batch
    with pytest.raises(gx.GrafxError):
        plan.backprop_steps_raw(src, torch.tensor(W.reshape(-1), device="cuda"), dP, dS, 1, 2, st)
