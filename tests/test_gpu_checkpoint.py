"""Signal checkpointing (plan option checkpoint_steps) on the GPU: the checkpointed
backward recomputes each earlier segment's forward with the same deterministic kernels,
so outputs and every gradient equal the plan without checkpointing bit for bit; and
both agree with the FP64 oracle."""
import numpy as np
import pytest

import synth
from gpu_common import GRAD_TOL, DeviceRun, assert_grad_close, flat_sources, union_params
from oracle import render as orr

pytestmark = pytest.mark.gpu


def _run(graphs, lengths, P, src, d_seed, **kw):
    run = DeviceRun(graphs, lengths, P, src, **kw)
    out = run.render().cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(d_seed))
    d_out = rng.standard_normal(out.shape).astype(np.float32)
    dP, dS = run.backprop(d_out)
    return run, out, d_out, dP, dS


@pytest.mark.parametrize("k", [2, 3])
def test_checkpointed_equals_plain_cfg1(k):
    g = synth.console_cfg1()
    L = 8192 + 13
    src, per = flat_sources([g], [L], [31])
    P = union_params([g], 32)
    _, o0, d, dP0, dS0 = _run([g], [L], P, src, 5, eq_taps=255)
    run, o1, _, dP1, dS1 = _run([g], [L], P, src, 5, eq_taps=255, checkpoint_steps=k)
    assert run.plan.info.ws_bytes <= DeviceRun([g], [L], P, src, eq_taps=255).plan.info.ws_bytes
    np.testing.assert_array_equal(o0, o1)
    for t in dP0:
        np.testing.assert_array_equal(dP0[t], dP1[t])
    np.testing.assert_array_equal(dS0, dS1)


def test_checkpointed_random_graphs_all_types_match_oracle():
    rng = np.random.Generator(np.random.PCG64(44))
    graphs = [synth.random_console(rng, budget_lo=20, budget_hi=40, kinds=(synth.G, synth.E, synth.C, synth.S,
                                                                          synth.D, synth.R)) for _ in range(3)]
    lengths = [6001, 9000, 7003]
    src, per = flat_sources(graphs, lengths, [50, 51, 52])
    P = union_params(graphs, 60)
    _, o0, d, dP0, dS0 = _run(graphs, lengths, P, src, 6, eq_taps=255)
    _, o1, _, dP1, dS1 = _run(graphs, lengths, P, src, 6, eq_taps=255, checkpoint_steps=2)
    np.testing.assert_array_equal(o0, o1)
    for t in dP0:
        np.testing.assert_array_equal(dP0[t], dP1[t])
    np.testing.assert_array_equal(dS0, dS1)
    # and the oracle's gradient of the first graph's gain parameters
    g0 = graphs[0]
    hp = {"eq_taps": 255, "reverb_noise": synth.reverb_noise().astype(np.float64)}
    P0 = {t: v[:g0.count(t)] for t, v in P.items() if g0.count(t)}
    n_out0 = g0.count(synth.O)
    P_ = (lengths[0] + 3) // 4 * 4
    dY = d[:n_out0 * 2 * P_].reshape(n_out0, 2, P_)[:, :, :lengths[0]].astype(np.float64)
    dP_ref, _ = orr.backward(g0.types, g0.edges, per[0][:, :, :lengths[0]], P0, dY, hp)
    if synth.G in dP_ref:
        assert_grad_close(dP1[synth.G][:g0.count(synth.G)], dP_ref[synth.G], GRAD_TOL, what="gain")


def test_checkpointed_step_graph_replay_equals_eager():
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.console_cfg1()
    L = 8192
    src, per = flat_sources([g], [L], [71])
    P = union_params([g], 72)
    run = DeviceRun([g], [L], P, src, eq_taps=255, checkpoint_steps=2)
    plan = run.plan
    tgt = run.render().clone() * 0.5
    out = torch.empty_like(tgt)
    loss = torch.zeros(1, device="cuda")
    d_out = torch.empty_like(tgt)
    dP = {t: torch.empty_like(p) for t, p in run.P.items()}
    s = torch.cuda.Stream()
    st = gx._stream_of(s)
    s.wait_stream(torch.cuda.current_stream())
    graph = plan.capture_step(run.src, out, tgt, loss, d_out, dP, None, st)
    graph.launch(st)
    s.synchronize()
    g_rep = {t: v.cpu().numpy() for t, v in dP.items()}
    l_rep = loss.item()
    with torch.cuda.stream(s):
        plan.render_raw(run.src, out, st)
        plan.loss_raw(out, tgt, loss, st)
        plan.loss_backward_raw(out, tgt, d_out, st)
        plan.backprop_raw(run.src, d_out, dP, None, st)
    s.synchronize()
    assert loss.item() == l_rep
    for t in dP:
        np.testing.assert_array_equal(dP[t].cpu().numpy(), g_rep[t])


def test_node_inputs_rejected_with_checkpointing():
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.console_cfg1()
    src, per = flat_sources([g], [4096], [1])
    run = DeviceRun([g], [4096], union_params([g], 2), src, eq_taps=255, checkpoint_steps=2)
    out = run.render()
    dst = torch.empty((1, 2, 4096), device="cuda")
    with pytest.raises(gx.GrafxError):
        run.plan.node_inputs_raw(run.src, out, [1], dst, 4096, gx._stream(torch, dst.device))
