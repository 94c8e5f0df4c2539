"""CUDA-graph replay of a whole fit step and the tile autotuner (batched rendering,
a fixed launch sequence per plan): replays must equal the eager calls exactly, and a
tuned plan must render the same mix as the default one."""
import numpy as np
import pytest

import synth
from tests.gpu_common import DeviceRun, assert_out_close, flat_sources, union_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


def test_step_graph_replay_equals_eager():
    import torch
    g = synth.console_cfg2(tracks=12, levels=2)
    L = 8192
    src_flat, _ = flat_sources([g], [L], [3])
    run = DeviceRun([g], [L], union_params([g], 7), src_flat, eq_taps=255)
    st = run.gx._stream(torch, run.src.device)
    tgt = run.render().clone() * 0.5 + 0.01
    out, loss, d_out = torch.empty_like(tgt), torch.empty(1, device="cuda"), torch.empty_like(tgt)
    dP = {t: torch.empty_like(p) for t, p in run.P.items()}
    # eager reference
    run.plan.render_raw(run.src, out, st)
    run.plan.loss_raw(out, tgt, loss, st)
    run.plan.loss_backward_raw(out, tgt, d_out, st)
    run.plan.backprop_raw(run.src, d_out, dP, None, st)
    torch.cuda.synchronize()
    ref = (out.clone(), loss.clone(), {t: v.clone() for t, v in dP.items()})
    side = torch.cuda.Stream()
    ss = run.gx._stream_of(side)
    graph = run.plan.capture_step(run.src, out, tgt, loss, d_out, dP, None, ss)
    assert graph.launches() > 10
    for _ in range(2):
        out.zero_(); loss.zero_()
        for v in dP.values():
            v.zero_()
        torch.cuda.synchronize()
        graph.launch(ss)
        torch.cuda.synchronize()
        assert torch.equal(out, ref[0]) and torch.equal(loss, ref[1])
        for t in dP:
            assert torch.equal(dP[t], ref[2][t]), t
    run.plan.sync_status(st)


def test_autotuner_picks_valid_tiles(tmp_path):
    import paper_2408_03204_b300 as gx
    from paper_2408_03204_b300 import autotune
    g = synth.console_cfg1()
    L = 2 ** 14
    lists = [[g.types, [list(e) for e in g.edges]]]
    best = autotune.autotune([gx.Graph.from_lists(g.types, g.edges)], [L], graph_lists=lists, eq_taps=255,
                             cache=str(tmp_path / "tune.json"))
    assert best in autotune.candidates(255)
    again = autotune.autotune([gx.Graph.from_lists(g.types, g.edges)], [L], graph_lists=lists, eq_taps=255,
                              cache=str(tmp_path / "tune.json"))
    assert again == best
    src_flat, _ = flat_sources([g], [L], [1])
    P = union_params([g], 1)
    a = DeviceRun([g], [L], P, src_flat, eq_taps=255).render().cpu().numpy()
    b = DeviceRun([g], [L], P, src_flat, eq_taps=255, **best).render().cpu().numpy()
    assert_out_close(b, a, tol=2e-6)


def test_fused_step_pair_matches_step_by_step():
    """The nested console's gain -> EQ, imager -> gain and mix -> output steps run fused
    in a whole render and backprop; one step at a time they run unfused.  Outputs, parameter gradients and
    source adjoints agree bit for bit."""
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.console_cfg2()
    L = 8192
    src_flat, _ = flat_sources([g], [L], [3])
    P = union_params([g], 3)
    run = DeviceRun([g], [L], P, src_flat, eq_taps=255)
    plan = run.plan
    assert plan.info.fused_pairs == 3
    N = plan.info.n_steps
    st = gx._stream(torch, run.src.device)
    out_f = torch.empty(plan.info.out_elems, device="cuda")
    out_s = torch.full_like(out_f, float("nan"))
    plan.render_raw(run.src, out_f, st)
    for k in range(1, N + 1):
        plan.render_steps_raw(run.src, out_s, k, k + 1, st)
    torch.cuda.synchronize()
    assert torch.equal(out_f, out_s)
    d_out = torch.randn(plan.info.out_elems, device="cuda")
    dP_f = {t: torch.full_like(p, float("nan")) for t, p in run.P.items()}
    dP_s = {t: torch.full_like(p, float("nan")) for t, p in run.P.items()}
    dS_f, dS_s = torch.full_like(run.src, float("nan")), torch.full_like(run.src, float("nan"))
    plan.render_raw(run.src, out_f, st)
    plan.backprop_raw(run.src, d_out, dP_f, dS_f, st)
    for k in range(N, -1, -1):
        plan.backprop_steps_raw(run.src, d_out, dP_s, dS_s, k, k + 1, st)
    torch.cuda.synchronize()
    plan.sync_status(st)
    for t in dP_f:
        assert torch.equal(dP_f[t], dP_s[t]), t
    assert torch.equal(dS_f, dS_s)


def test_fused_steps_with_a_source_batch():
    """Two source sets through the nested console in one plan (source_batch = 2; both
    fused step pairs apply to the union): each copy's output equals a one-copy plan's
    bit for bit, and the parameter gradients equal the sum of the one-copy plans'."""
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.console_cfg2()
    L, B = 4096, 2
    P = union_params([g], 5)
    Pt = {t: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for t, v in P.items()}
    srcs = [flat_sources([g], [L], [40 + b])[0] for b in range(B)]
    G = gx.Graph.from_lists(g.types, g.edges)
    batched = gx.Plan([G], [L], eq_taps=255, source_batch=B).bind_workspace("cuda")
    single = gx.Plan([G], [L], eq_taps=255).bind_workspace("cuda")
    assert batched.info.fused_pairs == 3 and single.info.fused_pairs == 3
    batched.bind_params(Pt)
    single.bind_params(Pt)
    st = gx._stream(torch, torch.device("cuda"))
    src_b = torch.tensor(np.concatenate(srcs), device="cuda")
    out_b = torch.empty(batched.info.out_elems, device="cuda")
    batched.render_raw(src_b, out_b, st)
    rng = np.random.Generator(np.random.PCG64(8))
    d_b = torch.tensor(rng.standard_normal(batched.info.out_elems).astype(np.float32), device="cuda")
    dP_b = {t: torch.empty_like(p) for t, p in Pt.items()}
    batched.backprop_raw(src_b, d_b, dP_b, None, st)
    n_out = single.info.out_elems
    sum_P = {t: torch.zeros_like(p, dtype=torch.float64) for t, p in Pt.items()}
    for b in range(B):
        src = torch.tensor(srcs[b], device="cuda")
        out = torch.empty(n_out, device="cuda")
        single.render_raw(src, out, st)
        torch.cuda.synchronize()
        assert torch.equal(out, out_b[b * n_out:(b + 1) * n_out])
        dP = {t: torch.empty_like(p) for t, p in Pt.items()}
        single.backprop_raw(src, d_b[b * n_out:(b + 1) * n_out].contiguous(), dP, None, st)
        torch.cuda.synchronize()
        for t in dP:
            sum_P[t] += dP[t].double()
    batched.sync_status(st)
    for t in dP_b:   # the batched plan folds the copies' gradients in copy order
        np.testing.assert_allclose(dP_b[t].cpu().numpy(), sum_P[t].cpu().numpy(), rtol=1e-5, atol=1e-6)
