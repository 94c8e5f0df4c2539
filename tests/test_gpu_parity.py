"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the same
seeded inputs.  Outputs within 1e-5 at full scale; parameter and source gradients
within 1e-3 relative (floor 1e-2 of the tensor's largest entry)."""
import numpy as np
import pytest

import synth
from oracle import render as orr, loss as ol
from tests.gpu_common import (DeviceRun, assert_grad_close, assert_out_close, flat_sources, split_rows,
                              union_params, per_graph_params)

pytestmark = pytest.mark.gpu

I, O, M, G, S, E, C = 0, 1, 2, 3, 4, 5, 6


def hparams(eq_taps=63):
    return dict(eq_taps=eq_taps, reverb_noise=synth.reverb_noise().astype(np.float64))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


def single_node_graph(t, fan_in=1):
    g = synth.Graph()
    ins = [g.add(I) for _ in range(fan_in)]
    v = g.add(t)
    o = g.add(O)
    for i in ins:
        g.connect(i, v)
    g.connect(v, o)
    return g


def run_case(graphs, lengths, seed=11, eq_taps=63, linear_loss=True, **kw):
    src_flat, src_per = flat_sources(graphs, lengths, [seed + k for k in range(len(graphs))])
    P = union_params(graphs, seed)
    run = DeviceRun(graphs, lengths, P, src_flat, eq_taps=eq_taps, **kw)
    out = run.render().cpu().numpy()
    hp = hparams(eq_taps)
    got_rows = split_rows(out, graphs, lengths)
    Pg = per_graph_params(graphs, P)
    for g, L, src, p, got in zip(graphs, lengths, src_per, Pg, got_rows):
        want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src[:, :, :L], p, hp, ports=g.ports))
        assert_out_close(got, want)
    return run, P, src_per, out


@pytest.mark.parametrize("t", [M, G, S, E, C])
@pytest.mark.parametrize("L", [4096, 5003, 2 ** 14 + 2])
def test_single_processor_fwd_bwd(t, L):
    g = single_node_graph(t, fan_in=2)
    run, P, src_per, out = run_case([g], [L])
    rng = np.random.Generator(np.random.PCG64(L + t))
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], dict(eq_taps=63))
    for tt in P:
        assert_grad_close(dP[tt], wP[tt], what=f"type {tt}")
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


@pytest.mark.parametrize("taps", [255, 1023])
def test_eq_long_filters(taps):
    g = single_node_graph(E)
    run, P, src_per, _ = run_case([g], [20000], eq_taps=taps)
    L, Pd = 20000, 20000
    W = np.random.Generator(np.random.PCG64(9)).standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0], P, W, dict(eq_taps=taps))
    assert_grad_close(dP[E], wP[E], what="eq bands")
    assert_grad_close(dS.reshape(-1, 2, Pd), wS, what="sources")


def test_cfg1_forward_full_size():
    """8 tracks i->g->e(255)->c, 2 buses, master; 2^15 samples."""
    run_case([synth.console_cfg1()], [2 ** 15], seed=1, eq_taps=255)


def test_compressor_long_chunks_and_extreme_alpha():
    g = single_node_graph(C)
    L = 2 ** 17 + 8
    src_flat, src_per = flat_sources([g], [L], [5])
    for alpha in (0.9, 0.9999):
        P = {C: np.array([[alpha, np.log(0.005), 0.6908, 6.0]], np.float32)}
        run = DeviceRun([g], [L], P, src_flat)
        got = run.render().cpu().numpy().reshape(1, 2, L)
        want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src_per[0], P))
        assert_out_close(got, want)
        W = np.random.Generator(np.random.PCG64(3)).standard_normal((1, 2, L)).astype(np.float32)
        dP, _ = run.backprop(W.reshape(-1), want_sources=False)
        wP, _ = orr.backward(g.types, g.edges, src_per[0], P, W)
        assert_grad_close(dP[C], wP[C], what=f"comp alpha={alpha}")


def test_compressor_steps_deterministic():
    """Render and backprop twice on a batch whose compressor steps hold many chunks per
    node: the chunk carries are fixed-order sums, so every bit repeats (a look-back that
    stops at the first finished predecessor rounds differently from run to run)."""
    rng = np.random.Generator(np.random.PCG64(31))
    graphs = [synth.random_console(rng, budget_lo=24, budget_hi=64, kinds=(G, E, C)) for _ in range(6)]
    lengths = [int(rng.integers(40000, 70000)) for _ in graphs]
    src_flat, _ = flat_sources(graphs, lengths, list(range(6)))
    P = union_params(graphs, 5)
    run = DeviceRun(graphs, lengths, P, src_flat, eq_taps=63)
    o1 = run.render().cpu().numpy()
    W = np.random.Generator(np.random.PCG64(32)).standard_normal(o1.shape).astype(np.float32)
    g1, s1 = run.backprop(W)
    o2 = run.render().cpu().numpy()
    g2, s2 = run.backprop(W)
    assert np.array_equal(o1, o2), "render is not deterministic"
    for t in g1:
        assert np.array_equal(g1[t], g2[t]), f"parameter gradient of type {t} is not deterministic"
    assert np.array_equal(s1, s2), "source gradient is not deterministic"


def test_random_graphs_fwd_bwd():
    from tests.helpers import random_dag
    rng = np.random.Generator(np.random.PCG64(21))
    for k in range(4):
        g = random_dag(rng, n_inputs=3, n_mid=10, n_outputs=2, kinds=(M, G, S, E, C))
        L = int(rng.integers(3000, 9000))
        run, P, src_per, out = run_case([g], [L], seed=100 + k)
        Pd = (L + 3) // 4 * 4
        W = np.zeros((2, 2, Pd), np.float32)
        W[:, :, :L] = rng.standard_normal((2, 2, L)).astype(np.float32)
        dP, dS = run.backprop(W.reshape(-1))
        wP, wS, wC = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], dict(eq_taps=63), cond=True)
        for t in P:
            assert_grad_close(dP[t], wP[t], what=f"type {t}", cond=wC[t])
        assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


def test_batched_equals_single_and_deterministic():
    rng = np.random.Generator(np.random.PCG64(8))
    graphs = [synth.random_console(rng, budget_lo=16, budget_hi=48, kinds=(G, S, E, C)) for _ in range(5)]
    lengths = [int(rng.integers(4000, 12000)) for _ in graphs]
    src_flat, _ = flat_sources(graphs, lengths, list(range(5)))
    P = union_params(graphs, 4)
    batched = DeviceRun(graphs, lengths, P, src_flat, eq_taps=63)
    ob = batched.render().cpu().numpy()
    ob2 = batched.render().cpu().numpy()
    assert np.array_equal(ob, ob2), "render is not deterministic"
    rows_b = split_rows(ob, graphs, lengths)
    off_s = 0
    Pg = per_graph_params(graphs, P)
    for g, L, p, rb in zip(graphs, lengths, Pg, rows_b):
        n = g.count(I) * 2 * ((L + 3) // 4 * 4)
        single = DeviceRun([g], [L], p, src_flat[off_s:off_s + n], eq_taps=63)
        off_s += n
        rs = split_rows(single.render().cpu().numpy(), [g], [L])[0]
        # identical per-node arithmetic; only the summation order of fan-in >= 3 may differ
        assert_out_close(rb, rs, tol=1e-6)


def test_schedule_methods_agree():
    g = synth.console_cfg2(tracks=12, levels=2)
    L = 6000
    src_flat, _ = flat_sources([g], [L], [2])
    P = union_params([g], 5)
    outs = [DeviceRun([g], [L], P, src_flat, eq_taps=63, schedule=m).render().cpu().numpy()
            for m in ("beam", "greedy", "one_by_one")]
    for o in outs[1:]:
        assert_out_close(o, outs[0], tol=1e-6)


def test_mrstft_loss_and_grad():
    import torch
    import paper_2408_03204_b300 as gx
    g = single_node_graph(M)
    L = 3 * 4096 + 7
    Pd = (L + 3) // 4 * 4
    rng = np.random.Generator(np.random.PCG64(17))
    y = np.zeros((1, 2, Pd), np.float32)
    t = np.zeros((1, 2, Pd), np.float32)
    y[:, :, :L] = 0.3 * rng.standard_normal((1, 2, L))
    t[:, :, :L] = 0.3 * rng.standard_normal((1, 2, L))
    plan = gx.Plan([gx.Graph.from_lists(g.types, g.edges)], [L]).bind_workspace("cuda")
    yd = torch.tensor(y.reshape(-1), device="cuda")
    td = torch.tensor(t.reshape(-1), device="cuda")
    loss = torch.empty(1, device="cuda")
    st = gx._stream(torch, yd.device)
    plan.loss_raw(yd, td, loss, st)
    d = torch.empty_like(yd)
    plan.loss_backward_raw(yd, td, d, st)
    plan.sync_status()
    want = ol.mrstft(y[:, :, :L].astype(np.float64), t[:, :, :L].astype(np.float64))
    assert abs(loss.item() - want) <= 1e-4 * abs(want), (loss.item(), want)
    wg = ol.mrstft_grad(y[:, :, :L].astype(np.float64), t[:, :, :L].astype(np.float64))
    gd = d.cpu().numpy().reshape(1, 2, Pd)
    assert np.all(gd[:, :, L:] == 0)
    # dL/dy is an element-wise intermediate: its log-magnitude term carries 1/|Y|, and
    # an FP32 spectrum resolves |Y| only to ~1e-7 of the frame norm, so on the few
    # smallest bins the relative error reaches a few 1e-3.  Parameter gradients (sums
    # over whole signals) are held to 1e-3 elsewhere.
    assert_grad_close(gd[:, :, :L], wg, tol=5e-3, what="dloss/dy")


def _cfg2_case(L):
    g = synth.console_cfg2()
    src_flat, src_per = flat_sources([g], [L], [2])
    P = union_params([g], 2)
    Ph = union_params([g], 102)
    hp = dict(eq_taps=1023)
    target = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src_per[0], Ph, hp))
    y_ref = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src_per[0], P, hp))
    run = DeviceRun([g], [L], P, src_flat, eq_taps=1023)
    return g, src_per, P, hp, target, y_ref, run


# Measured conditioning of the loss path (FP64 oracle, 64-track console): perturbing the
# rendered mix by 1e-7 (the FP32 rounding level at full scale) moves the oracle's own
# parameter gradients by up to 43% element-wise (relative to max(|g|, 1e-2 max|g|)) and
# by about 2% in norm at 2^17 samples, because the log-magnitude term's gradient
# sign(.)/|Y| flips and spikes on near-equal and tiny bins (one ulp of FP32 on Y alone
# moves the oracle's dL/dY by up to 2.2% element-wise).  Through the loss, the FP32 path
# is therefore checked norm-wise (5e-2) and by direction (cosine > 0.998) against the
# oracle's chain; element-wise, the backward kernels are held to the 1e-3 bar fed the
# oracle's dL/dY and fed the GPU's own, and the GPU's dL/dY is held to 1e-3 wherever the
# oracle's is stable under FP32 rounding of Y.
LOSS_CHAIN_NORM_TOL = 5e-2


@pytest.mark.parametrize("L", [2 ** 15, 2 ** 17])
def test_cfg2_fwd_bwd_mrstft(L):
    """64-track nested console, full chain, STFT loss against a target rendered (by the
    oracle) from hidden parameters; 2^17 is the benchmarked size and launch setup."""
    import torch
    g, src_per, P, hp, target, y_ref, run = _cfg2_case(L)
    out = run.render()
    assert_out_close(out.cpu().numpy().reshape(1, 2, L), y_ref)
    tgt = torch.tensor(target.astype(np.float32).reshape(-1), device="cuda")
    loss = torch.empty(1, device="cuda")
    st = run.gx._stream(torch, out.device)
    run.plan.loss_raw(out, tgt, loss, st)
    d_out = torch.empty_like(out)
    run.plan.loss_backward_raw(out, tgt, d_out, st)
    want_loss = ol.mrstft(y_ref, target)
    assert abs(loss.item() - want_loss) <= 1e-4 * abs(want_loss)
    dY = ol.mrstft_grad(y_ref, target)
    wP, _ = orr.backward(g.types, g.edges, src_per[0], P, dY, hp)
    # (1) backward through the graph from the oracle's dL/dY
    dP1, _ = run.backprop(dY.astype(np.float32).reshape(-1), want_sources=False)
    for t in P:
        assert_grad_close(dP1[t], wP[t], what=f"type {t} (oracle dL/dY)")
    # (2) the whole FP32 chain: GPU loss gradient, then GPU backward
    dP2, _ = run.backprop(d_out, want_sources=False)
    for t in P:
        a, b = dP2[t].astype(np.float64).ravel(), wP[t].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel <= LOSS_CHAIN_NORM_TOL and cos > 0.998, (t, rel, cos)
    # (3) the same FP32 chain element-wise: the oracle's backward fed the GPU's own dL/dY
    # (measured worst 2.6e-5 at 2^17: every backward kernel of the chain at the 1e-3 bar)
    dYg = d_out.cpu().numpy().astype(np.float64).reshape(1, 2, L)
    wPg, _ = orr.backward(g.types, g.edges, src_per[0], P, dYg, hp)
    for t in P:
        assert_grad_close(dP2[t], wPg[t], what=f"type {t} (GPU chain vs oracle backward of the GPU's dL/dY)")
    # (4) dL/dY element-wise against the oracle's at the GPU's own rendered Y (upcast) and
    # the same FP32 target.  An FP32 STFT of a 2048-point frame is good to a few ulps of
    # the frame's scale (its 11 radix passes each round), and where a change of Y by 4
    # ulps moves the oracle's own value by more than 1e-4 (bins with |Y| ~ |T| flip the
    # sign of the L1 log term; one ulp alone moves it by up to 2.2% at 2^17) no FP32 loss
    # can be held to 1e-3; on the other elements (86% of them at 2^17) it is.
    Yg = out.cpu().numpy().astype(np.float64).reshape(1, 2, L)
    T32 = target.astype(np.float32).astype(np.float64)
    dYo = ol.mrstft_grad(Yg, T32)
    ref = np.maximum(np.abs(dYo), 1e-2 * np.abs(dYo).max())
    rng = np.random.default_rng(L)
    ulp = np.spacing(Yg.astype(np.float32)).astype(np.float64)
    spread = np.zeros_like(dYo)
    for _ in range(4):
        sgn = np.where(rng.random(Yg.shape) < 0.5, -1.0, 1.0)
        spread = np.maximum(spread, np.abs(ol.mrstft_grad(Yg + 4.0 * sgn * ulp, T32) - dYo))
    stable = spread <= 1e-4 * ref
    assert stable.mean() >= 0.6, stable.mean()
    worst = float((np.abs(dYg - dYo) / ref)[stable].max())
    assert worst <= 1e-3, f"dL/dY on FP32-stable elements: {worst:.3e}"


D = 7


@pytest.mark.parametrize("L", [5003, 20000])
def test_delay_fwd_bwd(L):
    """Multitap delay: exact integer-delay forward; backward adjoint, FIR gradients and
    the surrogate z-gradient (Eq. 15)."""
    g = single_node_graph(D, fan_in=2)
    run, P, src_per, out = run_case([g], [L], seed=41)
    rng = np.random.Generator(np.random.PCG64(L))
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L])
    q = dP[D].reshape(-1, 2, 4, 22)
    wq = wP[D].reshape(-1, 2, 4, 22)
    assert_grad_close(q[..., :2], wq[..., :2], what="delay z (surrogate)")
    assert_grad_close(q[..., 2:], wq[..., 2:], what="delay FIR log-magnitudes")
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


def test_random_graphs_with_delay():
    from tests.helpers import random_dag
    rng = np.random.Generator(np.random.PCG64(77))
    for k in range(2):
        g = random_dag(rng, n_inputs=2, n_mid=7, n_outputs=1, kinds=(M, G, S, E, C, D))
        L = int(rng.integers(5000, 9000))
        run, P, src_per, out = run_case([g], [L], seed=300 + k)
        Pd = (L + 3) // 4 * 4
        W = np.zeros((1, 2, Pd), np.float32)
        W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
        dP, dS = run.backprop(W.reshape(-1))
        wP, wS, wC = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], dict(eq_taps=63), cond=True)
        for t in P:
            assert_grad_close(dP[t], wP[t], what=f"type {t}", cond=wC[t])
        assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


R = 8


@pytest.mark.parametrize("L", [6001, 20000])
def test_reverb_fwd_bwd(L):
    """Filtered-noise reverb: 88200-tap masked-noise IR, partitioned FFT convolution,
    and the adjoint through convolution, ISTFT, masks and bands."""
    g = single_node_graph(R, fan_in=2)
    run, P, src_per, out = run_case([g], [L], seed=51)
    rng = np.random.Generator(np.random.PCG64(L + 1))
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], hparams())
    assert_grad_close(dP[R], wP[R], what="reverb parameters")
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")
