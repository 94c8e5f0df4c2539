"""GPU parity of the processors in the paper's own settings (Sec. 3) against the FP64
oracle: the 2047-tap EQ parameterised by its 1024 log-magnitudes, the multitap delay
with 20 taps per channel in 100 ms slots (880 parameters) and the reverb with FFT 384 /
hop 192, 192 per-bin log-magnitudes per filter and wet output (768 parameters).
Tolerances as in the other parity tests: outputs 1e-5 at full scale, gradients 1e-3
relative with a floor of 1e-2 of the tensor's largest entry."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import (GpuRun, assert_grad_close, assert_out_close, flat_sources, split_rows,
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
    run = GpuRun(graphs, lengths, P, src_flat, preset="paper")
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
