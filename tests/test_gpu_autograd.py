"""The autograd functions pair every backward with its own forward (Algorithm 1: a
backprop reads the rows of the render it differentiates).  Two renders (or two loss
evaluations) on one plan before .backward() must each get the gradients of their own
forward: equal to the FP64 oracle's, and bit-equal to a plan that saw one render only."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import assert_grad_close, flat_sources

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


def _setup(L=6001):
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.console_cfg1()
    src_flat, src_per = flat_sources([g], [L], [5])
    P1 = synth.random_params(g, 21)
    P2 = synth.random_params(g, 22)
    plan = gx.Plan([gx.Graph.from_lists(g.types, g.edges)], [L], eq_taps=255)
    plan.bind_workspace("cuda")
    s = torch.tensor(src_flat, device="cuda")
    dev = lambda P: {t: torch.tensor(v, device="cuda").requires_grad_(True) for t, v in P.items()}
    return gx, torch, g, L, plan, s, src_per[0][:, :, :L], P1, P2, dev


def test_two_renders_before_backward():
    gx, torch, g, L, plan, s, src, P1, P2, dev = _setup()
    A, B = dev(P1), dev(P2)
    out1 = gx.render(plan, s, A)
    out2 = gx.render(plan, s, B)          # the plan's rows now hold the second render
    rng = np.random.Generator(np.random.PCG64(3))
    w1 = torch.tensor(rng.standard_normal(out1.numel()).astype(np.float32), device="cuda")
    w2 = torch.tensor(rng.standard_normal(out2.numel()).astype(np.float32), device="cuda")
    ((out1 * w1).sum() + (out2 * w2).sum()).backward()
    hp = dict(eq_taps=255)
    for P, D, w in ((P1, A, w1), (P2, B, w2)):
        pitch = (L + 3) // 4 * 4
        wP, _ = orr.backward(g.types, g.edges, src, P, w.cpu().numpy().reshape(-1, 2, pitch)[:, :, :L], hp)
        for t in P:
            assert_grad_close(D[t].grad.cpu().numpy(), wP[t], what=f"type {t}")
    # a plan that rendered once gives the same bits
    for P, D, w in ((P1, A, w1), (P2, B, w2)):
        E = dev(P)
        (gx.render(plan, s, E) * w).sum().backward()
        for t in P:
            assert torch.equal(E[t].grad, D[t].grad), t


def test_two_losses_before_backward():
    gx, torch, g, L, plan, s, src, P1, P2, dev = _setup()
    T = dev(synth.random_params(g, 23))
    with torch.no_grad():
        tgt = gx.render(plan, s, T).clone()
    A, B = dev(P1), dev(P2)
    out1 = gx.render(plan, s, A)
    l1 = gx.mrstft_loss(plan, out1, tgt)
    out2 = gx.render(plan, s, B)
    l2 = gx.mrstft_loss(plan, out2, tgt)   # replaces the loss's cached spectra and the rows
    (l1 + 2.0 * l2).backward()
    for P, D, k in ((P1, A, 1.0), (P2, B, 2.0)):
        E = dev(P)
        (k * gx.mrstft_loss(plan, gx.render(plan, s, E), tgt)).backward()
        for t in P:
            assert torch.equal(E[t].grad, D[t].grad), t
