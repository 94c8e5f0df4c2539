"""The fit loop (paper_2408_03204_b300.fit) and the warm-start pipeline
(paper_2408_03204_b300.warmstart) on the GPU: composition and training behaviour.
The kernels they call are checked against the oracle elsewhere."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2408_03204_b300 as gx
    from paper_2408_03204_b300 import fit as gfit
    from paper_2408_03204_b300 import warmstart as gws
    return gx, torch, gfit, gws


def _small_batch(gws, ws, n_graphs=3, L=8192, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    gl = gws.random_graph_lists(rng, n_graphs, lo=20, hi=40)
    return gws.make_batch(ws, gl, L, 100 + seed, 200 + seed)


def test_fit_graph_replay_equals_eager_and_descends(env):
    gx, torch, gfit, gws = env
    ws = gws.WarmStart(max_batch=256, max_rows=256, max_len=8192)
    batch, src, hidden, target, neutral = _small_batch(gws, ws)
    runs = []
    for use_graph in (True, False):
        P = {t: p.clone() for t, p in neutral.items()}
        f = gfit.Fit(batch.plan, src, target, P, lr=1e-2, use_graph=use_graph)
        losses = []
        for _ in range(25):
            f.step()
            losses.append(f.current_loss())
        runs.append((losses, {t: p.cpu().numpy() for t, p in P.items()}))
    assert runs[0][0] == runs[1][0]
    for t in runs[0][1]:
        np.testing.assert_array_equal(runs[0][1][t], runs[1][1][t])
    losses = runs[0][0]
    assert losses[-1] < 0.9 * losses[0], losses


def test_fit_from_theta0_maps_parameters(env):
    gx, torch, gfit, gws = env
    ws = gws.WarmStart(max_batch=256, max_rows=256, max_len=8192)
    batch, src, hidden, target, neutral = _small_batch(gws, ws, seed=2)
    th0 = {}
    for t, p in hidden.items():
        codes = torch.tensor(gfit.param_codes(t), dtype=torch.int8, device="cuda")
        th = torch.empty_like(p)
        gx._check(gx.lib().grafx_params_to_theta(gx._ptr(p), gx._ptr(codes), p.shape[1], p.numel(), gx._ptr(th),
                                                  gx._stream(torch, p.device)))
        th0[t] = th
    P = {t: p.clone() for t, p in neutral.items()}
    f = gfit.Fit(batch.plan, src, target, P, lr=1e-2, theta0=th0)
    for t in hidden:
        np.testing.assert_allclose(P[t].cpu().numpy(), hidden[t].cpu().numpy(), rtol=2e-4, atol=2e-4)
    # started at the hidden parameters: the loss is (close to) zero
    f.step()
    assert f.current_loss() < 1e-3


def test_features_compose_node_inputs_and_cross_gain(env):
    gx, torch, gfit, gws = env
    from oracle import warmstart as ow
    ws = gws.WarmStart(max_batch=512, max_rows=64, max_len=8192)
    batch, src, hidden, target, neutral = _small_batch(gws, ws, seed=3)
    feats = ws.features(batch, src, target, neutral)
    torch.cuda.synchronize()
    n = len(batch.ids)
    assert feats.shape == (n, 256, 32) and torch.isfinite(feats).all()
    f = feats.cpu().numpy()
    # node-input channels: the log-mel of grafx_node_inputs rows, recomputed separately;
    # cross-gain channels: the oracle's of those rows against the graph's target row
    P = (8192 + 3) // 4 * 4
    out = torch.empty(batch.plan.info.out_elems, device="cuda")
    st = gx._stream(torch, out.device)
    batch.plan.bind_params(neutral)
    batch.plan.render_raw(src, out, st)
    u = torch.empty((5, 2, P), device="cuda")
    batch.plan.node_inputs_raw(src, out, batch.ids[-5:], u, P, st)
    f2 = torch.empty((5, 256, 32), device="cuda")
    ws.net.logmel_raw(u, 5, 2 * P, P, 8192, None, 5, 0, f2, st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f2[:, :128].cpu().numpy(), f[-5:, :128])
    uh = u.cpu().numpy()
    th = target.cpu().numpy().reshape(-1, 2, P)
    for i in range(5):
        want = ow.xgain(uh[i, :, :8192], th[batch.outrow[n - 5 + i], :, :8192])
        np.testing.assert_allclose(f[n - 5 + i, 128:], want, rtol=0, atol=1e-3)
    # the samples are sorted by head and their counts match the graphs' processors
    heads = [gws.HEAD_OF[t] for t in batch.types]
    assert heads == sorted(heads)
    want = sum(sum(1 for t in tys if t in gws.HEAD_OF) for tys, _ in batch.graph_lists)
    assert n == want


def test_warm_start_training_reduces_loss_and_predicts(env):
    gx, torch, gfit, gws = env
    ws = gws.WarmStart(max_batch=256, max_rows=512, max_len=8192, lr=1e-3)
    losses, t_data, t_train, n = gws.train(ws, 12, 8192, graphs_per_batch=6, epochs=12, minibatch=64, seed=7)
    assert n > 64
    assert np.mean(losses[-5:]) < 0.8 * np.mean(losses[:5]), (losses[:5], losses[-5:])
    batch, src, hidden, target, neutral = _small_batch(gws, ws, seed=9)
    feats = ws.features(batch, src, target, neutral)
    theta = ws.predict(feats, batch.types)
    tabs = ws.theta_tables(batch, theta)
    torch.cuda.synchronize()
    assert torch.isfinite(theta).all()
    for t, tab in tabs.items():
        assert tab.shape == (batch.plan.info.n_type_rows[t], gx.PARAM_COLS[t])


def test_trained_network_beats_the_prior_mean():
    """What training gains: on held-out consoles of the training distribution (32-200
    nodes), the gain, imager, EQ and compressor heads beat the training-set mean
    (standardised MSE 1.0), the baseline a fit without the network would have to beat.
    (The delay head cannot: a tap up to 500 ms late has no frame overlap with its input.)"""
    gx, torch, gfit, gws = env_tuple()
    ws = gws.WarmStart(max_batch=512, max_rows=1024, max_len=32768, lr=1e-3)
    gws.train(ws, 480, 32768, graphs_per_batch=48, epochs=10, minibatch=256, seed=11)
    print("held-out standardised MSE per head:", ws.held_out)
    for h in "gsec":
        assert ws.held_out[h][0] < HEAD_BOUND, (h, ws.held_out)


HEAD_BOUND = 0.95


def env_tuple():
    import torch
    import paper_2408_03204_b300 as gx
    from paper_2408_03204_b300 import fit as gfit
    from paper_2408_03204_b300 import warmstart as gws
    return gx, torch, gfit, gws


def test_fit_resume_from_saved_state_is_bitwise_identical(env, tmp_path):
    gx, torch, gfit, gws = env
    ws = gws.WarmStart(max_batch=256, max_rows=256, max_len=8192)
    batch, src, hidden, target, neutral = _small_batch(gws, ws, seed=4)
    P = {t: p.clone() for t, p in neutral.items()}
    f = gfit.Fit(batch.plan, src, target, P, lr=1e-2)
    for _ in range(10):
        f.step()
    path = str(tmp_path / "fit.bin")
    f.save(path)
    ref = []
    for _ in range(10):
        f.step()
        ref.append(f.current_loss())
    P2 = {t: p.clone() for t, p in neutral.items()}
    f2 = gfit.Fit(batch.plan, src, target, P2, lr=1e-2)
    f2.load(path)
    got = []
    for _ in range(10):
        f2.step()
        got.append(f2.current_loss())
    assert got == ref


def test_warmstart_resume_from_saved_state(env, tmp_path):
    gx, torch, gfit, gws = env
    a = gws.WarmStart(max_batch=64, max_rows=64, max_len=8192, seed=3)
    feats = (-6 + 3 * torch.randn(32, 256, 32, device="cuda")).contiguous()
    types = sorted([3] * 8 + [5] * 12 + [6] * 12, key=lambda t: gws.HEAD_OF[t])
    tgt = torch.randn(32, 176, device="cuda")
    for _ in range(3):
        a.train_step(feats, tgt, types)
    path = str(tmp_path / "ws.bin")
    a.save(path)
    la = [float(a.train_step(feats, tgt, types)) for _ in range(3)]
    b = gws.WarmStart(max_batch=64, max_rows=64, max_len=8192, seed=99)
    b.load(path)
    lb = [float(b.train_step(feats, tgt, types)) for _ in range(3)]
    assert la == lb
    assert torch.equal(a.W, b.W)
