"""GPU parity of the fused Adam update with parameter maps (grafx_adam_step) and the
inverse map (grafx_params_to_theta) against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

from oracle import optim as oo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


@pytest.mark.parametrize("t", [6, 13])
def test_adam_steps_match_oracle(t):
    """Compressor columns [alpha, T, W, R] and attack/release columns [alpha_attack,
    alpha_release, T, W, R] (the attack map reaches down to 0.5)."""
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    rng = np.random.Generator(np.random.PCG64(5))
    rows = 37
    cols = 4 if t == 6 else 5
    codes = oo.param_codes(t, cols)
    lead = [rng.uniform(0.91, 0.999, rows)] if t == 6 else [rng.uniform(0.55, 0.98, rows), rng.uniform(0.91, 0.999, rows)]
    P0 = np.stack(lead + [rng.uniform(-9, 0, rows), rng.uniform(0.3, 1.0, rows),
                          rng.uniform(1.2, 8, rows)], axis=1).astype(np.float32)
    dev = torch.device("cuda")
    p = torch.tensor(P0, device=dev)
    cd = torch.tensor(codes, device=dev)
    th = torch.empty_like(p)
    st = gx._stream(torch, dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.grafx_params_to_theta(ptr(p), ptr(cd), cols, p.numel(), ptr(th), st) == 0
    torch.cuda.synchronize()
    th_ref = oo.to_theta(P0.astype(np.float64), codes)
    np.testing.assert_allclose(th.cpu().numpy(), th_ref, rtol=2e-5, atol=2e-5)
    th_o = th.cpu().numpy().astype(np.float64)      # continue both from the same theta
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    mo, vo = np.zeros_like(th_o), np.zeros_like(th_o)
    for t in range(1, 6):
        gp = rng.standard_normal((rows, cols)).astype(np.float32)
        g = torch.tensor(gp, device=dev)
        assert lib.grafx_adam_step(ptr(th), ptr(m), ptr(v), ptr(g), ptr(p), ptr(cd), cols, p.numel(), t,
                                   ctypes.c_float(1e-2), ctypes.c_float(0.9), ctypes.c_float(0.999),
                                   ctypes.c_float(1e-8), st) == 0
        gth = gp.astype(np.float64) * oo.dparam_dtheta(th_o, codes)
        th_o, mo, vo = oo.adam_step(th_o, mo, vo, gth, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(th.cpu().numpy(), th_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(p.cpu().numpy(), oo.to_param(th_o, codes), rtol=1e-5, atol=1e-6)


def test_adam_delay_taps_normalised_and_regularised():
    """Delay rows (Sec. 3 after Eq. 15): each tap's z-gradient scaled to unit length plus
    the unit-circle penalty's gradient, then Adam; the FIR log-magnitudes as plain Adam."""
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    rng = np.random.Generator(np.random.PCG64(7))
    rows, cols = 29, 176
    codes = oo.param_codes(7, cols)
    P0 = rng.uniform(-1.3, 1.3, (rows, cols)).astype(np.float32)
    P0[3, 0:2] = 0.0                                   # z = 0 (penalty gradient taken as 0)
    dev = torch.device("cuda")
    p = torch.tensor(P0, device=dev)
    cd = torch.tensor(codes, device=dev)
    th = p.clone()
    st = gx._stream(torch, dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    th_o = P0.astype(np.float64)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    mo, vo = np.zeros_like(th_o), np.zeros_like(th_o)
    for t in range(1, 7):
        gp = (rng.standard_normal((rows, cols)) * 10.0 ** rng.uniform(-6, 3, (rows, cols))).astype(np.float32)
        gp[5, 22:24] = 0.0                             # a zero z-gradient stays zero
        g = torch.tensor(gp, device=dev)
        assert lib.grafx_adam_step(ptr(th), ptr(m), ptr(v), ptr(g), ptr(p), ptr(cd), cols, p.numel(), t,
                                   ctypes.c_float(1e-2), ctypes.c_float(0.9), ctypes.c_float(0.999),
                                   ctypes.c_float(1e-8), st) == 0
        gth = oo.delay_z_grad(th_o, gp.astype(np.float64), codes)
        th_o, mo, vo = oo.adam_step(th_o, mo, vo, gth, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(th.cpu().numpy(), th_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(p.cpu().numpy(), th_o, rtol=1e-5, atol=1e-5)
