"""Shared helpers of the GPU tests: run a graph through the C-ABI library and compare
with the FP64 oracle on the same seeded inputs."""
import numpy as np

import synth

OUT_TOL = 1e-5      # max |y - y_ref| <= OUT_TOL * max(1, max|y_ref|)
GRAD_TOL = 1e-3     # |g - g_ref| <= GRAD_TOL * max(|g_ref|, GRAD_FLOOR * max|g_ref| of the tensor)
GRAD_FLOOR = 1e-2
# A gradient that is a plain sum over the signal (gain, imager) can cancel to far less
# than the sum of its terms' magnitudes C: its terms' inputs (the FP32 adjoint and
# signal rows) each carry at least half an ulp of rounding, which does not cancel with
# the terms, so no FP32 evaluation is good to better than about eps32/2 * C = 6e-8 C
# whatever the sum's size; that absolute bound is accepted too where the oracle
# supplies C.  (The one case that needs it, an imager sum cancelling to C/267000 in a
# random graph with noisegates, errs by 7.1e-9 C with the hardware ln/exp of the
# compressor's gain path and by the same bits with correctly rounded ones.)
GRAD_COND = 6e-8


def assert_out_close(got, want, tol=OUT_TOL):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    assert err <= tol * scale, f"max abs err {err:.3e} > {tol * scale:.3e}"
    return err / scale


def assert_grad_close(got, want, tol=GRAD_TOL, floor=GRAD_FLOOR, what="", cond=None):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    ref = np.maximum(np.abs(want), floor * float(np.abs(want).max()) + 1e-30)
    if cond is not None:
        ref = np.maximum(ref, GRAD_COND / tol * np.asarray(cond, dtype=np.float64))
    rel = np.abs(got - want) / ref
    worst = float(rel.max())
    assert worst <= tol, f"{what}: worst relative gradient error {worst:.3e} at {np.unravel_index(rel.argmax(), rel.shape)}"
    return worst


def flat_sources(graphs, lengths, seeds):
    """Per-graph source stacks [K_g, 2, pitch_g] concatenated into one flat buffer."""
    parts, per = [], []
    for g, L, s in zip(graphs, lengths, seeds):
        P = (L + 3) // 4 * 4
        src = synth.sources(s, g.count(synth.I), L, pitch=P)
        per.append(src)
        parts.append(src.reshape(-1))
    return np.concatenate(parts), per


def split_rows(flat, graphs, lengths, kind=synth.O):
    """Flat [rows][2][pitch] buffer back into per-graph arrays [rows_g, 2, L]."""
    out, off = [], 0
    for g, L in zip(graphs, lengths):
        P = (L + 3) // 4 * 4
        n = g.count(kind)
        a = flat[off:off + n * 2 * P].reshape(n, 2, P)[:, :, :L]
        out.append(a)
        off += n * 2 * P
    return out


def union_params(graphs, seed, preset="compact"):
    """One parameter table per type over the union (original order), seeded per graph."""
    return synth.union_params(graphs, seed, preset=preset)


def per_graph_params(graphs, P):
    out, cnt = [], {}
    for g in graphs:
        d = {}
        for t in P:
            n = g.count(t)
            if n:
                d[t] = P[t][cnt.get(t, 0):cnt.get(t, 0) + n]
            cnt[t] = cnt.get(t, 0) + n
        out.append(d)
    return out


class DeviceRun:
    """One plan bound to a workspace, with device copies of sources and parameters."""

    def __init__(self, graphs, lengths, P, src_flat, **plan_kw):
        import torch
        import paper_2408_03204_b300 as gx
        self.gx, self.torch = gx, torch
        self.graphs, self.lengths = graphs, lengths
        self.plan = gx.Plan([gx.Graph.from_lists(g.types, g.edges, g.ports) for g in graphs], lengths, **plan_kw)
        self.plan.bind_workspace("cuda")
        self.P = {t: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for t, v in P.items()}
        self.src = torch.tensor(src_flat, dtype=torch.float32, device="cuda")
        self.plan.bind_params(self.P)
        if any(g.count(8) for g in graphs):
            import synth
            self.noise = torch.tensor(synth.reverb_noise(), device="cuda").contiguous()
            self.plan.bind_reverb_noise(self.noise)

    def render(self):
        torch = self.torch
        out = torch.empty(self.plan.info.out_elems, dtype=torch.float32, device="cuda")
        self.plan.render_raw(self.src, out, self.gx._stream(torch, out.device))
        self.plan.sync_status()
        return out

    def backprop(self, d_out, want_sources=True):
        torch = self.torch
        d_out = torch.as_tensor(d_out, dtype=torch.float32, device="cuda").contiguous()
        dP = {t: torch.full_like(p, float("nan")) for t, p in self.P.items()}
        dS = torch.full_like(self.src, float("nan")) if want_sources else None
        self.plan.backprop_raw(self.src, d_out, dP, dS, self.gx._stream(torch, d_out.device))
        self.plan.sync_status()
        return {t: v.cpu().numpy() for t, v in dP.items()}, (dS.cpu().numpy() if want_sources else None)


def reverb_noise_device(torch):
    import synth
    return torch.tensor(synth.reverb_noise(), device="cuda").contiguous()
