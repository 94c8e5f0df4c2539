"""Graph rendering and its reverse-mode backward pass in float64 (oracle; test
infrastructure only, see ``oracle/__init__``).

Two renders that must agree (batching only reorders work, Sec. 2 "Batched
processing"):
  * ``render_one_by_one``: every node in topological order, Eq. 1b then Eq. 1a.
  * ``render_scheduled``: Algorithm 1 literally: schedule, reorder, index maps,
    U = S (+) 0, then for n = 1..N gather, aggregate, slice parameters, process,
    store; the output is Y_N.
``backward`` walks the nodes in reverse topological order: a node's output adjoint
is the sum of its consumers' input adjoints (plus dLoss/dY at outputs), and each
processor adjoint gives the node's input adjoint and parameter gradient.
"""
import numpy as np

from . import graph as og
from . import processors as op

I_, O_, M_, G_, S_, E_, C_, D_, R_, N_ = range(10)

DEFAULT_HP = dict(eq_taps=1023, fs=44100, comp_eps=op.COMP_EPS, eq_params="bands")


def paper_hp(fs=44100):
    """The processor settings of the paper's Sec. 3: EQ of 2047 taps parameterised by
    its 1024 log-magnitudes, multitap delay with 20 taps per channel in 100 ms slots
    (880 parameters), reverb with FFT 384 / hop 192 and 192 log-magnitudes per
    filter (768 parameters)."""
    hp = dict(eq_taps=2047, fs=fs, eq_params="logmag")
    hp.update(op.delay_paper_hp(fs))
    hp.update(op.RV_PAPER)
    return hp


def _delay_args(hp):
    return dict(nfft=hp.get("delay_nfft", op.DELAY_NFFT), taps=hp.get("delay_taps", op.DELAY_TAPS),
                slot=hp.get("delay_slot", 0))


def _hp(hp):
    out = dict(DEFAULT_HP)
    if hp:
        out.update(hp)
    return out


def process(t, u, p, hp):
    """Process(t, U_n, P_n) of Algorithm 1 for one node."""
    if t in (M_, O_):
        return op.identity_fwd(u)
    if t == G_:
        return op.gain_fwd(u, p)
    if t == S_:
        return op.imager_fwd(u, p)
    if t == E_:
        if hp["eq_params"] == "logmag":
            return op.eq_fwd_logmag(u, p, hp["eq_taps"])
        return op.eq_fwd(u, p, hp["eq_taps"], hp["fs"])
    if t == C_:
        return op.compressor_fwd(u, p, hp["comp_eps"])
    if t == N_:
        return op.noisegate_fwd(u, p, hp["comp_eps"])
    if t == D_:
        return op.delay_fwd(u, p, **_delay_args(hp))
    if t == R_:
        return op.reverb_fwd(u, p, hp["reverb_noise"], hp)
    raise NotImplementedError(f"type {t}")


def process_bwd(t, u, p, ybar, hp):
    if t in (M_, O_):
        return op.identity_bwd(u, p, ybar)
    if t == G_:
        return op.gain_bwd(u, p, ybar)
    if t == S_:
        return op.imager_bwd(u, p, ybar)
    if t == E_:
        if hp["eq_params"] == "logmag":
            return op.eq_bwd_logmag(u, p, ybar, hp["eq_taps"])
        return op.eq_bwd(u, p, ybar, hp["eq_taps"], hp["fs"])
    if t == C_:
        return op.compressor_bwd(u, p, ybar, hp["comp_eps"])
    if t == N_:
        return op.noisegate_bwd(u, p, ybar, hp["comp_eps"])
    if t == D_:
        return op.delay_bwd(u, p, ybar, **_delay_args(hp))
    if t == R_:
        return op.reverb_bwd(u, p, ybar, hp["reverb_noise"], hp)
    raise NotImplementedError(f"type {t}")


def _rows_of(types):
    """Row of each node inside P[t] (original order of that type)."""
    cnt, rows = {}, []
    for t in types:
        rows.append(cnt.get(t, 0))
        cnt[t] = rows[-1] + 1
    return rows


def _topo(types, edges):
    import heapq
    n = len(types)
    preds, succs = og.preds_succs(n, edges)
    indeg = [len(p) for p in preds]
    heap = [v for v in range(n) if indeg[v] == 0]
    heapq.heapify(heap)
    order = []
    while heap:
        v = heapq.heappop(heap)
        order.append(v)
        for w in succs[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                heapq.heappush(heap, w)
    return order


def _param(params, t, row):
    if t in (I_, O_, M_):
        return None
    return np.asarray(params[t][row], dtype=np.float64)


def render_one_by_one(types, edges, sources, params, hp=None):
    """All node outputs Y[v] (original ids), nodes visited in topological order.
    Aggregation (Eq. 1b) sums in-edges in edge-insertion order."""
    hp = _hp(hp)
    og.validate(types, edges)
    n = len(types)
    rows = _rows_of(types)
    L = sources.shape[-1]
    in_edges = [[] for _ in range(n)]
    for s, d in edges:
        in_edges[d].append(s)
    Y = [None] * n
    for v in _topo(types, edges):
        t = types[v]
        if t == I_:
            Y[v] = np.asarray(sources[rows[v]], dtype=np.float64)
            continue
        u = np.zeros((2, L))
        for s in in_edges[v]:
            u = u + Y[s]
        Y[v] = process(t, u, _param(params, t, rows[v]), hp)
    return Y


def outputs_of(types, Y):
    return np.stack([Y[v] for v in range(len(types)) if types[v] == O_])


def render_scheduled(types, edges, sources, params, hp=None, method="beam", width=32):
    """Algorithm 1: returns (Y_N stacked over output nodes, U in new order, maps)."""
    hp = _hp(hp)
    string, steps = og.schedule(types, edges, method, width)
    mp = og.index_maps(types, edges, steps)
    n = len(types)
    L = sources.shape[-1]
    K = sum(1 for t in types if t == I_)
    U = np.zeros((n, 2, L))
    U[:K] = np.asarray(sources, dtype=np.float64)          # U = S (+) 0
    sp, cp, cs = mp["step_ptr"], mp["csr_ptr"], mp["csr_src"]
    for k in range(1, len(string)):
        t = string[k]
        a, b = sp[k], sp[k + 1]                            # I^S_n: a slice
        # gather + aggregate (I^G_n, I^A_n)
        Un = np.zeros((b - a, 2, L))
        for v in range(a, b):
            for e in range(cp[v], cp[v + 1]):
                Un[v - a] += U[cs[e]]
        # parameter slice (I^P_n) and processing
        for v in range(a, b):
            p = _param(params, t, mp["param_row"][v])
            U[v] = process(t, Un[v - a], p, hp)
    return U[sp[-2]:sp[-1]], U, dict(mp, string=string, steps=steps)


def backward(types, edges, sources, params, dY, hp=None, cond=False):
    """Reverse-mode pass.  dY[j] is dLoss/dY for the j-th output node (original
    order).  Returns (dparams {type: [rows, cols]}, dsources [K, 2, L]); with
    ``cond`` also {type: [rows, cols]} holding, for the gain and imager gradients
    (plain sums over the signal), the sum of the magnitudes of their terms (0 for the
    other types): a sum that cancels to much less than that is ill-conditioned, and
    no FP32 evaluation can match it to a relative bound."""
    hp = _hp(hp)
    n = len(types)
    rows = _rows_of(types)
    L = sources.shape[-1]
    Y = render_one_by_one(types, edges, sources, params, hp)
    preds, succs = og.preds_succs(n, edges)
    outs = [v for v in range(n) if types[v] == O_]
    ybar = [np.zeros((2, L)) for _ in range(n)]
    for j, v in enumerate(outs):
        ybar[v] = ybar[v] + np.asarray(dY[j], dtype=np.float64)
    ubar = [None] * n
    dparams = {t: np.zeros(np.shape(params[t]), dtype=np.float64) for t in params}
    dcond = {t: np.zeros(np.shape(params[t]), dtype=np.float64) for t in params}
    K = sum(1 for t in types if t == I_)
    dsrc = np.zeros((K, 2, L))
    for v in reversed(_topo(types, edges)):
        t = types[v]
        for w in succs[v]:          # each edge v -> w contributes w's input adjoint
            ybar[v] = ybar[v] + ubar[w]
        if t == I_:
            dsrc[rows[v]] = ybar[v]
            continue
        u = np.zeros((2, L))
        for s in preds[v]:
            u = u + Y[s]
        ubar[v], pbar = process_bwd(t, u, _param(params, t, rows[v]), ybar[v], hp)
        if pbar.size:
            dparams[t][rows[v]] = pbar
        if cond and t == G_:
            dcond[t][rows[v]] = op.gain_bwd_abs(u, _param(params, t, rows[v]), ybar[v])
        if cond and t == S_:
            dcond[t][rows[v]] = op.imager_bwd_abs(u, _param(params, t, rows[v]), ybar[v])
    if cond:
        return dparams, dsrc, dcond
    return dparams, dsrc
