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

Ports (Eq. 1a/1b with M inputs and N outputs): ``ports[e] = (k, l)`` says that edge e
carries output k of its source to input l of its destination (default (0, 0) for every
edge).  Input l of a node is the sum of its edges into l; U holds one row per output
port (N_sum rows).  ``render_ports`` returns every node's list of outputs;
``render_one_by_one`` returns each node's first output (the only one of a
single-output node).
"""
import numpy as np

from . import graph as og
from . import processors as op

I_, O_, M_, G_, S_, E_, C_, D_, R_, N_, P_, J_, K_, A_ = range(14)

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
    if t == A_:
        return op.ballistic_fwd(u, p, hp["comp_eps"])
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
    if t == A_:
        return op.ballistic_bwd(u, p, ybar, hp["comp_eps"])
    if t == D_:
        return op.delay_bwd(u, p, ybar, **_delay_args(hp))
    if t == R_:
        return op.reverb_bwd(u, p, ybar, hp["reverb_noise"], hp)
    raise NotImplementedError(f"type {t}")


def process_ports(t, us, p, hp):
    """Process of a node with its list of inputs; returns its list of outputs."""
    if t == P_:
        return op.split_fwd(us[0])
    if t == J_:
        return [op.merge_fwd(us)]
    if t == K_:
        return [op.sidechain_fwd(us, p, hp["comp_eps"])]
    return [process(t, us[0], p, hp)]


def process_bwd_ports(t, us, p, ybars, hp):
    """Adjoint of ``process_ports``: (list of input adjoints, parameter gradient)."""
    if t == P_:
        return op.split_bwd(us[0], ybars), np.zeros(0)
    if t == J_:
        return op.merge_bwd(us, ybars[0]), np.zeros(0)
    if t == K_:
        return op.sidechain_bwd(us, p, ybars[0], hp["comp_eps"])
    ub, pb = process_bwd(t, us[0], p, ybars[0], hp)
    return [ub], pb


def _ports(edges, ports):
    return list(ports) if ports is not None else [(0, 0)] * len(edges)


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
    if t in (I_, O_, M_, P_, J_):
        return None
    return np.asarray(params[t][row], dtype=np.float64)


def render_ports(types, edges, sources, params, hp=None, ports=None):
    """Every node's list of outputs (original ids), nodes visited in topological order.
    Aggregation (Eq. 1b) sums each input's edges in edge-insertion order."""
    hp = _hp(hp)
    og.validate(types, edges, ports=ports)
    pt = _ports(edges, ports)
    n = len(types)
    rows = _rows_of(types)
    L = sources.shape[-1]
    in_edges = [[] for _ in range(n)]
    for (s, d), (k, l) in zip(edges, pt):
        in_edges[d].append((s, k, l))
    Y = [None] * n
    for v in _topo(types, edges):
        t = types[v]
        if t == I_:
            Y[v] = [np.asarray(sources[rows[v]], dtype=np.float64)]
            continue
        us = [np.zeros((2, L)) for _ in range(og.PORTS[t][0])]
        for s, k, l in in_edges[v]:
            us[l] = us[l] + Y[s][k]
        Y[v] = process_ports(t, us, _param(params, t, rows[v]), hp)
    return Y


def render_one_by_one(types, edges, sources, params, hp=None, ports=None):
    """All node outputs Y[v] (original ids; a multi-output node's first output)."""
    return [ys[0] for ys in render_ports(types, edges, sources, params, hp, ports)]


def outputs_of(types, Y):
    return np.stack([Y[v] for v in range(len(types)) if types[v] == O_])


def render_scheduled(types, edges, sources, params, hp=None, method="beam", width=32, ports=None):
    """Algorithm 1: returns (Y_N stacked over output nodes, U in new order with one row
    per output port (N_sum rows), maps)."""
    hp = _hp(hp)
    pt = _ports(edges, ports)
    og.validate(types, edges, ports=ports)
    string, steps = og.schedule(types, edges, method, width)
    mp = og.index_maps(types, edges, steps)
    n = len(types)
    L = sources.shape[-1]
    K = sum(1 for t in types if t == I_)
    sigma = mp["sigma"]
    inv = [0] * n
    for v in range(n):
        inv[sigma[v]] = v
    new_types = [types[inv[v]] for v in range(n)]
    # first U row of each node (new order): its output ports are consecutive rows
    first = [0] * (n + 1)
    for v in range(n):
        first[v + 1] = first[v] + og.PORTS[new_types[v]][1]
    U = np.zeros((first[n], 2, L))
    U[:K] = np.asarray(sources, dtype=np.float64)          # U = S (+) 0
    # in-edges of each new id with their ports
    ins = [[] for _ in range(n)]
    for (s, d), (k, l) in zip(edges, pt):
        ins[sigma[d]].append((sigma[s], k, l))
    sp = mp["step_ptr"]
    for st in range(1, len(string)):
        t = string[st]
        a, b = sp[st], sp[st + 1]                            # I^S_n: a slice
        # gather + aggregate per input port (I^G_n, I^A_n)
        Un = [[np.zeros((2, L)) for _ in range(og.PORTS[t][0])] for _ in range(a, b)]
        for v in range(a, b):
            for s, k, l in sorted(ins[v]):
                Un[v - a][l] += U[first[s] + k]
        # parameter slice (I^P_n) and processing
        for v in range(a, b):
            p = _param(params, t, mp["param_row"][v])
            for k, y in enumerate(process_ports(t, Un[v - a], p, hp)):
                U[first[v] + k] = y
    return U[first[sp[-2]]:first[sp[-1]]], U, dict(mp, string=string, steps=steps)


def backward(types, edges, sources, params, dY, hp=None, cond=False, ports=None):
    """Reverse-mode pass.  dY[j] is dLoss/dY for the j-th output node (original
    order).  Returns (dparams {type: [rows, cols]}, dsources [K, 2, L]); with
    ``cond`` also {type: [rows, cols]} holding, for the gain and imager gradients
    (plain sums over the signal), the sum of the magnitudes of their terms (0 for the
    other types): a sum that cancels to much less than that is ill-conditioned, and
    no FP32 evaluation can match it to a relative bound."""
    hp = _hp(hp)
    pt = _ports(edges, ports)
    n = len(types)
    rows = _rows_of(types)
    L = sources.shape[-1]
    Y = render_ports(types, edges, sources, params, hp, ports)
    in_edges = [[] for _ in range(n)]
    out_edges = [[] for _ in range(n)]
    for (s, d), (k, l) in zip(edges, pt):
        in_edges[d].append((s, k, l))
        out_edges[s].append((d, k, l))
    outs = [v for v in range(n) if types[v] == O_]
    ybar = [[np.zeros((2, L)) for _ in range(og.PORTS[types[v]][1])] for v in range(n)]
    for j, v in enumerate(outs):
        ybar[v][0] = ybar[v][0] + np.asarray(dY[j], dtype=np.float64)
    ubar = [None] * n
    dparams = {t: np.zeros(np.shape(params[t]), dtype=np.float64) for t in params}
    dcond = {t: np.zeros(np.shape(params[t]), dtype=np.float64) for t in params}
    K = sum(1 for t in types if t == I_)
    dsrc = np.zeros((K, 2, L))
    for v in reversed(_topo(types, edges)):
        t = types[v]
        for w, k, l in out_edges[v]:   # each edge v:k -> w:l contributes w's input-l adjoint
            ybar[v][k] = ybar[v][k] + ubar[w][l]
        if t == I_:
            dsrc[rows[v]] = ybar[v][0]
            continue
        us = [np.zeros((2, L)) for _ in range(og.PORTS[t][0])]
        for s, k, l in in_edges[v]:
            us[l] = us[l] + Y[s][k]
        p = _param(params, t, rows[v])
        ubar[v], pbar = process_bwd_ports(t, us, p, ybar[v], hp)
        if pbar.size:
            dparams[t][rows[v]] = pbar
        if cond and t == G_:
            dcond[t][rows[v]] = op.gain_bwd_abs(us[0], p, ybar[v][0])
        if cond and t == S_:
            dcond[t][rows[v]] = op.imager_bwd_abs(us[0], p, ybar[v][0])
    if cond:
        return dparams, dsrc, dcond
    return dparams, dsrc
