"""Graph checks, type scheduling, node reordering and index maps (FP64 oracle; test
infrastructure only, see ``oracle/__init__``).

Follows the paper's Sec. 2:
  * Definitions (Eq. 1a/1b): node i computes y_i = f_i(u_i, p_i) with u_i the sum of
    its predecessors' outputs; cycles are not allowed.
  * Batched processing: a schedule is a sequence V_0..V_N that is a partition, causal
    and homogeneous (conditions (i)-(iii)).
  * Type scheduling: for a chosen type the subset is maximal, so a schedule is a type
    string; V_0 holds every input and V_N every output.  Greedy picks the type with
    the most computable nodes; beam search keeps several partial schedules; the
    brute-force search gives the shortest string.
  * Algorithm 1: the reordering sigma makes each step a contiguous range of node ids,
    then the read/write index maps are built.

Readings of what the paper leaves open:
  * Types i and o are never chosen mid-schedule; the o step comes last, once every
    non-output node is scheduled.
  * Greedy ties go to the smallest type id.
  * Beam(B): expand every candidate by every type with a non-empty ready set; merge
    equal scheduled sets keeping the lexicographically smallest type string; stop as
    soon as an expansion is complete (smallest complete string wins); otherwise keep
    the B best by (most nodes scheduled, then smallest string).  Beam(1) is greedy.
  * Optimal is the same search with no pruning (tiny graphs only).
  * One-by-one: one non-i/o node per step, smallest original id first among the
    ready ones; the outputs still form the last step.
  * sigma ranks nodes by (step, original id).  In-edge lists are sorted by the new
    source id, consumer lists by the new consumer id; multi-edges repeat.
"""
import heapq

I_TYPE, O_TYPE = 0, 1
N_TYPES = 14

# (inputs M, outputs N) of every type (Eq. 1a): the sources have no input; split gives
# two outputs (mid, side); merge and the sidechain compressor take two inputs (merge:
# mid, side; sidechain: main, key); every other processor, mix and output is 1 x 1.
PORTS = {t: (1, 1) for t in range(N_TYPES)}
PORTS.update({0: (0, 1), 10: (1, 2), 11: (2, 1), 12: (2, 1)})


class GraphError(ValueError):
    def __init__(self, code, msg):
        super().__init__(f"{code}: {msg}")
        self.code = code


def preds_succs(n, edges):
    preds = [[] for _ in range(n)]
    succs = [[] for _ in range(n)]
    for s, d in edges:
        preds[d].append(s)
        succs[s].append(d)
    return preds, succs


def validate(types, edges, n_types=N_TYPES, ports=None):
    """Reject what the paper's graph model does not allow (Sec. 2 Definitions).  With
    ``ports`` (one (k, l) per edge) an edge must leave an existing output k of its
    source and enter an existing input l of its destination."""
    n = len(types)
    if n == 0:
        raise GraphError("EINVAL", "empty graph")
    for t in types:
        if not (0 <= t < n_types):
            raise GraphError("ETYPE", f"unknown type {t}")
    for s, d in edges:
        if not (0 <= s < n and 0 <= d < n):
            raise GraphError("EINVAL", f"edge ({s},{d}) out of range")
    if ports is not None:
        if len(ports) != len(edges):
            raise GraphError("EINVAL", "one port pair per edge")
        for (s, d), (k, l) in zip(edges, ports):
            if not (0 <= k < PORTS[types[s]][1] and 0 <= l < PORTS[types[d]][0]):
                raise GraphError("EINVAL", f"edge ({s},{d}) ports ({k},{l}) out of range")
    preds, succs = preds_succs(n, edges)
    for v in range(n):
        if types[v] == I_TYPE and preds[v]:
            raise GraphError("EINVAL", f"input node {v} has in-edges")
        if types[v] != I_TYPE and not preds[v]:
            raise GraphError("EINVAL", f"node {v} has no input")
        if types[v] == O_TYPE and succs[v]:
            raise GraphError("EINVAL", f"output node {v} has out-edges")
    if not any(t == O_TYPE for t in types):
        raise GraphError("EINVAL", "graph has no output node")
    # Kahn's algorithm: every node must be reached
    indeg = [len(p) for p in preds]
    stack = [v for v in range(n) if indeg[v] == 0]
    seen = 0
    while stack:
        v = stack.pop()
        seen += 1
        for w in succs[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                stack.append(w)
    if seen != n:
        raise GraphError("ECYCLE", "graph has a cycle")


def _ready(types, preds, sched, t):
    return frozenset(v for v in range(len(types))
                     if types[v] == t and v not in sched and all(p in sched for p in preds[v]))


def _proc_types(types):
    return sorted(set(t for t in types if t not in (I_TYPE, O_TYPE)))


def _steps_from_string(types, edges, string):
    """Replay a type string into the node subsets V_0..V_N (maximal ready sets)."""
    preds, _ = preds_succs(len(types), edges)
    sched = frozenset(v for v, t in enumerate(types) if t == I_TYPE)
    steps = [sorted(sched)]
    for t in string[1:-1]:
        r = _ready(types, preds, sched, t)
        assert r, "type string does not replay"
        steps.append(sorted(r))
        sched = sched | r
    steps.append(sorted(v for v, t in enumerate(types) if t == O_TYPE))
    return steps


def beam_schedule(types, edges, width):
    """Beam search over partial schedules; width=None means no pruning (optimal)."""
    n = len(types)
    preds, _ = preds_succs(n, edges)
    non_out = frozenset(v for v in range(n) if types[v] != O_TYPE)
    start = frozenset(v for v in range(n) if types[v] == I_TYPE)
    if start >= non_out:
        return (I_TYPE, O_TYPE)
    ptypes = _proc_types(types)
    cands = [(start, (I_TYPE,))]
    while True:
        expanded = {}
        for sched, string in cands:
            for t in ptypes:
                r = _ready(types, preds, sched, t)
                if not r:
                    continue
                new, s2 = sched | r, string + (t,)
                old = expanded.get(new)
                if old is None or s2 < old:
                    expanded[new] = s2
        complete = [s for st, s in expanded.items() if st >= non_out]
        if complete:
            return min(complete) + (O_TYPE,)
        ranked = sorted(expanded.items(), key=lambda kv: (-len(kv[0]), kv[1]))
        cands = ranked if width is None else ranked[:width]


def greedy_schedule(types, edges):
    n = len(types)
    preds, _ = preds_succs(n, edges)
    non_out = frozenset(v for v in range(n) if types[v] != O_TYPE)
    sched = frozenset(v for v in range(n) if types[v] == I_TYPE)
    string = [I_TYPE]
    ptypes = _proc_types(types)
    while not sched >= non_out:
        best_t, best_r = None, frozenset()
        for t in ptypes:  # ascending id, strict '>' keeps the smallest id on ties
            r = _ready(types, preds, sched, t)
            if len(r) > len(best_r):
                best_t, best_r = t, r
        string.append(best_t)
        sched = sched | best_r
    return tuple(string) + (O_TYPE,)


def one_by_one_schedule(types, edges):
    """Returns (type string, steps) with one processing node per step."""
    n = len(types)
    preds, succs = preds_succs(n, edges)
    indeg = [len(p) for p in preds]
    inputs = [v for v in range(n) if types[v] == I_TYPE]
    outputs = [v for v in range(n) if types[v] == O_TYPE]
    heap = []
    for v in inputs:
        for w in succs[v]:
            indeg[w] -= 1
    for v in range(n):
        if types[v] not in (I_TYPE, O_TYPE) and indeg[v] == 0:
            heapq.heappush(heap, v)
    steps, string = [inputs], [I_TYPE]
    while heap:
        v = heapq.heappop(heap)
        steps.append([v])
        string.append(types[v])
        for w in succs[v]:
            indeg[w] -= 1
            if types[w] not in (I_TYPE, O_TYPE) and indeg[w] == 0:
                heapq.heappush(heap, w)
    steps.append(outputs)
    string.append(O_TYPE)
    return tuple(string), steps


def schedule(types, edges, method="beam", width=32):
    """Type string and node subsets [V_0, .., V_N] (original ids, ascending)."""
    validate(types, edges)
    if method == "one_by_one":
        return one_by_one_schedule(types, edges)
    if method == "greedy":
        s = greedy_schedule(types, edges)
    elif method == "beam":
        s = beam_schedule(types, edges, width)
    elif method == "optimal":
        s = beam_schedule(types, edges, None)
    else:
        raise ValueError(method)
    return s, _steps_from_string(types, edges, s)


def check_schedule(types, edges, steps):
    """Conditions (i)-(iii) of Sec. 2 plus V_0 = inputs and V_N = outputs."""
    n = len(types)
    flat = [v for st in steps for v in st]
    assert sorted(flat) == list(range(n)), "not a partition"
    where = {v: k for k, st in enumerate(steps) for v in st}
    for s, d in edges:
        assert where[s] < where[d], "not causal"
    for st in steps:
        assert len(set(types[v] for v in st)) == 1, "not homogeneous"
    assert sorted(steps[0]) == sorted(v for v in range(n) if types[v] == I_TYPE)
    assert sorted(steps[-1]) == sorted(v for v in range(n) if types[v] == O_TYPE)


def index_maps(types, edges, steps):
    """Algorithm 1 (OptimizeNodeOrder, Reorder, GetReadWriteIndex): sigma (original ->
    new id), the step ranges I^S (as ``step_ptr``), the in-edge CSR (I^G / I^A), the
    consumer CSR for the backward pass and the parameter row of each node (I^P, rows in
    original type order)."""
    n = len(types)
    order = [v for st in steps for v in sorted(st)]  # rank by (step, original id)
    sigma = [0] * n
    for new, old in enumerate(order):
        sigma[old] = new
    step_ptr = [0]
    for st in steps:
        step_ptr.append(step_ptr[-1] + len(st))
    new_edges = sorted((sigma[d], sigma[s]) for s, d in edges)  # by (dst, src)
    csr_ptr = [0] * (n + 1)
    for d, _ in new_edges:
        csr_ptr[d + 1] += 1
    for v in range(n):
        csr_ptr[v + 1] += csr_ptr[v]
    csr_src = [s for _, s in new_edges]
    t_edges = sorted((sigma[s], sigma[d]) for s, d in edges)  # by (src, dst)
    tcsr_ptr = [0] * (n + 1)
    for s, _ in t_edges:
        tcsr_ptr[s + 1] += 1
    for v in range(n):
        tcsr_ptr[v + 1] += tcsr_ptr[v]
    tcsr_dst = [d for _, d in t_edges]
    counters = {}
    row_of_orig = [0] * n
    for v in range(n):
        row_of_orig[v] = counters.get(types[v], 0)
        counters[types[v]] = row_of_orig[v] + 1
    param_row = [0] * n
    new_types = [0] * n
    for old in range(n):
        param_row[sigma[old]] = row_of_orig[old]
        new_types[sigma[old]] = types[old]
    return dict(sigma=sigma, step_ptr=step_ptr, csr_ptr=csr_ptr, csr_src=csr_src,
                tcsr_ptr=tcsr_ptr, tcsr_dst=tcsr_dst, param_row=param_row, types=new_types)


def union(graphs):
    """Graph-level parallelism (Sec. 2): a batch of graphs is one disconnected graph.
    Returns (types, edges, node offset of each graph)."""
    types, edges, offs = [], [], []
    for g in graphs:
        off = len(types)
        offs.append(off)
        types.extend(g.types)
        edges.extend((s + off, d + off) for s, d in g.edges)
    return types, edges, offs
