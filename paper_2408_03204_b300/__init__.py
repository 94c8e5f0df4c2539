"""Python binding of libgrafx (include/grafx.h): argument marshalling only.

Every step of the render, its backward pass and the loss runs in the library's
CUDA kernels; this module turns torch tensors into raw pointers and streams, and
wraps the calls in ``torch.autograd.Function``s.  It fails loudly if the compiled
library is missing: there is no CPU fallback.

    g = Graph(); i = g.add(T_IN); a, b = g.add_serial_chain([T_GAIN, T_EQ]); ...
    plan = Plan([g], [L])                         # compute_render_data (Algorithm 1)
    plan.bind_workspace()                         # torch.empty on the current device
    out = render(plan, sources, {T_GAIN: pg, T_EQ: pe})   # differentiable
    loss = mrstft_loss(plan, out, target)
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GRAFX_VARIANT=precise selects the measurement build of build.py (libgrafx_precise.so)
LIB_PATH = os.path.join(HERE, "libgrafx_precise.so" if os.environ.get("GRAFX_VARIANT") == "precise"
                        else "libgrafx.so")

T_IN, T_OUT, T_MIX, T_GAIN, T_IMAGER, T_EQ, T_COMP, T_DELAY, T_REVERB, T_GATE = range(10)
T_SPLIT, T_MERGE, T_SIDECHAIN = 10, 11, 12   # multi-port processors (inputs x outputs: 1x2, 2x1, 2x1)
T_BALLISTIC = 13                              # compressor with attack/release ballistics
N_TYPES = 14
PARAM_COLS = {T_GAIN: 2, T_IMAGER: 1, T_EQ: 8, T_COMP: 4, T_DELAY: 176, T_REVERB: 50, T_GATE: 4, T_SIDECHAIN: 4,
              T_BALLISTIC: 5}
# processor layouts (grafx_plan_opts): "compact" (the widths above) or "paper" (Sec. 3)
EQ_PARAMS = {"bands": 0, "logmag": 1}
DELAY_LAYOUT = {"compact": 0, "slots": 1}
REVERB_LAYOUT = {"compact": 0, "paper": 1}
PRESETS = {"compact": dict(eq_taps=1023, eq_params="bands", delay_layout="compact", reverb_layout="compact"),
           "paper": dict(eq_taps=2047, eq_params="logmag", delay_layout="slots", reverb_layout="paper")}
SCHED = {"beam": 0, "greedy": 1, "optimal": 2, "one_by_one": 3}
ERRORS = {1: "EINVAL", 2: "ECYCLE", 3: "ESHAPE", 4: "ETYPE", 5: "ENOMEM", 6: "ECUDA", 7: "ETIMEOUT",
          8: "ESTATE"}


class GrafxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class PlanOpts(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("beam_width", ctypes.c_int32), ("eq_taps", ctypes.c_int32),
                ("sample_rate", ctypes.c_int32), ("n_threads", ctypes.c_int32), ("eq_fft", ctypes.c_int32),
                ("comp_chunk", ctypes.c_int32), ("checkpoint_steps", ctypes.c_int32),
                ("eq_params", ctypes.c_int32), ("delay_layout", ctypes.c_int32), ("reverb_layout", ctypes.c_int32),
                ("source_batch", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("n_steps", ctypes.c_int32), ("n_inputs", ctypes.c_int32), ("n_outputs", ctypes.c_int32),
                ("n_type_rows", ctypes.c_int32 * N_TYPES), ("src_elems", ctypes.c_int64),
                ("out_elems", ctypes.c_int64), ("node_samples", ctypes.c_int64), ("ws_bytes", ctypes.c_size_t),
                ("eq_fft", ctypes.c_int32), ("comp_chunk", ctypes.c_int32),
                ("param_cols", ctypes.c_int32 * N_TYPES), ("source_batch", ctypes.c_int32),
                ("fused_pairs", ctypes.c_int32)]


_lib = None
# name -> (restype, argtypes); mirrors include/grafx.h
_P, _I32, _I64, _SZ, _F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "grafx_last_error": (ctypes.c_char_p, []),
    "grafx_pitch": (_I64, [_I64]),
    "grafx_graph_create": (ctypes.c_int, [ctypes.POINTER(_P)]),
    "grafx_graph_destroy": (ctypes.c_int, [_P]),
    "grafx_graph_add": (ctypes.c_int, [_P, _I32, _I32P]),
    "grafx_graph_add_serial_chain": (ctypes.c_int, [_P, _I32P, _I32, _I32P, _I32P]),
    "grafx_graph_connect": (ctypes.c_int, [_P, _I32, _I32]),
    "grafx_graph_connect_ports": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32]),
    "grafx_type_ports": (ctypes.c_int, [_I32, _I32P, _I32P]),
    "grafx_graph_size": (ctypes.c_int, [_P, _I32P, _I32P]),
    "grafx_plan_opts_default": (None, [ctypes.POINTER(PlanOpts)]),
    "grafx_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_I64),
                                         ctypes.POINTER(PlanOpts), ctypes.POINTER(_P)]),
    "grafx_plan_destroy": (ctypes.c_int, [_P]),
    "grafx_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(PlanInfo)]),
    "grafx_plan_export": (ctypes.c_int, [_P] + [_I32P] * 8),
    "grafx_plan_step_items": (ctypes.c_int, [_P, _I32, _I32, _I32P, _I32, _I32P]),
    "grafx_plan_bind_workspace": (ctypes.c_int, [_P, _P, _SZ, _P]),
    "grafx_bind_params": (ctypes.c_int, [_P, _I32, _F, _I64, _I64]),
    "grafx_bind_reverb_noise": (ctypes.c_int, [_P, _F, _I64]),
    "grafx_render": (ctypes.c_int, [_P, _F, _F, _P]),
    "grafx_backprop": (ctypes.c_int, [_P, _F, _F, ctypes.POINTER(_P), _F, _P]),
    "grafx_render_steps": (ctypes.c_int, [_P, _F, _F, _I32, _I32, _P]),
    "grafx_backprop_steps": (ctypes.c_int, [_P, _F, _F, ctypes.POINTER(_P), _F, _I32, _I32, _P]),
    "grafx_mrstft_forward": (ctypes.c_int, [_P, _F, _F, _F, _P]),
    "grafx_mrstft_backward": (ctypes.c_int, [_P, _F, _F, _F, _P]),
    "grafx_sync_status": (ctypes.c_int, [_P, _P]),
    "grafx_last_launch_count": (ctypes.c_int, [_P, _I32P]),
    "grafx_compressor_forward_noalloc": (ctypes.c_int, [_F, _I64, _I64, _F, _F, _P, _P]),
    "grafx_adam_step": (ctypes.c_int, [_F, _F, _F, _F, _F, _P, _I32, _I64, _I32, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, _P]),
    "grafx_params_to_theta": (ctypes.c_int, [_F, _P, _I32, _I64, _F, _P]),
    "grafx_adam_step_dev": (ctypes.c_int, [_F, _F, _F, _F, _F, _P, _I32, _I64, _P, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_float, _P]),
    "grafx_step_graph_create": (ctypes.c_int, [_P, _F, _F, _F, _F, _F, ctypes.POINTER(_P), _F, _P,
                                               ctypes.POINTER(_P)]),
    "grafx_step_graph_launch": (ctypes.c_int, [_P, _P]),
    "grafx_step_graph_launches": (ctypes.c_int, [_P, _I32P]),
    "grafx_step_graph_destroy": (ctypes.c_int, [_P]),
    "grafx_node_inputs": (ctypes.c_int, [_P, _F, _F, _I32P, _I32, _F, _I64, _P]),
    "grafx_selftest_bounded_wait": (ctypes.c_int, [_P, _P, _I32, _F, _P]),
    "grafx_ws_create": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_P)]),
    "grafx_ws_destroy": (ctypes.c_int, [_P]),
    "grafx_ws_param_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "grafx_ws_workspace_bytes": (ctypes.c_int, [_P, _I32, _I64, ctypes.POINTER(_SZ)]),
    "grafx_ws_bind": (ctypes.c_int, [_P, _P, _SZ, _P]),
    "grafx_ws_logmel": (ctypes.c_int, [_P, _F, _I32, _I64, _I64, _I64, _P, _I32, _I32, _F, _P]),
    "grafx_ws_standardise": (ctypes.c_int, [_F, _F, _F, _F, _F, _I32, _I32, _I32, _F, _P]),
    "grafx_ws_xgain": (ctypes.c_int, [_P, _F, _I32, _I64, _F, _I32, _I64, _F, _I64, _I64, _I32, _F, _P]),
    "grafx_ws_forward": (ctypes.c_int, [_P, _F, _F, _I32P, _I32, _F, _P]),
    "grafx_ws_backward": (ctypes.c_int, [_P, _F, _F, _I32P, _I32, _F, _F, _P]),
    "grafx_ws_mse": (ctypes.c_int, [_F, _F, _P, _I32, _F, _F, _P]),
    "grafx_ws_sync_status": (ctypes.c_int, [_P, _P]),
    "grafx_gemm_bf16": (ctypes.c_int, [_I32, _I32, _I32, _F, _I64, _I64, _F, _I64, _I64, _F, _I64, ctypes.c_float,
                                       ctypes.c_float, _F, _I64, _P]),
}


def lib():
    """Load libgrafx.so (build it first with ``python -m paper_2408_03204_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); "
                               "run python -m paper_2408_03204_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise GrafxError(rc, lib().grafx_last_error().decode())


def pitch(L):
    return int(lib().grafx_pitch(int(L)))


class Graph:
    """Mutable graph (Sec. 2 "Graph representations"; Fig. 2a builder calls)."""

    def __init__(self):
        h = _P()
        _check(lib().grafx_graph_create(ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.grafx_graph_destroy(self._h)
            self._h = None

    def add(self, t):
        i = ctypes.c_int32()
        _check(lib().grafx_graph_add(self._h, int(t), ctypes.byref(i)))
        return i.value

    def add_serial_chain(self, types):
        arr = (ctypes.c_int32 * len(types))(*[int(t) for t in types])
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().grafx_graph_add_serial_chain(self._h, arr, len(types), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def connect(self, src, dst, out_port=0, in_port=0):
        """Edge from output ``out_port`` of src to input ``in_port`` of dst (T_E)."""
        if out_port or in_port:
            _check(lib().grafx_graph_connect_ports(self._h, int(src), int(dst), int(out_port), int(in_port)))
        else:
            _check(lib().grafx_graph_connect(self._h, int(src), int(dst)))

    @classmethod
    def from_lists(cls, types, edges, ports=None):
        g = cls()
        for t in types:
            g.add(t)
        for e, (s, d) in enumerate(edges):
            k, l = ports[e] if ports is not None else (0, 0)
            g.connect(s, d, k, l)
        return g


def type_ports(t):
    """(inputs, outputs) of node type t (Eq. 1a)."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().grafx_type_ports(int(t), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _stream_of(s):
    """ctypes handle of a torch.cuda.Stream."""
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Render data of one graph or a batch of graphs (Algorithm 1: ScheduleBatchedProcessing,
    OptimizeNodeOrder, Reorder, GetReadWriteIndex)."""

    def __init__(self, graphs, lengths, schedule="beam", beam_width=32, eq_taps=None, sample_rate=44100,
                 n_threads=0, eq_fft=0, comp_chunk=0, checkpoint_steps=0, preset="compact", eq_params=None,
                 delay_layout=None, reverb_layout=None, source_batch=1):
        """preset "compact" (8 EQ bands, 4-tap delays, 1024/256 reverb with 12 bands) or
        "paper" (Sec. 3: 2047-tap EQ by its 1024 log-magnitudes, 20 delay taps in 100 ms
        slots, 384/192 reverb with 192 log-magnitudes per filter); the keyword
        arguments override single settings of the preset.  source_batch B > 1 renders
        the graphs on B source sets with shared parameters: sources and outputs are
        [B][rows of one pass], gradients are summed over the copies."""
        pre = PRESETS[preset]
        o = PlanOpts()
        lib().grafx_plan_opts_default(ctypes.byref(o))
        o.schedule, o.beam_width = SCHED[schedule], beam_width
        o.eq_taps = pre["eq_taps"] if eq_taps is None else eq_taps
        o.sample_rate, o.n_threads, o.eq_fft, o.comp_chunk = sample_rate, n_threads, eq_fft, comp_chunk
        o.checkpoint_steps = checkpoint_steps
        o.eq_params = EQ_PARAMS[eq_params or pre["eq_params"]]
        o.delay_layout = DELAY_LAYOUT[delay_layout or pre["delay_layout"]]
        o.reverb_layout = REVERB_LAYOUT[reverb_layout or pre["reverb_layout"]]
        o.source_batch = int(source_batch)
        hs = (_P * len(graphs))(*[g._h for g in graphs])
        ls = (ctypes.c_int64 * len(lengths))(*[int(x) for x in lengths])
        h = _P()
        _check(lib().grafx_plan_create(hs, len(graphs), ls, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.lengths = [int(x) for x in lengths]
        self.sample_rate = int(sample_rate)
        inf = PlanInfo()
        _check(lib().grafx_plan_info(self._h, ctypes.byref(inf)))
        self.info = inf
        # columns of P[t] under this plan's layouts
        self.param_cols = {t: int(inf.param_cols[t]) for t in range(N_TYPES) if inf.param_cols[t] > 0}
        self.ws = None
        self.params = {}
        # Workspace generations: bumped by every call that rewrites the rows a backprop
        # reads (a render, a parameter binding) or the spectra a loss gradient reads (a
        # loss forward), so the autograd functions can tell whether their forward's state
        # is still the plan's.
        self.render_gen = 0
        self.loss_gen = 0

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.grafx_plan_destroy(self._h)
            self._h = None

    # ---- host-side render data
    def export(self):
        import numpy as np
        inf = self.info
        n, e, N = inf.n_nodes, inf.n_edges, inf.n_steps
        arrs = dict(type_string=np.zeros(N + 1, np.int32), step_ptr=np.zeros(N + 2, np.int32),
                    sigma=np.zeros(n, np.int32), csr_ptr=np.zeros(n + 1, np.int32),
                    csr_src=np.zeros(max(e, 1), np.int32), tcsr_ptr=np.zeros(n + 1, np.int32),
                    tcsr_dst=np.zeros(max(e, 1), np.int32), param_row=np.zeros(n, np.int32))
        ptrs = [a.ctypes.data_as(_I32P) for a in arrs.values()]
        _check(lib().grafx_plan_export(self._h, *ptrs))
        arrs["csr_src"] = arrs["csr_src"][:e]
        arrs["tcsr_dst"] = arrs["tcsr_dst"][:e]
        return {k: v.tolist() for k, v in arrs.items()}

    def step_items(self, step, backward=False):
        """The work items of schedule step `step` (1..N), forward or backward, as an
        [n, 4] int32 array in launch order (grafx_plan_step_items)."""
        import numpy as np
        n = ctypes.c_int32(0)
        _check(lib().grafx_plan_step_items(self._h, int(step), int(bool(backward)), None, 0, ctypes.byref(n)))
        a = np.zeros((max(n.value, 1), 4), np.int32)
        _check(lib().grafx_plan_step_items(self._h, int(step), int(bool(backward)), a.ctypes.data_as(_I32P),
                                           n.value, ctypes.byref(n)))
        return a[:n.value]

    # ---- device binding (torch supplies memory and streams only)
    def bind_workspace(self, device="cuda"):
        import torch
        nbytes = int(self.info.ws_bytes)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-ws.data_ptr()) % 256
        self.ws = ws
        self._ws_ptr = ws.data_ptr() + off
        _check(lib().grafx_plan_bind_workspace(self._h, ctypes.c_void_p(self._ws_ptr), nbytes,
                                               _stream(torch, ws.device)))
        return self

    def bind_params(self, params):
        for t, p in params.items():
            assert p.dtype.is_floating_point and p.is_contiguous()
            _check(lib().grafx_bind_params(self._h, int(t), _ptr(p), p.shape[0], p.shape[1]))
            self.params[int(t)] = p
        self.render_gen += 1

    def bind_reverb_noise(self, noise):
        """noise: device float32 [2, 88200] (mid, side), kept by reference."""
        _check(lib().grafx_bind_reverb_noise(self._h, _ptr(noise), noise.numel()))
        self.rv_noise = noise

    def render_raw(self, sources, out, stream):
        self.render_gen += 1
        _check(lib().grafx_render(self._h, _ptr(sources), _ptr(out), stream))

    def backprop_raw(self, sources, d_out, d_params, d_sources, stream):
        arr = (_P * N_TYPES)(*[_ptr(d_params.get(t)) for t in range(N_TYPES)])
        _check(lib().grafx_backprop(self._h, _ptr(sources), _ptr(d_out), arr, _ptr(d_sources), stream))

    def render_steps_raw(self, sources, out, first, last, stream):
        self.render_gen += 1
        _check(lib().grafx_render_steps(self._h, _ptr(sources), _ptr(out), int(first), int(last), stream))

    def backprop_steps_raw(self, sources, d_out, d_params, d_sources, first, last, stream):
        arr = (_P * N_TYPES)(*[_ptr(d_params.get(t)) for t in range(N_TYPES)])
        _check(lib().grafx_backprop_steps(self._h, _ptr(sources), _ptr(d_out), arr, _ptr(d_sources),
                                          int(first), int(last), stream))

    def loss_raw(self, out, target, loss, stream):
        self.loss_gen += 1
        _check(lib().grafx_mrstft_forward(self._h, _ptr(out), _ptr(target), _ptr(loss), stream))

    def loss_backward_raw(self, out, target, d_out, stream):
        _check(lib().grafx_mrstft_backward(self._h, _ptr(out), _ptr(target), _ptr(d_out), stream))

    def node_inputs_raw(self, sources, out, ids, dst, dst_pitch, stream):
        """u_v of the nodes ``ids`` (union numbering) into dst [n][2][dst_pitch] after a render."""
        arr = (ctypes.c_int32 * max(len(ids), 1))(*[int(i) for i in ids])
        _check(lib().grafx_node_inputs(self._h, _ptr(sources), _ptr(out), arr, len(ids), _ptr(dst),
                                       int(dst_pitch), stream))

    def capture_step(self, sources, out, target, loss, d_out, d_params, d_sources, stream):
        """Record render + loss + loss gradient + backprop with these buffers as one CUDA
        graph; returns a StepGraph whose launch() replays it."""
        arr = (_P * N_TYPES)(*[_ptr(d_params.get(t)) for t in range(N_TYPES)])
        h = _P()
        _check(lib().grafx_step_graph_create(self._h, _ptr(sources), _ptr(out), _ptr(target), _ptr(loss),
                                             _ptr(d_out), arr, _ptr(d_sources), stream, ctypes.byref(h)))
        return StepGraph(h, (sources, out, target, loss, d_out, d_params, d_sources), self)

    def sync_status(self, stream=None):
        import torch
        s = stream if stream is not None else _stream(torch, self.ws.device)
        _check(lib().grafx_sync_status(self._h, s))

    def last_launches(self):
        n = ctypes.c_int32()
        _check(lib().grafx_last_launch_count(self._h, ctypes.byref(n)))
        return n.value


WS_HEAD_TYPES = (T_GAIN, T_IMAGER, T_EQ, T_COMP, T_DELAY, T_REVERB)
WS_HEAD_OUT = (2, 1, 8, 4, 176, 50)
WS_OUTMAX = 176
WS_T = 32


class WarmStartNet:
    """Handle of the warm-start network (grafx_ws_*): host tables plus a device workspace
    sized for ``max_batch`` samples and ``max_rows`` log-mel rows of ``max_len`` samples.
    Weights and gradients are caller tensors (flat float32, ``n_params``)."""

    def __init__(self, max_batch, max_rows, max_len, sample_rate=44100, device="cuda"):
        import torch
        h = _P()
        _check(lib().grafx_ws_create(int(max_batch), int(sample_rate), ctypes.byref(h)))
        self._h = h
        c = ctypes.c_int64()
        _check(lib().grafx_ws_param_count(self._h, ctypes.byref(c)))
        self.n_params = c.value
        self.max_batch = int(max_batch)
        nb = ctypes.c_size_t()
        _check(lib().grafx_ws_workspace_bytes(self._h, int(max_rows), int(max_len), ctypes.byref(nb)))
        ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=device)
        off = (-ws.data_ptr()) % 256
        self.ws = ws
        _check(lib().grafx_ws_bind(self._h, ctypes.c_void_p(ws.data_ptr() + off), nb.value,
                                   _stream(torch, ws.device)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.grafx_ws_destroy(self._h)
            self._h = None

    def logmel_raw(self, rows, n_rows, row_stride, pitch, length, row_of_sample, n_samples, coff, feats, stream):
        _check(lib().grafx_ws_logmel(self._h, _ptr(rows), int(n_rows), int(row_stride), int(pitch), int(length),
                                     _ptr(row_of_sample), int(n_samples), int(coff), _ptr(feats), stream))

    def xgain_raw(self, u_rows, n_samples, u_stride, t_rows, n_trows, t_stride, row_of_sample, pitch, length, coff,
                  feats, stream):
        _check(lib().grafx_ws_xgain(self._h, _ptr(u_rows), int(n_samples), int(u_stride), _ptr(t_rows), int(n_trows),
                                    int(t_stride), _ptr(row_of_sample), int(pitch), int(length), int(coff),
                                    _ptr(feats), stream))

    @staticmethod
    def _heads(head_count):
        return (ctypes.c_int32 * 6)(*[int(x) for x in head_count])

    def forward_raw(self, weights, feats, head_count, out, stream):
        B = int(sum(head_count))
        _check(lib().grafx_ws_forward(self._h, _ptr(weights), _ptr(feats), self._heads(head_count), B, _ptr(out),
                                      stream))

    def backward_raw(self, weights, feats, head_count, d_out, d_weights, stream):
        B = int(sum(head_count))
        _check(lib().grafx_ws_backward(self._h, _ptr(weights), _ptr(feats), self._heads(head_count), B,
                                       _ptr(d_out), _ptr(d_weights), stream))

    def sync_status(self, stream):
        _check(lib().grafx_ws_sync_status(self._h, stream))

    @staticmethod
    def mse_raw(out, target, n_out, loss, d_out, stream):
        _check(lib().grafx_ws_mse(_ptr(out), _ptr(target), _ptr(n_out), out.shape[0], _ptr(loss), _ptr(d_out),
                                  stream))


def gemm_bf16_raw(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta, stream, scratch=None):
    _check(lib().grafx_gemm_bf16(int(M), int(N), int(K), _ptr(A), int(sam), int(sak), _ptr(B), int(sbk), int(sbn),
                                 _ptr(C), int(ldc), float(alpha), float(beta), _ptr(scratch),
                                 0 if scratch is None else scratch.numel(), stream))


class StepGraph:
    """A captured fit step (grafx_step_graph_*); keeps its buffers alive."""

    def __init__(self, h, keep, plan=None):
        self._h, self._keep, self._plan = h, keep, plan

    def launch(self, stream):
        if self._plan is not None:          # the step renders and evaluates the loss
            self._plan.render_gen += 1
            self._plan.loss_gen += 1
        _check(lib().grafx_step_graph_launch(self._h, stream))

    def launches(self):
        n = ctypes.c_int32()
        _check(lib().grafx_step_graph_launches(self._h, ctypes.byref(n)))
        return n.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.grafx_step_graph_destroy(self._h)
            self._h = None


def _autograd():
    import torch

    class _Render(torch.autograd.Function):
        @staticmethod
        def forward(ctx, plan, types, sources, *ps):
            plan.bind_params(dict(zip(types, ps)))
            out = torch.empty(plan.info.out_elems, dtype=torch.float32, device=sources.device)
            plan.render_raw(sources, out, _stream(torch, sources.device))
            ctx.plan, ctx.types, ctx.gen = plan, types, plan.render_gen
            ctx.save_for_backward(sources, *ps)
            return out

        @staticmethod
        def backward(ctx, d_out):
            plan, types = ctx.plan, ctx.types
            sources, *ps = ctx.saved_tensors
            if plan.render_gen != ctx.gen:
                # The plan rendered or re-bound parameters since this forward: its rows
                # belong to another render.  Restore this forward's state first.
                plan.bind_params(dict(zip(types, ps)))
                scratch = torch.empty(plan.info.out_elems, dtype=torch.float32, device=sources.device)
                plan.render_raw(sources, scratch, _stream(torch, sources.device))
            d_out = d_out.contiguous()
            dps = {t: torch.empty_like(p) for t, p in zip(types, ps)}
            d_src = torch.empty_like(sources) if ctx.needs_input_grad[2] else None
            plan.backprop_raw(sources, d_out, dps, d_src, _stream(torch, sources.device))
            return (None, None, d_src) + tuple(dps[t] for t in types)

    class _Loss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, plan, out, target):
            loss = torch.empty(1, dtype=torch.float32, device=out.device)
            plan.loss_raw(out, target, loss, _stream(torch, out.device))
            ctx.plan, ctx.gen = plan, plan.loss_gen
            ctx.save_for_backward(out, target)
            return loss[0]

        @staticmethod
        def backward(ctx, g):
            out, target = ctx.saved_tensors
            if ctx.plan.loss_gen != ctx.gen:
                # another loss forward replaced the cached spectra: recompute this one's
                scratch = torch.empty(1, dtype=torch.float32, device=out.device)
                ctx.plan.loss_raw(out, target, scratch, _stream(torch, out.device))
            d_out = torch.empty_like(out)
            ctx.plan.loss_backward_raw(out, target, d_out, _stream(torch, out.device))
            return None, d_out * g, None

    return _Render, _Loss


_FN = None


def _fns():
    global _FN
    if _FN is None:
        _FN = _autograd()
    return _FN


def render(plan, sources, params):
    """Differentiable render: ``sources`` flat float32 (src_elems), ``params`` {type: [rows, cols]}.
    Returns the flat output buffer (out_elems floats)."""
    types = tuple(sorted(params))
    return _fns()[0].apply(plan, types, sources, *[params[t] for t in types])


def mrstft_loss(plan, out, target):
    """Differentiable multi-resolution STFT loss over the plan's output rows."""
    return _fns()[1].apply(plan, out, target)
