// C ABI (include/grafx.h): graph building, planning, device binding, and the step
// loops of Algorithm 1 (render) and its reverse (backprop), plus the loss.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "plan.h"

using namespace grafx;

namespace {

#define GX_TRY try {
#define GX_CATCH                                                              \
  }                                                                           \
  catch (const std::bad_alloc&) { return fail(GRAFX_ENOMEM, "host allocation failed"); } \
  catch (...) { return fail(GRAFX_EINVAL, "unexpected exception"); }

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GRAFX_OK;
  return fail(GRAFX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
T* at(const Plan* p, size_t off) { return reinterpret_cast<T*>(p->dev_ws + off); }

DevCtx make_ctx(const Plan* p, const float* src, float* out, const float* d_out, float* d_src) {
  DevCtx c;
  std::memset(&c, 0, sizeof(c));
  c.nodes = at<const NodeDev>(p, p->ws.nodes);
  c.ext = at<const int4_>(p, p->ws.node_ext);
  c.csr_ptr = at<const int32_t>(p, p->ws.csr_ptr);
  c.csr_src = at<const int32_t>(p, p->ws.csr_src);
  c.tcsr_ptr = at<const int32_t>(p, p->ws.tcsr_ptr);
  c.tcsr_dst = at<const int32_t>(p, p->ws.tcsr_dst);
  c.items = at<const int4_>(p, p->ws.items);
  c.csr_row = at<const int64_t>(p, p->ws.csr_row);
  c.tcsr_row = at<const int64_t>(p, p->ws.tcsr_row);
  c.in1_begin = at<const int32_t>(p, p->ws.in1_begin);
  c.out1_begin = at<const int32_t>(p, p->ws.out1_begin);
  c.tw = at<const float2_>(p, p->ws.twiddle);
  c.ptw = at<const float2_>(p, p->ws.ptw);
  c.eq_cos = at<const float>(p, p->ws.eq_cos);
  c.eq_hann = at<const float>(p, p->ws.eq_hann);
  c.eq_band = at<const float>(p, p->ws.eq_band);
  c.status = at<uint32_t>(p, p->ws.status);
  c.tickets = at<int32_t>(p, p->ws.tickets);
  c.flags = at<unsigned long long>(p, p->ws.flags);
  c.eq_spec = at<float>(p, p->ws.eq_spec);
  c.eq_aux = at<float>(p, p->ws.eq_aux);
  c.eq_bandpart = at<float>(p, p->ws.eq_bandpart);
  c.comp_carry = at<float>(p, p->ws.comp_carry);
  c.dl_aux = at<float>(p, p->ws.dl_aux);
  c.dl_spec = at<float2>(p, p->ws.dl_spec);
  c.dl_R = at<float2>(p, p->ws.dl_R);
  c.dl_r = at<float>(p, p->ws.dl_r);
  for (int j = 0; j < 9; ++j) c.dl_taylor[j] = float(p->dl_taylor[j]);
  c.rv_noise = p->rv_noise;
  c.rv_band = at<const float>(p, p->ws.rv_band);
  c.rv_win = at<const float>(p, p->ws.rv_win);
  c.rv_cs = at<const float2_>(p, p->ws.rv_cs);
  c.rv_U = at<float2>(p, p->ws.rv_U);
  c.rv_fr = at<float2>(p, p->ws.rv_fr);
  c.rv_h = at<float>(p, p->ws.rv_h);
  c.rv_H = at<float2>(p, p->ws.rv_H);
  c.rv_Y = at<float2>(p, p->ws.rv_Y);
  c.rv_R = at<float2>(p, p->ws.rv_R);
  c.rv_r = at<float>(p, p->ws.rv_r);
  c.rv_mm = at<float2>(p, p->ws.rv_mm);
  c.rv_lm = at<float>(p, p->ws.rv_lm);
  c.rv_dot = at<float>(p, p->ws.rv_dot);
  c.rv_nbmax = p->rv_nbmax;
  c.bal = at<float>(p, p->ws.bal);
  c.bal_maxlen = int32_t(p->L.empty() ? 0 : *std::max_element(p->L.begin(), p->L.end()));
  c.partial = at<float4>(p, p->ws.partial);
  c.eq_partial = at<float2>(p, p->ws.eq_partial);
  c.eq_uspec = at<float2>(p, p->ws.eq_uspec);
  c.eq_ola = at<float>(p, p->ws.eq_ola);
  c.ybase[KIND_INPUT] = const_cast<float*>(src);
  c.ybase[KIND_OUTPUT] = out;
  c.ybase[KIND_INTERNAL] = at<float>(p, p->ws.U);
  c.abase[KIND_INPUT] = d_src;
  c.abase[KIND_OUTPUT] = const_cast<float*>(d_out);
  c.abase[KIND_INTERNAL] = at<float>(p, p->ws.A);
  c.eq_taps = p->eq_taps;
  c.eq_H = p->eq_H;
  c.eq_Hal = (p->eq_H + 3) & ~3;
  c.eq_fft = p->eq_fft;
  c.eq_step = p->eq_step;
  c.comp_chunk = p->comp_chunk;
  c.sample_rate = float(p->opts.sample_rate);
  c.eq_logmag = p->eq_logmag;
  c.dl_taps = p->dl_taps;
  c.dl_nd = p->dl_nd;
  c.dl_slot = p->dl_slot;
  c.dl_P = p->dl_P;
  c.dl_nbmax = p->dl_nbmax;
  c.rv_paper = p->rv_paper;
  c.rv_n = p->rv_n;
  c.rv_hop = p->rv_hop;
  c.rv_f = p->rv_f;
  return c;
}

int check_ready(const Plan* p) {
  if (!p->dev_ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_plan_bind_workspace)");
  for (int t : {GRAFX_T_GAIN, GRAFX_T_IMAGER, GRAFX_T_EQ, GRAFX_T_COMP, GRAFX_T_DELAY, GRAFX_T_REVERB, GRAFX_T_GATE,
                GRAFX_T_SIDECHAIN, GRAFX_T_BALLISTIC})
    if (p->n_type_rows[t] > 0 && !p->params[t])
      return fail(GRAFX_ESTATE, "parameters of type " + std::to_string(t) + " not bound");
  if (p->n_type_rows[GRAFX_T_REVERB] > 0 && !p->rv_noise)
    return fail(GRAFX_ESTATE, "reverb noise not bound (grafx_bind_reverb_noise)");
  return GRAFX_OK;
}

int param_cols(const Plan* p, int t) { return t >= 0 && t < GRAFX_N_TYPES ? p->pcols[t] : 0; }


LossLaunch make_loss(const Plan* p, const float* y, const float* tgt) {
  LossLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.rows = at<const LossRow>(p, p->ws.loss_rows);
  L.items = at<const int4_>(p, p->ws.loss_items);
  L.n_items = int(p->loss.items.size());
  L.row_loss = at<float>(p, p->ws.loss_rowloss);
  L.y = y;
  L.tgt = tgt;
  L.part = at<float4>(p, p->ws.loss_part);
  L.stats = at<float4>(p, p->ws.loss_stats);
  L.frames = at<float>(p, p->ws.loss_frames);
  L.spec = at<float2>(p, p->ws.loss_spec);
  L.tw = at<const float2_>(p, p->ws.twiddle);
  L.ptw = at<const float2_>(p, p->ws.ptw);
  L.n_rows = int(p->loss.rows.size());
  for (auto& r : p->loss.rows) L.max_pitch = std::max(L.max_pitch, r.pitch);
  return L;
}

// Kernel attributes and launch shapes (dynamic shared-memory limits, resident CTAs per
// SM), set once per process by each launcher's first call.  Done when a workspace is
// bound and again before a capture, so that a render captured by the caller's own graph
// (e.g. a framework's CUDA graph over a whole fit step) never makes those calls inside
// its capture.
void init_launchers(const Plan* p, cudaStream_t s) {
  const DevCtx c0 = make_ctx(p, nullptr, nullptr, nullptr, nullptr);
  launch_eq(-1, c0, 0, 0, s);
  launch_comp(-1, c0, 0, 0, 0, 0, 0, 0, s);
  launch_delay(-1, c0, 0, 0, s);
  launch_reverb(-1, c0, 0, 0, s);
  launch_loss(-1, make_loss(p, nullptr, nullptr), s);
}

}  // namespace

extern "C" {

const char* grafx_last_error(void) { return last_error_cstr(); }

int64_t grafx_pitch(int64_t L) { return pitch_of(L); }

int grafx_graph_create(grafx_graph** out) {
  GX_TRY
  if (!out) return fail(GRAFX_EINVAL, "null output pointer");
  *out = new grafx_graph();
  return GRAFX_OK;
  GX_CATCH
}

int grafx_graph_destroy(grafx_graph* g) {
  delete g;
  return GRAFX_OK;
}

int grafx_graph_add(grafx_graph* g, int32_t type, int32_t* id_out) {
  GX_TRY
  if (!g) return fail(GRAFX_EINVAL, "null graph");
  if (type < 0 || type >= GRAFX_N_TYPES) return fail(GRAFX_ETYPE, "unknown node type");
  g->types.push_back(type);
  if (id_out) *id_out = int32_t(g->types.size()) - 1;
  return GRAFX_OK;
  GX_CATCH
}

int grafx_graph_add_serial_chain(grafx_graph* g, const int32_t* types, int32_t n, int32_t* first_id,
                                 int32_t* last_id) {
  GX_TRY
  if (!g || !types || n < 1) return fail(GRAFX_EINVAL, "bad chain");
  for (int32_t i = 0; i < n; ++i)
    if (types[i] < 0 || types[i] >= GRAFX_N_TYPES) return fail(GRAFX_ETYPE, "unknown node type");
  int32_t first = int32_t(g->types.size());
  for (int32_t i = 0; i < n; ++i) {
    g->types.push_back(types[i]);
    if (i) {
      g->edges.push_back({first + i - 1, first + i});
      g->ports.push_back({0, 0});
    }
  }
  if (first_id) *first_id = first;
  if (last_id) *last_id = first + n - 1;
  return GRAFX_OK;
  GX_CATCH
}

int grafx_graph_connect(grafx_graph* g, int32_t src, int32_t dst) {
  return grafx_graph_connect_ports(g, src, dst, 0, 0);
}

int grafx_graph_connect_ports(grafx_graph* g, int32_t src, int32_t dst, int32_t src_port, int32_t dst_port) {
  GX_TRY
  if (!g) return fail(GRAFX_EINVAL, "null graph");
  const int32_t n = int32_t(g->types.size());
  if (src < 0 || src >= n || dst < 0 || dst >= n) return fail(GRAFX_EINVAL, "node id out of range");
  if (src_port < 0 || src_port >= type_outputs(g->types[src]) || dst_port < 0 ||
      dst_port >= type_inputs(g->types[dst]))
    return fail(GRAFX_EINVAL, "port out of range for the node types");
  g->edges.push_back({src, dst});
  g->ports.push_back({src_port, dst_port});
  return GRAFX_OK;
  GX_CATCH
}

int grafx_type_ports(int32_t type, int32_t* n_inputs, int32_t* n_outputs) {
  if (type < 0 || type >= GRAFX_N_TYPES) return fail(GRAFX_EINVAL, "unknown node type");
  if (n_inputs) *n_inputs = type_inputs(type);
  if (n_outputs) *n_outputs = type_outputs(type);
  return GRAFX_OK;
}

int grafx_graph_size(const grafx_graph* g, int32_t* n_nodes, int32_t* n_edges) {
  if (!g) return fail(GRAFX_EINVAL, "null graph");
  if (n_nodes) *n_nodes = int32_t(g->types.size());
  if (n_edges) *n_edges = int32_t(g->edges.size());
  return GRAFX_OK;
}

void grafx_plan_opts_default(grafx_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->schedule = GRAFX_SCHED_BEAM;
  o->beam_width = 32;
  o->eq_taps = 1023;
  o->sample_rate = 44100;
}

int grafx_plan_create(const grafx_graph* const* graphs, int32_t n_graphs, const int64_t* lengths,
                      const grafx_plan_opts* opts, grafx_plan** out) {
  GX_TRY
  if (!graphs || !lengths || !out || n_graphs < 1) return fail(GRAFX_EINVAL, "bad arguments");
  grafx_plan_opts o;
  if (opts) o = *opts;
  else grafx_plan_opts_default(&o);
  std::vector<const grafx_graph*> gs(graphs, graphs + n_graphs);
  grafx_plan* p = new grafx_plan();
  int rc = build_plan(gs, lengths, o, p);
  if (rc) {
    delete p;
    return rc;
  }
  *out = p;
  return GRAFX_OK;
  GX_CATCH
}

static void release_side(Plan* p) {
  for (void* e : p->events) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  p->events.clear();
  if (p->side) cudaStreamDestroy(static_cast<cudaStream_t>(p->side));
  p->side = nullptr;
}

// The side stream and its events, created once per plan (no device memory).
static int ensure_side(Plan* p) {
  if (p->side) return GRAFX_OK;
  cudaStream_t st;
  int rc = cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "side stream");
  if (rc) return rc;
  p->side = st;
  const int N = int(p->sched.string.size()) - 1;
  for (int i = 0; i < 2 * (N + 1) + 2; ++i) {
    cudaEvent_t e;
    rc = cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "side events");
    if (rc) {
      release_side(p);
      return rc;
    }
    p->events.push_back(e);
  }
  return GRAFX_OK;
}

static cudaEvent_t ev_fork(const Plan* p) { return static_cast<cudaEvent_t>(p->events[0]); }
static cudaEvent_t ev_join(const Plan* p) { return static_cast<cudaEvent_t>(p->events[1]); }
static cudaEvent_t ev_fwd(const Plan* p, int k) { return static_cast<cudaEvent_t>(p->events[2 + k]); }
static cudaEvent_t ev_bwd(const Plan* p, int k) {
  return static_cast<cudaEvent_t>(p->events[2 + (p->sched.string.size()) + k]);
}

int grafx_plan_destroy(grafx_plan* p) {
  if (p) release_side(p);
  delete p;
  return GRAFX_OK;
}

int grafx_plan_info(const grafx_plan* p, grafx_plan_info_t* info) {
  if (!p || !info) return fail(GRAFX_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->n_graphs = p->n_graphs;
  info->n_nodes = int32_t(p->types.size());
  info->n_edges = int32_t(p->edges.size());
  info->n_steps = int32_t(p->sched.string.size()) - 1;
  info->n_inputs = p->step_ptr[1];
  info->n_outputs = int32_t(p->outputs_new.size());
  std::memcpy(info->n_type_rows, p->n_type_rows, sizeof(info->n_type_rows));
  info->src_elems = p->src_elems;
  info->out_elems = p->out_elems;
  info->node_samples = p->node_samples;
  info->ws_bytes = p->ws.total;
  info->eq_fft = p->eq_fft;
  info->comp_chunk = p->comp_chunk;
  std::memcpy(info->param_cols, p->pcols, sizeof(info->param_cols));
  info->source_batch = p->source_batch;
  for (const StepInfo& st : p->steps) info->fused_pairs += st.fuse_next != 0;
  return GRAFX_OK;
}

int grafx_plan_export(const grafx_plan* p, int32_t* type_string, int32_t* step_ptr, int32_t* sigma,
                      int32_t* csr_ptr, int32_t* csr_src, int32_t* tcsr_ptr, int32_t* tcsr_dst,
                      int32_t* param_row) {
  if (!p) return fail(GRAFX_EINVAL, "null plan");
  auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
  };
  cp(type_string, p->sched.string);
  cp(step_ptr, p->step_ptr);
  cp(sigma, p->sigma);
  cp(csr_ptr, p->csr_ptr);
  cp(csr_src, p->csr_src);
  cp(tcsr_ptr, p->tcsr_ptr);
  cp(tcsr_dst, p->tcsr_dst);
  cp(param_row, p->param_row);
  return GRAFX_OK;
}

int grafx_plan_step_items(const grafx_plan* p, int32_t step, int32_t backward, int32_t* items, int32_t capacity,
                          int32_t* count) {
  if (!p || !count) return fail(GRAFX_EINVAL, "null argument");
  const int32_t N = int32_t(p->steps.size()) - 1;
  if (step < 1 || step > N) return fail(GRAFX_EINVAL, "step out of range");
  const StepInfo& st = p->steps[step];
  const int32_t begin = backward ? st.bitem_begin : st.fitem_begin;
  const int32_t n = backward ? st.bitem_count : st.fitem_count;
  *count = n;
  if (!items) return GRAFX_OK;
  if (n > capacity) return fail(GRAFX_ESHAPE, "items capacity too small");
  for (int32_t i = 0; i < n; ++i) {
    const int4_ w = p->items[size_t(begin) + i];
    items[4 * i] = w.x, items[4 * i + 1] = w.y, items[4 * i + 2] = w.z, items[4 * i + 3] = w.w;
  }
  return GRAFX_OK;
}

int grafx_plan_bind_workspace(grafx_plan* p, void* dev_ws, size_t bytes, void* stream) {
  GX_TRY
  if (!p || !dev_ws) return fail(GRAFX_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(dev_ws) % 256) return fail(GRAFX_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < p->ws.total) return fail(GRAFX_ESHAPE, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<char> img(p->ws.tables_end, 0);
  auto put = [&](size_t off, const void* src, size_t n) {
    if (n) std::memcpy(img.data() + off, src, n);
  };
  put(p->ws.nodes, p->nodes.data(), p->nodes.size() * sizeof(NodeDev));
  put(p->ws.node_ext, p->node_ext.data(), p->node_ext.size() * sizeof(int4_));
  put(p->ws.csr_ptr, p->csr_ptr.data(), p->csr_ptr.size() * 4);
  put(p->ws.csr_src, p->csr_src.data(), p->csr_src.size() * 4);
  put(p->ws.tcsr_ptr, p->tcsr_ptr.data(), p->tcsr_ptr.size() * 4);
  put(p->ws.tcsr_dst, p->tcsr_dst.data(), p->tcsr_dst.size() * 4);
  put(p->ws.items, p->items.data(), p->items.size() * sizeof(int4_));
  put(p->ws.csr_row, p->csr_row.data(), p->csr_row.size() * 8);
  put(p->ws.tcsr_row, p->tcsr_row.data(), p->tcsr_row.size() * 8);
  put(p->ws.in1_begin, p->in1_begin.data(), p->in1_begin.size() * 4);
  put(p->ws.out1_begin, p->out1_begin.data(), p->out1_begin.size() * 4);
  put(p->ws.twiddle, p->twiddle.data(), p->twiddle.size() * sizeof(float2_));
  put(p->ws.ptw, p->ptw.data(), p->ptw.size() * sizeof(float2_));
  put(p->ws.eq_cos, p->eq_cos.data(), p->eq_cos.size() * 4);
  put(p->ws.eq_hann, p->eq_hann.data(), p->eq_hann.size() * 4);
  put(p->ws.eq_band, p->eq_band.data(), p->eq_band.size() * 4);
  put(p->ws.rv_band, p->rv_band.data(), p->rv_band.size() * 4);
  put(p->ws.rv_win, p->rv_win.data(), p->rv_win.size() * 4);
  put(p->ws.rv_cs, p->rv_cs.data(), p->rv_cs.size() * sizeof(float2_));
  put(p->ws.loss_rows, p->loss.rows.data(), p->loss.rows.size() * sizeof(LossRow));
  put(p->ws.loss_items, p->loss.items.data(), p->loss.items.size() * sizeof(int4_));
  int rc = cuda_check(cudaMemcpyAsync(dev_ws, img.data(), img.size(), cudaMemcpyHostToDevice, s), "upload tables");
  if (rc) return rc;
  rc = cuda_check(cudaMemsetAsync(static_cast<char*>(dev_ws) + p->ws.status, 0, 16, s), "clear status");
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(s), "upload tables");
  if (rc) return rc;
  rc = ensure_side(p);
  if (rc) return rc;
  p->dev_ws = static_cast<char*>(dev_ws);
  init_launchers(p, s);
  return GRAFX_OK;
  GX_CATCH
}

int grafx_bind_params(grafx_plan* p, int32_t type, const float* dev, int64_t rows, int64_t cols) {
  if (!p) return fail(GRAFX_EINVAL, "null plan");
  if (type < 0 || type >= GRAFX_N_TYPES) return fail(GRAFX_ETYPE, "unknown node type");
  if (param_cols(p, type) == 0) return fail(GRAFX_ETYPE, "type has no parameters");
  if (rows != p->n_type_rows[type] || cols != param_cols(p, type))
    return fail(GRAFX_ESHAPE, "parameter table shape mismatch");
  if (rows > 0 && !dev) return fail(GRAFX_EINVAL, "null parameter pointer");
  p->params[type] = dev;
  p->param_rows[type] = rows;
  return GRAFX_OK;
}

int grafx_bind_reverb_noise(grafx_plan* p, const float* dev, int64_t n) {
  if (!p) return fail(GRAFX_EINVAL, "null plan");
  if (n != 2 * int64_t(RV_LEN)) return fail(GRAFX_ESHAPE, "reverb noise must hold 2 x 88200 floats");
  if (!dev) return fail(GRAFX_EINVAL, "null noise pointer");
  p->rv_noise = dev;
  return GRAFX_OK;
}

// Forward steps [first, last) (already validated); returns the number of launches.
// NVTX range per schedule step (visible in a profiler's timeline; no cost otherwise)
struct StepRange {
  StepRange(const char* dir, int k, int type) {
    char name[48];
    std::snprintf(name, sizeof(name), "grafx %s step %d type %d", dir, k, type);
    nvtxRangePushA(name);
  }
  ~StepRange() { nvtxRangePop(); }
};

// Forward steps whose processors have a parameter-only design (EQ filter spectra,
// delay taps, reverb impulse responses): the design depends on no signal, so it runs on
// the side stream from the start of the range and the step waits for it.
// kernel variant of the compressor family (compressor, noisegate, sidechain)
static int comp_mode_of(int type) { return type == GRAFX_T_GATE ? 1 : type == GRAFX_T_SIDECHAIN ? 2 : 0; }

static bool has_design(int type) {
  return type == GRAFX_T_EQ || type == GRAFX_T_DELAY || type == GRAFX_T_REVERB;
}

static int render_range(grafx_plan* p, const float* sources, float* out, int32_t first, int32_t last,
                        cudaStream_t s) {
  DevCtx c = make_ctx(p, sources, out, nullptr, nullptr);
  int launches = 0;
  cudaStream_t side = static_cast<cudaStream_t>(p->side);
  bool forked = false;
  for (int k = first; k < last; ++k) {
    const StepInfo& st = p->steps[k];
    if (!has_design(st.type)) continue;
    if (!forked) {
      cudaEventRecord(ev_fork(p), s);
      cudaStreamWaitEvent(side, ev_fork(p), 0);
      forked = true;
    }
    c.params = p->params[st.type];
    c.pcols = param_cols(p, st.type);
    if (st.type == GRAFX_T_EQ) launches += launch_eq(0, c, st.node_begin, st.node_end, side);
    if (st.type == GRAFX_T_DELAY) launches += launch_delay(0, c, st.node_begin, st.node_end, side);
    if (st.type == GRAFX_T_REVERB) launches += launch_reverb(0, c, st.node_begin, st.node_end, side);
    cudaEventRecord(ev_fwd(p, k), side);
  }
  for (int k = first; k < last; ++k) {
    const StepInfo& st = p->steps[k];
    StepRange range("fwd", k, st.type);
    if (st.fuse_next && k + 1 < last) {   // fused pair: one kernel over step k+1's items
      const StepInfo& sw = p->steps[k + 1];
      c.params = p->params[sw.type];
      c.params2 = p->params[st.type];
      if (st.fuse_next == 1 || st.fuse_next == 3) {
        launches += launch_ew2(false, st.type, sw.type, c, sw.fitem_begin, sw.fitem_count, s);
      } else {   // gain -> EQ: the EQ forward with the gain prologue
        c.pcols = param_cols(p, sw.type);
        cudaStreamWaitEvent(s, ev_fwd(p, k + 1), 0);
        launches += launch_eq(4, c, sw.fitem_begin, sw.fitem_count, s);
      }
      ++k;
      continue;
    }
    c.params = p->params[st.type];
    c.pcols = param_cols(p, st.type);
    if (has_design(st.type)) cudaStreamWaitEvent(s, ev_fwd(p, k), 0);
    switch (st.type) {
      case GRAFX_T_EQ:
        launches += launch_eq(1, c, st.fitem_begin, st.fitem_count, s);
        break;
      case GRAFX_T_BALLISTIC:
        launches += launch_bal_fwd(c, st.fitem_begin, st.fitem_count, st.node_begin, st.node_end, s);
        break;
      case GRAFX_T_COMP:
      case GRAFX_T_GATE:
      case GRAFX_T_SIDECHAIN:
        launches += launch_comp(0, c, st.fitem_begin, st.fitem_count, st.node_begin, st.node_end, 2 * k,
                                comp_mode_of(st.type), s);
        break;
      case GRAFX_T_DELAY:
        launches += launch_delay(1, c, st.fitem_begin, st.fitem_count, s);
        break;
      case GRAFX_T_REVERB:
        launches += launch_delay(3, c, st.fitem_begin, st.fitem_count, s);   // u window spectra
        launches += launch_reverb(1, c, st.node_begin, st.node_end, s);
        break;
      default:
        launches += launch_ew_fwd(st.type, c, st.fitem_begin, st.fitem_count, s);
    }
  }
  return launches;
}

int grafx_render_steps(grafx_plan* p, const float* sources, float* out, int32_t first, int32_t last,
                       void* stream) {
  if (!p || !sources || !out) return fail(GRAFX_EINVAL, "null argument");
  int rc = check_ready(p);
  if (rc) return rc;
  const int N = int(p->sched.string.size()) - 1;
  if (first < 1 || last > N + 1 || first > last) return fail(GRAFX_EINVAL, "step range out of bounds");
  p->last_launches = render_range(p, sources, out, first, last, static_cast<cudaStream_t>(stream));
  return cuda_check(cudaGetLastError(), "render launch");
}

int grafx_render(grafx_plan* p, const float* sources, float* out, void* stream) {
  if (!p) return fail(GRAFX_EINVAL, "null argument");
  return grafx_render_steps(p, sources, out, 1, int32_t(p->sched.string.size()), stream);
}

int grafx_node_inputs(grafx_plan* p, const float* sources, const float* out, const int32_t* ids, int32_t n,
                      float* dst, int64_t dst_pitch, void* stream) {
  if (!p || !sources || !out || (!ids && n > 0) || (!dst && n > 0)) return fail(GRAFX_EINVAL, "null argument");
  int rc = check_ready(p);
  if (rc) return rc;
  if (!p->seg_ptr.empty()) return fail(GRAFX_ESTATE, "node inputs need a plan without checkpointing");
  const int32_t nv = int32_t(p->types.size());
  if (n < 0 || dst_pitch < 4 || (dst_pitch & 3)) return fail(GRAFX_ESHAPE, "bad node-input shape");
  for (int32_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= nv) return fail(GRAFX_EINVAL, "node id out of range");
    if (p->types[ids[i]] == GRAFX_T_IN) return fail(GRAFX_EINVAL, "input nodes have no node input");
    if (p->L[p->node_graph[ids[i]]] > dst_pitch) return fail(GRAFX_ESHAPE, "dst_pitch below the node's length");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevCtx c = make_ctx(p, sources, const_cast<float*>(out), nullptr, nullptr);
  int launches = 0;
  for (int32_t i0 = 0; i0 < n; i0 += NI_MAX) {
    NodeIds b;
    std::memset(&b, 0, sizeof(b));
    b.first = i0;
    const int m = std::min<int32_t>(NI_MAX, n - i0);
    for (int j = 0; j < m; ++j) b.v[j] = p->sigma[ids[i0 + j]];
    launches += launch_node_inputs(c, b, m, dst, dst_pitch, s);
  }
  p->last_launches = launches;
  return cuda_check(cudaGetLastError(), "node-input launch");
}

static int backprop_range(grafx_plan* p, const float* sources, const float* d_out, float* const* d_params,
                          float* d_sources, int32_t first, int32_t last, cudaStream_t s);

// Source batch: sum the B copies' gradient rows into the caller's tables.
static int fold_copies(grafx_plan* p, float* const* d_params, cudaStream_t s) {
  if (p->source_batch <= 1 || !d_params) return 0;
  int launches = 0;
  for (int t = 0; t < GRAFX_N_TYPES; ++t)
    if (d_params[t] && p->n_type_rows[t] > 0 && p->pcols[t] > 0)
      launches += launch_fold_copies(at<float>(p, p->ws.dgrad) + p->dgrad_off[t], d_params[t],
                                     int64_t(p->n_type_rows[t]) * p->pcols[t], p->source_batch, s);
  return launches;
}

int grafx_backprop_steps(grafx_plan* p, const float* sources, const float* d_out, float* const* d_params,
                         float* d_sources, int32_t first, int32_t last, void* stream) {
  if (!p || !sources || !d_out) return fail(GRAFX_EINVAL, "null argument");
  int rc = check_ready(p);
  if (rc) return rc;
  const int N = int(p->sched.string.size()) - 1;
  if (first < 0 || last > N + 1 || first > last) return fail(GRAFX_EINVAL, "step range out of bounds");
  if (p->source_batch > 1 && (first != 0 || last != N + 1))
    return fail(GRAFX_ESTATE, "with a source batch the backward runs over every step");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->last_launches = backprop_range(p, sources, d_out, d_params, d_sources, first, last, s);
  p->last_launches += fold_copies(p, d_params, s);
  return cuda_check(cudaGetLastError(), "backprop launch");
}

// Backward steps [first, last) in reverse (already validated); returns the launches.
static int backprop_range(grafx_plan* p, const float* sources, const float* d_out, float* const* d_params,
                          float* d_sources, int32_t first, int32_t last, cudaStream_t s) {
  DevCtx c = make_ctx(p, sources, nullptr, d_out, d_sources);
  int launches = 0;
  // Parameter-gradient finalizers that read only their step's private partial slots and
  // spectra (EQ, compressor/noisegate, gain/imager, reverb) run on the side stream after
  // their step's kernels, off the critical path of the input adjoints; the range joins
  // the side stream at its end.  (The delay's gradient kernels read signal rows, whose
  // adjoint storage is recycled by later steps, and stay on the main stream.)
  cudaStream_t side = static_cast<cudaStream_t>(p->side);
  bool used_side = false;
  auto to_side = [&](int k) {
    cudaEventRecord(ev_bwd(p, k), s);
    cudaStreamWaitEvent(side, ev_bwd(p, k), 0);
    used_side = true;
  };
  auto dparams_of = [&](int type) -> float* {
    float* d = d_params ? d_params[type] : nullptr;
    if (d && p->source_batch > 1) d = at<float>(p, p->ws.dgrad) + p->dgrad_off[type];
    return d;
  };
  for (int k = last - 1; k >= std::max(first, 1); --k) {
    const StepInfo& st = p->steps[k];
    if (st.type == GRAFX_T_OUT) continue;  // adjoint rows of outputs are d_out itself
    StepRange range("bwd", k, st.type);
    if (k - 1 >= std::max(first, 1) && p->steps[k - 1].fuse_next == 1) {   // fused gain/imager pair
      const StepInfo& sv = p->steps[k - 1];
      c.params = p->params[st.type];
      c.params2 = p->params[sv.type];
      launches += launch_ew2(true, sv.type, st.type, c, st.bitem_begin, st.bitem_count, s);
      float* dw = dparams_of(st.type);
      float* dv = dparams_of(sv.type);
      if (dw || dv) to_side(k);
      if (dw) {
        c.dparams = dw;
        launches += launch_ew_finalize(c, st.node_begin, st.node_end, param_cols(p, st.type), side);
      }
      if (dv) {
        c.dparams = dv;
        launches += launch_ew_finalize(c, sv.node_begin, sv.node_end, param_cols(p, sv.type), side);
      }
      --k;
      continue;
    }
    c.params = p->params[st.type];
    c.pcols = param_cols(p, st.type);
    c.dparams = dparams_of(st.type);
    switch (st.type) {
      case GRAFX_T_EQ:
        launches += launch_eq(2, c, st.bitem_begin, st.bitem_count, s);
        if (c.dparams) {
          to_side(k);
          launches += launch_eq(3, c, st.node_begin, st.node_end, side);
        }
        break;
      case GRAFX_T_COMP:
      case GRAFX_T_GATE:
      case GRAFX_T_SIDECHAIN:
        launches += launch_comp(1, c, st.bitem_begin, st.bitem_count, st.node_begin, st.node_end, 2 * k + 1,
                                comp_mode_of(st.type), s);
        if (c.dparams) {
          to_side(k);
          launches += launch_comp(2, c, 0, 0, st.node_begin, st.node_end, 0, 0, side);
        }
        break;
      case GRAFX_T_REVERB:
        launches += launch_delay(3, c, st.dsub_begin[0], st.dsub_count[0], s);   // ybar spectra
        launches += launch_reverb(2, c, st.node_begin, st.node_end, s);
        if (c.dparams) {
          to_side(k);
          launches += launch_reverb(3, c, st.node_begin, st.node_end, side);
        }
        break;
      case GRAFX_T_DELAY:
        launches += launch_delay(2, c, st.dsub_begin[0], st.dsub_count[0], s);
        if (c.dparams) {
          for (int i = 1; i < 5; ++i) launches += launch_delay(2 + i, c, st.dsub_begin[i], st.dsub_count[i], s);
        }
        break;
      case GRAFX_T_GAIN:
      case GRAFX_T_IMAGER:
        if (!d_sources && st.in_from_sources)   // the input adjoints would have no reader
          launches += launch_ew_bwd_nostore(st.type, c, st.bitem_begin, st.bitem_count, s);
        else
          launches += launch_ew_bwd(st.type, c, st.bitem_begin, st.bitem_count, s);
        if (c.dparams) {
          to_side(k);
          launches += launch_ew_finalize(c, st.node_begin, st.node_end, param_cols(p, st.type), side);
        }
        break;
      case GRAFX_T_SPLIT:
      case GRAFX_T_MERGE:
        launches += launch_ew_bwd(st.type, c, st.bitem_begin, st.bitem_count, s);
        break;
      case GRAFX_T_BALLISTIC:
        launches += launch_bal_bwd(c, st.bitem_begin, st.bitem_count, st.node_begin, st.node_end, s);
        if (c.dparams) {
          to_side(k);
          launches += launch_bal_finalize(c, st.node_begin, st.node_end, side);
        }
        break;
      default:
        if (!d_sources && st.in_from_sources) break;   // a mix of sources: no adjoint has a reader
        launches += launch_ew_bwd(GRAFX_T_MIX, c, st.bitem_begin, st.bitem_count, s);
    }
  }
  if (first == 0 && d_sources) launches += launch_ew_bwd(GRAFX_T_MIX, c, p->in_bitem_begin, p->in_bitem_count, s);
  if (used_side) {   // join: the gradients are complete when the main stream moves on
    cudaEventRecord(ev_join(p), side);
    cudaStreamWaitEvent(s, ev_join(p), 0);
  }
  return launches;
}

int grafx_backprop(grafx_plan* p, const float* sources, const float* d_out, float* const* d_params,
                   float* d_sources, void* stream) {
  if (!p) return fail(GRAFX_EINVAL, "null argument");
  const int32_t end = int32_t(p->sched.string.size());
  if (p->seg_ptr.empty()) return grafx_backprop_steps(p, sources, d_out, d_params, d_sources, 0, end, stream);
  if (!sources || !d_out) return fail(GRAFX_EINVAL, "null argument");
  int rc = check_ready(p);
  if (rc) return rc;
  // checkpointed: segments in reverse; every segment but the last (whose rows the
  // forward pass left in place) is re-rendered before its backward steps
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nseg = int(p->seg_ptr.size()) - 1;
  int launches = 0;
  for (int j = nseg - 1; j >= 0; --j) {
    const int32_t a = p->seg_ptr[j], b = p->seg_ptr[j + 1];
    if (j < nseg - 1) launches += render_range(p, sources, nullptr, a, b, s);
    launches += backprop_range(p, sources, d_out, d_params, d_sources, j == 0 ? 0 : a, b, s);
  }
  launches += fold_copies(p, d_params, s);
  p->last_launches = launches;
  return cuda_check(cudaGetLastError(), "checkpointed backprop launch");
}

int grafx_mrstft_forward(grafx_plan* p, const float* out, const float* target, float* loss, void* stream) {
  if (!p || !out || !target || !loss) return fail(GRAFX_EINVAL, "null argument");
  if (!p->dev_ws) return fail(GRAFX_ESTATE, "workspace not bound");
  if (!p->loss.ok) return fail(GRAFX_ESHAPE, "every output length must be >= 2048 for the STFT loss");
  LossLaunch L = make_loss(p, out, target);
  L.loss = loss;
  p->last_launches = launch_loss(0, L, static_cast<cudaStream_t>(stream));
  return cuda_check(cudaGetLastError(), "loss launch");
}

int grafx_mrstft_backward(grafx_plan* p, const float* out, const float* target, float* d_out, void* stream) {
  if (!p || !out || !target || !d_out) return fail(GRAFX_EINVAL, "null argument");
  if (!p->dev_ws) return fail(GRAFX_ESTATE, "workspace not bound");
  if (!p->loss.ok) return fail(GRAFX_ESHAPE, "every output length must be >= 2048 for the STFT loss");
  LossLaunch L = make_loss(p, out, target);
  L.d_out = d_out;
  p->last_launches = launch_loss(2, L, static_cast<cudaStream_t>(stream));
  return cuda_check(cudaGetLastError(), "loss launch");
}

int grafx_sync_status(grafx_plan* p, void* stream) {
  if (!p || !p->dev_ws) return fail(GRAFX_ESTATE, "workspace not bound");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = cuda_check(cudaStreamSynchronize(s), "synchronize");
  if (rc) return rc;
  uint32_t st = 0;
  rc = cuda_check(cudaMemcpy(&st, p->dev_ws + p->ws.status, 4, cudaMemcpyDeviceToHost), "read status");
  if (rc) return rc;
  if (st) {
    cudaMemset(p->dev_ws + p->ws.status, 0, 4);
    if (st & ST_TIMEOUT) return fail(GRAFX_ETIMEOUT, "a bounded device wait expired");
    return fail(GRAFX_EINVAL, "a device bounds check failed");
  }
  return GRAFX_OK;
}

int grafx_last_launch_count(const grafx_plan* p, int32_t* n) {
  if (!p || !n) return fail(GRAFX_EINVAL, "null argument");
  *n = p->last_launches;
  return GRAFX_OK;
}

struct grafx_step_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t launches = 0;
};

int grafx_step_graph_create(grafx_plan* p, const float* sources, float* out, const float* target, float* loss,
                            float* d_out, float* const* d_params, float* d_sources, void* stream,
                            grafx_step_graph** out_graph) {
  GX_TRY
  if (!p || !sources || !out || !target || !loss || !d_out || !out_graph) return fail(GRAFX_EINVAL, "null argument");
  int rc = check_ready(p);
  if (rc) return rc;
  if (!p->loss.ok) return fail(GRAFX_ESHAPE, "every output length must be >= 2048 for the STFT loss");
  if (!stream) return fail(GRAFX_EINVAL, "capture needs a non-default stream (the legacy NULL stream cannot be captured)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  init_launchers(p, s);   // kernel attributes are set outside the capture
  rc = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc) return rc;
  int32_t n = 0;
  int st = grafx_render(p, sources, out, stream);
  n += p->last_launches;
  if (!st) st = grafx_mrstft_forward(p, out, target, loss, stream), n += p->last_launches;
  if (!st) st = grafx_mrstft_backward(p, out, target, d_out, stream), n += p->last_launches;
  if (!st) st = grafx_backprop(p, sources, d_out, d_params, d_sources, stream), n += p->last_launches;
  std::string err = st ? grafx_last_error() : "";
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return fail(st, "during capture: " + err);
  }
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(GRAFX_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  }
  grafx_step_graph* g = new grafx_step_graph();
  g->graph = graph;
  g->exec = exec;
  g->launches = n;
  *out_graph = g;
  return GRAFX_OK;
  GX_CATCH
}

int grafx_step_graph_launch(grafx_step_graph* g, void* stream) {
  if (!g) return fail(GRAFX_EINVAL, "null graph");
  return cuda_check(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), "graph launch");
}

int grafx_step_graph_launches(const grafx_step_graph* g, int32_t* n) {
  if (!g || !n) return fail(GRAFX_EINVAL, "null argument");
  *n = g->launches;
  return GRAFX_OK;
}

int grafx_step_graph_destroy(grafx_step_graph* g) {
  if (!g) return GRAFX_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return GRAFX_OK;
}

}  // extern "C"
