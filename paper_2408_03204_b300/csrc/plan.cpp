// Plan building: the OptimizeNodeOrder, Reorder and GetReadWriteIndex steps of Algorithm 1
// (reordering sigma, index maps) on the host, plus the device-side work lists, constant
// tables and workspace layout.
#include "plan.h"

#include "fft.cuh"

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

namespace grafx {

namespace {
thread_local std::string g_err;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// EQ band matrix: bin k of an N-tap zero-phase FIR sits at k*fs/N; its gain in dB is
// the linear interpolation in log2(f) between the two nearest of 8 log-spaced band
// centres 20*1000^((b+0.5)/8) Hz, and the end bands' gains beyond the end centres.
void eq_band_table(int N, int fs, std::vector<float>* out) {
  const int K = (N + 1) / 2, NB = 8;
  double c[NB], lc[NB];
  for (int b = 0; b < NB; ++b) {
    c[b] = 20.0 * std::pow(1000.0, (b + 0.5) / NB);
    lc[b] = std::log2(c[b]);
  }
  out->assign(size_t(K) * NB, 0.f);
  for (int k = 0; k < K; ++k) {
    double f = double(k) * fs / N;
    float* row = out->data() + size_t(k) * NB;
    if (f <= c[0]) { row[0] = 1.f; continue; }
    if (f >= c[NB - 1]) { row[NB - 1] = 1.f; continue; }
    int b = 0;
    while (b + 1 < NB && c[b + 1] <= f) ++b;
    double w = (std::log2(f) - lc[b]) / (lc[b + 1] - lc[b]);
    row[b] = float(1.0 - w);
    row[b + 1] = float(w);
  }
}

// Block FFT size with the least transform work per output sample, M log2 M / S with
// S = M - 2H outputs per block; 8192-point blocks are charged 30% for their lower
// occupancy (512 threads, twice the shared memory).
int pick_eq_fft(int taps) {
  const int H = (taps - 1) / 2;
  int best = 0;
  double best_cost = 1e30;
  for (int m = 1024, lg = 10; m <= 8192; m *= 2, ++lg) {
    int S = (m - 2 * H) & ~3;
    if (S < 256 || S < 2 * H) continue;
    double cost = double(m) * lg / S * (m == 8192 ? 1.3 : 1.0);
    if (cost < best_cost) { best_cost = cost; best = m; }
  }
  return best ? best : 8192;
}
}  // namespace

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
void clear_error() { g_err.clear(); }
const char* last_error_cstr() { return g_err.c_str(); }

void fill_fft_tables(std::vector<float2_>& twiddle, std::vector<float2_>& ptw) {
  twiddle.resize(TWIDDLE_N);
  for (int m = 0; m < TWIDDLE_N; ++m) {
    double a = 2.0 * M_PI * m / TWIDDLE_N;
    twiddle[m] = float2_{float(std::cos(a)), float(-std::sin(a))};
  }
  // FFT pass twiddles W_{Ns R}^{r k} at [(r-1) Ns + k] for every pass of every size
  ptw.assign(fft::PTW_TOTAL, float2_{0.f, 0.f});
  for (int M = 512; M <= 8192; M *= 2) {
    for (int pass = 1, Ns = 16; pass < fft::geo_npass(M); ++pass, Ns *= 16) {
      const int R = fft::pass_radix(M, pass);
      float2_* t = ptw.data() + fft::ptw_base(M) + fft::ptw_pass_off(M, pass);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          double a = -2.0 * M_PI * double(r) * k / (double(Ns) * R);
          t[(r - 1) * Ns + k] = float2_{float(std::cos(a)), float(std::sin(a))};
        }
    }
  }
}

int build_plan(const std::vector<const grafx_graph*>& graphs_in, const int64_t* lengths_in,
               const grafx_plan_opts& opts, Plan* p) {
  p->opts = opts;
  if (graphs_in.empty()) return fail(GRAFX_EINVAL, "no graphs");
  // source-level batch: B copies of the graph list, copy-major (copy b's rows follow copy b-1's)
  if (opts.source_batch < 0 || opts.source_batch > 65536) return fail(GRAFX_EINVAL, "source_batch must be in [0, 65536]");
  p->source_batch = std::max(opts.source_batch, 1);
  p->graphs_per_copy = int32_t(graphs_in.size());
  std::vector<const grafx_graph*> graphs;
  std::vector<int64_t> lens;
  for (int32_t b = 0; b < p->source_batch; ++b)
    for (size_t g = 0; g < graphs_in.size(); ++g) {
      graphs.push_back(graphs_in[g]);
      lens.push_back(lengths_in[g]);
    }
  const int64_t* lengths = lens.data();
  p->n_graphs = int32_t(graphs.size());
  // ---- union (graph-level parallelism: one disconnected graph)
  for (int32_t g = 0; g < p->n_graphs; ++g) {
    if (!graphs[g]) return fail(GRAFX_EINVAL, "null graph");
    int64_t L = lengths[g];
    if (L < 1 || L > (int64_t(1) << 24)) return fail(GRAFX_ESHAPE, "length out of range [1, 2^24]");
    p->L.push_back(L);
    p->pitch.push_back(pitch_of(L));
    int32_t off = int32_t(p->types.size());
    for (int32_t t : graphs[g]->types) {
      p->types.push_back(t);
      p->node_graph.push_back(g);
    }
    for (size_t i = 0; i < graphs[g]->edges.size(); ++i) {
      const auto& e = graphs[g]->edges[i];
      int32_t n_g = int32_t(graphs[g]->types.size());
      if (e.first < 0 || e.first >= n_g || e.second < 0 || e.second >= n_g)
        return fail(GRAFX_EINVAL, "edge out of range");
      p->edges.push_back({e.first + off, e.second + off});
      p->ports.push_back(i < graphs[g]->ports.size() ? graphs[g]->ports[i] : std::pair<int32_t, int32_t>{0, 0});
    }
  }
  const int32_t n = int32_t(p->types.size());
  const int32_t n_e = int32_t(p->edges.size());
  int rc = validate(p->types, p->edges);
  if (rc) return rc;
  for (int32_t e = 0; e < n_e; ++e) {   // edge types t_ij = (k, l) against the node types' ports
    const int32_t k = p->ports[e].first, l = p->ports[e].second;
    if (k < 0 || k >= type_outputs(p->types[p->edges[e].first]) || l < 0 || l >= type_inputs(p->types[p->edges[e].second]))
      return fail(GRAFX_EINVAL, "edge port out of range for its node types");
  }
  for (int32_t v = 0; v < n; ++v) {
    if ((p->types[v] == GRAFX_T_DELAY || p->types[v] == GRAFX_T_REVERB) &&
        p->L[p->node_graph[v]] > int64_t(DL_MAX_BLOCKS) * DL_B)
      return fail(GRAFX_ESHAPE, "graphs with delay or reverb nodes are limited to 2^19 samples");
  }
  if (opts.eq_taps < 3 || opts.eq_taps % 2 == 0 || opts.eq_taps > 2047)
    return fail(GRAFX_EINVAL, "eq_taps must be odd in [3, 2047]");
  if (opts.sample_rate < 8000 || opts.sample_rate > 192000)
    return fail(GRAFX_EINVAL, "sample_rate must be in [8000, 192000] Hz");
  // ---- processor layouts (Sec. 3 settings)
  if (opts.eq_params != GRAFX_EQ_BANDS && opts.eq_params != GRAFX_EQ_LOGMAG)
    return fail(GRAFX_EINVAL, "eq_params must be GRAFX_EQ_BANDS or GRAFX_EQ_LOGMAG");
  if (opts.delay_layout != GRAFX_DELAY_COMPACT && opts.delay_layout != GRAFX_DELAY_SLOTS)
    return fail(GRAFX_EINVAL, "delay_layout must be GRAFX_DELAY_COMPACT or GRAFX_DELAY_SLOTS");
  if (opts.reverb_layout != GRAFX_REVERB_COMPACT && opts.reverb_layout != GRAFX_REVERB_PAPER)
    return fail(GRAFX_EINVAL, "reverb_layout must be GRAFX_REVERB_COMPACT or GRAFX_REVERB_PAPER");
  p->eq_logmag = opts.eq_params == GRAFX_EQ_LOGMAG;
  if (opts.delay_layout == GRAFX_DELAY_SLOTS) {
    p->dl_taps = DL_SLOT_TAPS;
    p->dl_nd = p->dl_slot = opts.sample_rate / 10;   // 100 ms
  }
  {
    // lags [-B, (P-1) B) must cover [-H, reach + H), reach = (taps-1) slot + N_d, plus the
    // z-gradient's read-ahead of up to 32 lags (float4 windows of its last run)
    const int64_t reach = int64_t(p->dl_taps - 1) * p->dl_slot + p->dl_nd + (DL_FIR - 1) / 2 + 32;
    p->dl_P = int32_t(1 + (reach + DL_B - 1) / DL_B);
    if (p->dl_P > DL_PMAX) return fail(GRAFX_EINVAL, "delay slots too long for this sample rate (at most 63.46 kHz)");
  }
  if (opts.reverb_layout == GRAFX_REVERB_PAPER) {
    p->rv_paper = 1;
    p->rv_n = RV_PN;
    p->rv_hop = RV_PHOP;
    p->rv_f = 1 + RV_LEN / RV_PHOP;
  }
  {
    int32_t* c = p->pcols;
    c[GRAFX_T_GAIN] = 2;
    c[GRAFX_T_IMAGER] = 1;
    c[GRAFX_T_EQ] = p->eq_logmag ? (opts.eq_taps + 1) / 2 : 8;
    c[GRAFX_T_COMP] = c[GRAFX_T_GATE] = c[GRAFX_T_SIDECHAIN] = 4;
    c[GRAFX_T_BALLISTIC] = 5;
    c[GRAFX_T_DELAY] = 2 * p->dl_taps * DL_ROW;
    c[GRAFX_T_REVERB] = p->rv_paper ? 4 * (p->rv_n / 2) : RV_COLS;
  }
  int nthr = opts.n_threads > 0 ? opts.n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  rc = make_schedule(p->types, p->edges, opts.schedule, opts.beam_width, nthr, &p->sched);
  if (rc) return rc;

  // ---- sigma: rank by (step, original id); steps become contiguous ranges (I^S)
  const int32_t N = int32_t(p->sched.string.size()) - 1;
  p->sigma.assign(n, 0);
  p->step_ptr.assign(1, 0);
  {
    int32_t next = 0;
    for (auto& st : p->sched.steps) {
      std::vector<int32_t> s = st;
      std::sort(s.begin(), s.end());
      for (int32_t v : s) p->sigma[v] = next++;
      p->step_ptr.push_back(next);
    }
  }
  p->new_types.assign(n, 0);
  p->param_row.assign(n, 0);
  p->grad_row.assign(n, 0);
  {
    int32_t cnt[GRAFX_N_TYPES] = {0};
    for (int32_t v = 0; v < n; ++v) {
      p->new_types[p->sigma[v]] = p->types[v];
      p->grad_row[p->sigma[v]] = cnt[p->types[v]]++;
    }
    std::memcpy(p->n_rows_union, cnt, sizeof(cnt));
    // the copies are identical and copy-major: union row r of type t is row r mod R_t of copy r / R_t
    for (int t = 0; t < GRAFX_N_TYPES; ++t) p->n_type_rows[t] = cnt[t] / p->source_batch;
    for (int32_t v = 0; v < n; ++v) {
      const int32_t R = p->n_type_rows[p->new_types[v]];
      p->param_row[v] = R > 0 ? p->grad_row[v] % R : 0;
    }
  }
  // ---- in-edge CSR by (dst, input port, src, output port) = I^G / I^A; consumer CSR by
  // (src, output port, dst, input port) for backward.  Each node's in-edges are grouped
  // by input port, its consumer edges by output port (in1_begin / out1_begin split them).
  std::vector<int32_t> csr_k(n_e), tcsr_l(n_e);   // the other end's port of each entry
  {
    std::vector<std::array<int32_t, 4>> ed(n_e), te(n_e);
    for (int32_t e = 0; e < n_e; ++e) {
      int32_t s = p->sigma[p->edges[e].first], d = p->sigma[p->edges[e].second];
      const int32_t k = p->ports[e].first, l = p->ports[e].second;
      ed[e] = {d, l, s, k};
      te[e] = {s, k, d, l};
    }
    std::sort(ed.begin(), ed.end());
    std::sort(te.begin(), te.end());
    p->csr_ptr.assign(n + 1, 0);
    p->tcsr_ptr.assign(n + 1, 0);
    p->csr_src.resize(n_e);
    p->tcsr_dst.resize(n_e);
    for (int32_t e = 0; e < n_e; ++e) {
      ++p->csr_ptr[ed[e][0] + 1];
      p->csr_src[e] = ed[e][2];
      csr_k[e] = ed[e][3];
      ++p->tcsr_ptr[te[e][0] + 1];
      p->tcsr_dst[e] = te[e][2];
      tcsr_l[e] = te[e][3];
    }
    for (int32_t v = 0; v < n; ++v) {
      p->csr_ptr[v + 1] += p->csr_ptr[v];
      p->tcsr_ptr[v + 1] += p->tcsr_ptr[v];
    }
    p->in1_begin.assign(n, 0);
    p->out1_begin.assign(n, 0);
    for (int32_t v = 0; v < n; ++v) {
      int32_t e = p->csr_ptr[v];
      while (e < p->csr_ptr[v + 1] && ed[e][1] < 1) ++e;
      p->in1_begin[v] = e;
      e = p->tcsr_ptr[v];
      while (e < p->tcsr_ptr[v + 1] && te[e][1] < 1) ++e;
      p->out1_begin[v] = e;
    }
  }
  // ---- row placement: inputs read the caller's sources, outputs write the caller's
  // out buffer, everything else lives in the workspace (U rows and adjoint rows)
  p->nodes.assign(n, NodeDev{});
  p->node_ext.assign(n, int4_{0, 0, 0, 0});
  int64_t src_off = 0, out_off = 0, int_off = 0;
  std::vector<int32_t> inv(n);
  for (int32_t v = 0; v < n; ++v) inv[p->sigma[v]] = v;
  p->src_graph_off.assign(p->n_graphs, -1);
  p->out_graph_off.assign(p->n_graphs, -1);
  for (int32_t vn = 0; vn < n; ++vn) {
    int32_t vo = inv[vn];
    int32_t g = p->node_graph[vo];
    NodeDev& nd = p->nodes[vn];
    nd.len = int32_t(p->L[g]);
    nd.pitch = int32_t(p->pitch[g]);
    nd.prow = p->param_row[vn];
    nd.grow = p->source_batch > 1 ? p->grad_row[vn] : p->param_row[vn];
    nd.type = int16_t(p->types[vo]);
    int64_t row = 2 * p->pitch[g];
    if (nd.type == GRAFX_T_IN) {
      nd.kind = KIND_INPUT;
      nd.off_y = nd.off_a = src_off;
      src_off += row;
    } else if (nd.type == GRAFX_T_OUT) {
      nd.kind = KIND_OUTPUT;
      nd.off_y = nd.off_a = out_off;
      out_off += row;
      p->outputs_new.push_back(vn);
    } else {
      nd.kind = KIND_INTERNAL;
      nd.off_y = nd.off_a = int_off;
      nd.rstride = int32_t(align_up(size_t(row), 64));
      int_off += int64_t(type_outputs(nd.type)) * nd.rstride;   // one row per output port
      p->node_samples += nd.len;
    }
    if (nd.kind != KIND_INTERNAL) nd.rstride = int32_t(row);
    if (nd.type == GRAFX_T_OUT) p->node_samples += nd.len;
  }
  // inputs and outputs are ordered graph-major because sigma keeps original order
  // inside a step and the union concatenates graphs in order
  p->src_elems = src_off;
  p->out_elems = out_off;
  const int64_t internal_floats = int_off;  // U rows: one per output port of each internal node
  // ---- signal checkpointing: with segments of opts.checkpoint_steps schedule steps,
  // a U row is kept for the whole pass only if a consumer lies in a later segment
  // (its forward value is needed when a later segment is recomputed or run); all other
  // rows of a segment share one scratch region, reused by every segment.  The backward
  // pass recomputes each earlier segment's forward before its own steps.
  // ---- fusable step pairs (k, k+1): every node w of step k+1 has one in-edge, from a
  // node v of step k whose only consumer is w, and the node counts agree (so the map is a
  // bijection).  Both gain/imager: fused forward and backward (fuse 1); gain then EQ: the
  // EQ forward applies the gain on load (fuse 2, backward unfused).  Not with
  // checkpointing (a pair could straddle a segment).  A fused backward writes a_v while
  // it reads the adjoints of w's consumers, so a_v's life starts at step k+1's backward
  // (below).
  std::vector<int8_t> fuse(N + 1, 0);
  {
    auto pointwise = [](int t) { return t == GRAFX_T_GAIN || t == GRAFX_T_IMAGER; };
    for (int32_t k = 1; opts.checkpoint_steps == 0 && k + 1 <= N; ++k) {
      const int32_t a0 = p->step_ptr[k], a1 = p->step_ptr[k + 1], b0 = p->step_ptr[k + 1], b1 = p->step_ptr[k + 2];
      const int32_t ta = p->sched.string[k], tb = p->sched.string[k + 1];
      int8_t kind = 0;
      if (tb != GRAFX_T_OUT && pointwise(ta) && pointwise(tb)) kind = 1;
      else if (ta == GRAFX_T_GAIN && tb == GRAFX_T_EQ) kind = 2;
      else if (ta == GRAFX_T_MIX && tb == GRAFX_T_OUT) kind = 3;   // the output copies its mix
      if (!kind || a1 - a0 != b1 - b0) continue;
      bool ok = true;
      for (int32_t w = b0; ok && w < b1; ++w) {
        ok = p->csr_ptr[w + 1] - p->csr_ptr[w] == 1;
        if (!ok) break;
        const int32_t v = p->csr_src[p->csr_ptr[w]];
        ok = v >= a0 && v < a1 && p->tcsr_ptr[v + 1] - p->tcsr_ptr[v] == 1;
      }
      if (ok) {
        fuse[k] = kind;
        ++k;   // a fused pair does not chain into a third step
      }
    }
  }
  // ---- adjoint rows by liveness: a_w (the input adjoint of w) is written by the backward
  // step of w and read by the backward steps of w's producers (step 0 = the source
  // adjoints), so in backward order it lives over [N - step(w), N - min step(producer)].
  // Rows of the same size whose intervals do not meet share memory (first free slot).
  int64_t a_floats = 0;
  {
    std::vector<int32_t> step_of(n, 0);
    for (int32_t st = 0; st <= N; ++st)
      for (int32_t v = p->step_ptr[st]; v < p->step_ptr[st + 1]; ++v) step_of[v] = st;
    struct Live { int32_t start, end, v; int64_t size; };
    std::vector<Live> lives;
    for (int32_t v = 0; v < n; ++v) {
      if (p->nodes[v].kind != KIND_INTERNAL) continue;
      int32_t lo = step_of[v];
      for (int32_t e = p->csr_ptr[v]; e < p->csr_ptr[v + 1]; ++e) lo = std::min(lo, step_of[p->csr_src[e]]);
      // one adjoint row per input port; a fused pair's first node is written one step early
      const int32_t written = fuse[step_of[v]] == 1 ? step_of[v] + 1 : step_of[v];
      lives.push_back({N - written, N - lo, v, int64_t(type_inputs(p->nodes[v].type)) * p->nodes[v].rstride});
    }
    std::stable_sort(lives.begin(), lives.end(), [](const Live& a, const Live& b) { return a.start < b.start; });
    struct Pool { std::vector<int64_t> free_slots; std::vector<std::pair<int32_t, int64_t>> busy; };
    std::map<int64_t, Pool> pools;
    for (const Live& l : lives) {
      Pool& pl = pools[l.size];
      for (size_t i = 0; i < pl.busy.size();) {  // release slots whose interval ended
        if (pl.busy[i].first < l.start) {
          pl.free_slots.push_back(pl.busy[i].second);
          pl.busy[i] = pl.busy.back();
          pl.busy.pop_back();
        } else {
          ++i;
        }
      }
      int64_t off;
      if (!pl.free_slots.empty()) {
        std::sort(pl.free_slots.begin(), pl.free_slots.end(), std::greater<int64_t>());
        off = pl.free_slots.back();
        pl.free_slots.pop_back();
      } else {
        off = a_floats;
        a_floats += l.size;
      }
      p->nodes[l.v].off_a = off;
      pl.busy.push_back({l.end, off});
    }
  }
  int64_t u_floats = internal_floats;
  p->ckpt_steps = opts.checkpoint_steps;
  p->seg_ptr.clear();
  if (opts.checkpoint_steps < 0) return fail(GRAFX_EINVAL, "checkpoint_steps must be >= 0");
  if (opts.checkpoint_steps > 0) {
    const int32_t k = opts.checkpoint_steps;
    for (int32_t s0 = 1; s0 <= N; s0 += k) p->seg_ptr.push_back(s0);
    p->seg_ptr.push_back(N + 1);
    std::vector<int32_t> seg_of_node(n, -1);
    for (int32_t st = 1; st <= N; ++st)
      for (int32_t v = p->step_ptr[st]; v < p->step_ptr[st + 1]; ++v) seg_of_node[v] = (st - 1) / k;
    std::vector<char> keep(n, 0);
    for (int32_t v = 0; v < n; ++v) {
      if (p->nodes[v].kind != KIND_INTERNAL) continue;
      for (int32_t e = p->tcsr_ptr[v]; e < p->tcsr_ptr[v + 1]; ++e)
        if (seg_of_node[p->tcsr_dst[e]] > seg_of_node[v]) keep[v] = 1;
    }
    int64_t kept = 0;
    for (int32_t v = 0; v < n; ++v)
      if (keep[v]) {
        p->nodes[v].off_y = kept;
        kept += int64_t(type_outputs(p->nodes[v].type)) * p->nodes[v].rstride;
      }
    int64_t scratch = 0, cur = 0;
    int32_t cur_seg = -1;
    for (int32_t v = 0; v < n; ++v) {  // new ids run step by step, so segment by segment
      if (p->nodes[v].kind != KIND_INTERNAL || keep[v]) continue;
      if (seg_of_node[v] != cur_seg) cur_seg = seg_of_node[v], cur = 0;
      p->nodes[v].off_y = kept + cur;
      cur += int64_t(type_outputs(p->nodes[v].type)) * p->nodes[v].rstride;
      scratch = std::max(scratch, cur);
    }
    u_floats = kept + scratch;
  }
  // ---- row references of the CSR entries (the rows are placed now): the source's output
  // port row for every in-edge, the consumer's input-port adjoint row for every consumer edge
  p->csr_row.resize(n_e);
  p->tcsr_row.resize(n_e);
  for (int32_t e = 0; e < n_e; ++e) {
    const NodeDev& s = p->nodes[p->csr_src[e]];
    p->csr_row[e] = (int64_t(s.kind) << REF_SHIFT) | (s.off_y + int64_t(csr_k[e]) * s.rstride);
    const NodeDev& w = p->nodes[p->tcsr_dst[e]];
    p->tcsr_row[e] = (int64_t(w.kind) << REF_SHIFT) | (w.off_a + int64_t(tcsr_l[e]) * w.rstride);
  }

  // ---- tile sizes
  p->eq_taps = opts.eq_taps;
  p->eq_H = (opts.eq_taps - 1) / 2;
  p->eq_fft = opts.eq_fft ? opts.eq_fft : pick_eq_fft(opts.eq_taps);
  if (p->eq_fft != 1024 && p->eq_fft != 2048 && p->eq_fft != 4096 && p->eq_fft != 8192)
    return fail(GRAFX_EINVAL, "eq_fft must be 1024, 2048, 4096 or 8192");
  const int32_t Hal = (p->eq_H + 3) & ~3;
  p->eq_step = (p->eq_fft - 2 * p->eq_H) & ~3;
  // S >= 2H: an input-adjoint block's head and tail reach only its two neighbours, and
  // into disjoint parts of their output ranges
  if (p->eq_step < 256 || p->eq_step < 2 * p->eq_H) return fail(GRAFX_EINVAL, "eq_fft too small for eq_taps");
  p->comp_chunk = opts.comp_chunk ? opts.comp_chunk : 2048;
  if (p->comp_chunk != 1024 && p->comp_chunk != 2048 && p->comp_chunk != 4096)
    return fail(GRAFX_EINVAL, "comp_chunk must be 1024, 2048 or 4096");

  // ---- work lists: forward items of every step, then backward items of every step
  p->steps.assign(N + 1, StepInfo{});
  std::vector<int4_> fwd, bwd;
  int32_t slot = 0, run = 0, chunk_id = 0;
  for (int32_t k = 1; k <= N; ++k) {
    StepInfo& s = p->steps[k];
    s.type = p->sched.string[k];
    s.fuse_next = fuse[k];
    s.in_from_sources = 1;
    for (int32_t v = p->step_ptr[k]; s.in_from_sources && v < p->step_ptr[k + 1]; ++v)
      for (int32_t e = p->csr_ptr[v]; e < p->csr_ptr[v + 1]; ++e)
        if (p->nodes[p->csr_src[e]].kind != KIND_INPUT) s.in_from_sources = 0;
    s.node_begin = p->step_ptr[k];
    s.node_end = p->step_ptr[k + 1];
    s.fitem_begin = int32_t(fwd.size());
    int32_t fmax_nc = 0;
    for (int32_t v = s.node_begin; v < s.node_end; ++v) {
      const int32_t L = p->nodes[v].len;
      switch (s.type) {
        case GRAFX_T_EQ: {
          p->node_ext[v].z = p->n_eq++;
          int32_t nb = int32_t((int64_t(L) + Hal - p->eq_H + p->eq_step - 1) / p->eq_step);
          // w: the node's first block in the input-spectrum store (the forward writes block
          // j's spectrum at w + j, the backward reads it)
          p->node_ext[v].w = int32_t(p->n_eq_blocks);
          for (int32_t j = 0; j < nb; ++j) fwd.push_back({v, j, p->node_ext[v].z, int32_t(p->n_eq_blocks + j)});
          p->n_eq_blocks += nb;
          break;
        }
        case GRAFX_T_DELAY: {
          const int32_t nb = (L + DL_B - 1) / DL_B;
          p->node_ext[v].z = p->n_delay++;
          p->node_ext[v].w = nb;
          p->dl_nbmax = std::max(p->dl_nbmax, nb);
          for (int32_t ch = 0; ch < 2; ++ch)
            for (int32_t t0 = 0; t0 < L; t0 += DL_TILE) fwd.push_back({v, t0, ch, 0});
          break;
        }
        case GRAFX_T_REVERB: {
          // u window spectra (kind 0) from window -RV_P; slots: windows, ybar blocks, ybar windows
          const int32_t nb = (L + DL_B - 1) / DL_B, nw = nb + RV_P;
          p->node_ext[v] = int4_{p->n_dl_slots, 0, p->n_reverb++, nb};
          p->rv_nbmax = std::max(p->rv_nbmax, nb);
          for (int32_t w = -RV_P; w < nb; ++w) fwd.push_back({v, w, 0, p->n_dl_slots + w + RV_P});
          p->n_dl_slots += nw + nb + nw;
          break;
        }
        case GRAFX_T_BALLISTIC: {
          // scratch block of 4 rows (mid, envelope, adjoint, coefficient), offset in 64-float units
          p->node_ext[v].z = p->n_bal++;
          p->node_ext[v].w = int32_t(p->bal_floats / 64);
          p->bal_floats += 4 * int64_t(align_up(size_t(p->nodes[v].pitch), 64));
          for (int32_t t0 = 0; t0 < L; t0 += EW_TILE) fwd.push_back({v, t0, 0, 0});
          break;
        }
        case GRAFX_T_COMP:
        case GRAFX_T_GATE:
        case GRAFX_T_SIDECHAIN: {
          // chunk ids contiguous per node; the items follow the loop, round by round
          int32_t nc = (L + p->comp_chunk - 1) / p->comp_chunk;
          p->node_ext[v].z = chunk_id;
          chunk_id += nc;
          fmax_nc = std::max(fmax_nc, nc);
          break;
        }
        default:
          for (int32_t t0 = 0; t0 < L; t0 += EW_TILE) fwd.push_back({v, t0, 0, 0});
      }
    }
    // compressor-like forward: the c-th chunk of every node before any node's (c+1)-th
    // (the one-pass look-back takes its tickets in this order: a chunk's predecessor is,
    // on steps of many nodes, a whole round of tickets earlier)
    for (int32_t ck = 0; ck < fmax_nc; ++ck)
      for (int32_t v = s.node_begin; v < s.node_end; ++v) {
        const int32_t nc = (p->nodes[v].len + p->comp_chunk - 1) / p->comp_chunk;
        if (ck < nc) fwd.push_back({v, ck, p->node_ext[v].z + ck, 0});
      }
    s.fitem_count = int32_t(fwd.size()) - s.fitem_begin;
  }
  for (int32_t k = N; k >= 1; --k) {
    StepInfo& s = p->steps[k];
    s.bitem_begin = int32_t(bwd.size());
    if (s.type == GRAFX_T_OUT) { s.bitem_count = 0; continue; }  // adjoint rows alias d_out
    if (s.type == GRAFX_T_REVERB) {
      for (int i = 0; i < 5; ++i) s.dsub_begin[i] = int32_t(bwd.size()), s.dsub_count[i] = 0;
      for (int32_t v = s.node_begin; v < s.node_end; ++v) {
        const int32_t nb = p->node_ext[v].w, nw = nb + RV_P, base = p->node_ext[v].x;
        for (int32_t b = 0; b < nb; ++b) bwd.push_back({v, b, 1, base + nw + b});
        for (int32_t w = 0; w < nw; ++w) bwd.push_back({v, w, 2, base + nw + nb + w});
      }
      s.dsub_count[0] = int32_t(bwd.size()) - s.dsub_begin[0];
      s.bitem_count = int32_t(bwd.size()) - s.bitem_begin;
      continue;
    }
    if (s.type == GRAFX_T_DELAY) {
      std::vector<int4_> sub[5];
      for (int32_t v = s.node_begin; v < s.node_end; ++v) {
        const int32_t L = p->nodes[v].len, nb = p->node_ext[v].w;
        for (int32_t ch = 0; ch < 2; ++ch)
          for (int32_t t0 = 0; t0 < L; t0 += DL_TILE) sub[0].push_back({v, t0, ch, 0});
        p->node_ext[v].x = p->n_dl_slots;
        p->node_ext[v].y = p->node_ext[v].z * p->dl_P;
        // u windows from -P; those before -1 hold no sample (zero spectra, which the lag
        // accumulation takes as such): their slots are kept but not computed
        for (int32_t w = -p->dl_P; w < nb; ++w) {
          if (w >= -1) sub[1].push_back({v, w, 0, p->n_dl_slots});
          ++p->n_dl_slots;
        }
        for (int32_t b = 0; b < nb; ++b) sub[1].push_back({v, b, 1, p->n_dl_slots++});
        // bins 0..M/2 (the lag spectra are conjugate-symmetric per channel)
        for (int32_t ck = 0; ck <= DL_M / 2 / DL_CHUNK; ++ck) sub[2].push_back({v, ck, 0, 0});
        for (int32_t q = 0; q < p->dl_P; ++q) sub[3].push_back({v, q, 0, 0});
        for (int32_t xm = 0; xm < 2 * p->dl_taps; ++xm) sub[4].push_back({v, xm, 0, 0});
      }
      for (int i = 0; i < 5; ++i) {
        s.dsub_begin[i] = int32_t(bwd.size());
        s.dsub_count[i] = int32_t(sub[i].size());
        bwd.insert(bwd.end(), sub[i].begin(), sub[i].end());
      }
      s.bitem_count = int32_t(bwd.size()) - s.bitem_begin;
      continue;
    }
    // EQ: runs of consecutive blocks, sized for about two waves of resident CTAs
    int32_t run_len = 1;
    if (s.type == GRAFX_T_EQ) {
      int64_t blocks = 0;
      for (int32_t v = s.node_begin; v < s.node_end; ++v)
        blocks += (int64_t(p->nodes[v].len) + Hal - p->eq_H + p->eq_step - 1) / p->eq_step;
      const int64_t target = 148 * 3 * 2;
      run_len = int32_t(std::max<int64_t>(1, (blocks + target - 1) / target));
    }
    int32_t max_nc = 0;
    for (int32_t v = s.node_begin; v < s.node_end; ++v) {
      const int32_t L = p->nodes[v].len;
      switch (s.type) {
        case GRAFX_T_EQ: {
          int32_t nb = int32_t((int64_t(L) + Hal - p->eq_H + p->eq_step - 1) / p->eq_step);
          p->node_ext[v].x = run;
          for (int32_t j = 0; j < nb; j += run_len) bwd.push_back({v, j, std::min(run_len, nb - j), run++});
          p->node_ext[v].y = run - p->node_ext[v].x;
          break;
        }
        case GRAFX_T_COMP:
        case GRAFX_T_GATE:
        case GRAFX_T_SIDECHAIN: {
          // partial slot x + r for the node's r-th chunk from its end (the items follow the
          // loop, round by round)
          int32_t nc = (L + p->comp_chunk - 1) / p->comp_chunk;
          p->node_ext[v].x = slot;
          p->node_ext[v].y = nc;
          slot += nc;
          max_nc = std::max(max_nc, nc);
          break;
        }
        default: {
          bool has_p = s.type == GRAFX_T_GAIN || s.type == GRAFX_T_IMAGER || s.type == GRAFX_T_BALLISTIC;
          p->node_ext[v].x = slot;
          int32_t cnt = 0;
          const int32_t per = s.type == GRAFX_T_BALLISTIC ? 2 : 1;   // partial slots per tile
          for (int32_t t0 = 0; t0 < L; t0 += EW_TILE, ++cnt) {
            bwd.push_back({v, t0, 0, has_p ? slot : -1});
            if (has_p) slot += per;
          }
          p->node_ext[v].y = has_p ? cnt : 0;
        }
      }
    }
    // compressor-like backward: the r-th chunk from the end of every node before any
    // node's (r+1)-th, so that a chunk's successor in the reverse recursion (handed out by
    // ticket in this order) is, on steps of many nodes, a whole round of tickets later
    for (int32_t r = 0; r < max_nc; ++r)
      for (int32_t v = s.node_begin; v < s.node_end; ++v) {
        const int32_t nc = p->node_ext[v].y, c = nc - 1 - r;
        if (c >= 0) bwd.push_back({v, c, p->node_ext[v].z + c, p->node_ext[v].x + r});
      }
    s.bitem_count = int32_t(bwd.size()) - s.bitem_begin;
  }
  // input step (adjoints of the sources), after the others in the backward list
  p->in_bitem_begin = int32_t(bwd.size());
  for (int32_t v = 0; v < p->step_ptr[1]; ++v)
    for (int32_t t0 = 0; t0 < p->nodes[v].len; t0 += EW_TILE) bwd.push_back({v, t0, 0, -1});
  p->in_bitem_count = int32_t(bwd.size()) - p->in_bitem_begin;
  p->n_partials = slot;
  p->n_eq_runs = run;
  p->n_comp_chunks = chunk_id;
  p->n_fitems = int32_t(fwd.size());
  for (int32_t k = 1; k <= N; ++k) {
    p->steps[k].bitem_begin += p->n_fitems;
    for (int i = 0; i < 5; ++i) p->steps[k].dsub_begin[i] += p->n_fitems;
  }
  p->in_bitem_begin += p->n_fitems;
  p->items = fwd;
  p->items.insert(p->items.end(), bwd.begin(), bwd.end());

  // ---- constant tables (double precision on the host, stored as float)
  fill_fft_tables(p->twiddle, p->ptw);
  // Taylor coefficients of F(e^s) = sum_{k<N} k e^{ks} = N^2 sum_j e_j (N s)^j,
  // e_j = sum_k (k/N)^(j+1) / (N j!)  (delay surrogate near its pole)
  {
    double fact = 1.0;
    for (int j = 0; j < 9; ++j) {
      if (j) fact *= j;
      double s = 0.0;
      for (int k = 0; k < p->dl_nd; ++k) s += std::pow(double(k) / p->dl_nd, j + 1);
      p->dl_taylor[j] = s / p->dl_nd / fact;
    }
  }
  // reverb frame window (periodic Hann) and DFT twiddles of its STFT size
  p->rv_win.resize(p->rv_n);
  p->rv_cs.resize(p->rv_n);
  for (int j = 0; j < p->rv_n; ++j) {
    const double a = 2.0 * M_PI * j / p->rv_n;
    p->rv_win[j] = float(0.5 - 0.5 * std::cos(a));
    p->rv_cs[j] = float2_{float(std::cos(a)), float(std::sin(a))};
  }
  // reverb band interpolation over the 513 STFT bins (same rule as the EQ's bands)
  {
    const int NB = RV_BANDS;
    double cb[RV_BANDS], lc[RV_BANDS];
    for (int b = 0; b < NB; ++b) {
      cb[b] = 20.0 * std::pow(1000.0, (b + 0.5) / NB);
      lc[b] = std::log2(cb[b]);
    }
    p->rv_band.assign(size_t(RV_BINS) * NB, 0.f);
    for (int k = 0; k < RV_BINS; ++k) {
      const double f = double(k) * opts.sample_rate / RV_N;
      float* row = p->rv_band.data() + size_t(k) * NB;
      if (f <= cb[0]) { row[0] = 1.f; continue; }
      if (f >= cb[NB - 1]) { row[NB - 1] = 1.f; continue; }
      int b = 0;
      while (b + 1 < NB && cb[b + 1] <= f) ++b;
      const double w = (std::log2(f) - lc[b]) / (lc[b + 1] - lc[b]);
      row[b] = float(1.0 - w);
      row[b + 1] = float(w);
    }
  }
  {
    const int Nt = p->eq_taps, H = p->eq_H;
    p->eq_cos.resize(Nt);
    for (int j = 0; j < Nt; ++j) p->eq_cos[j] = float(std::cos(2.0 * M_PI * j / Nt));
    p->eq_hann.resize(H + 1);
    for (int j = 0; j <= H; ++j) p->eq_hann[j] = float(0.5 * (1.0 + std::cos(2.0 * M_PI * j / (Nt + 1))));
    eq_band_table(Nt, opts.sample_rate, &p->eq_band);
  }

  // ---- loss plan over the output rows
  {
    const int Ms[N_RES] = {512, 1024, 2048};
    int64_t foff = 0, soff = 0;
    int32_t groups = 0;
    p->loss.ok = true;
    for (int32_t j = 0; j < int32_t(p->outputs_new.size()); ++j) {
      const NodeDev& nd = p->nodes[p->outputs_new[j]];
      LossRow r{};
      r.off = nd.off_y;
      r.len = nd.len;
      r.pitch = nd.pitch;
      if (nd.len < 2048) p->loss.ok = false;
      for (int q = 0; q < N_RES; ++q) {
        int M = Ms[q], hop = M / 4;
        int32_t F = nd.len >= M ? 1 + (nd.len - M) / hop : 0;
        r.n_frames[q] = F;
        r.frame_off[q] = foff;
        foff += int64_t(F) * 2 * M;
        r.spec_off[q] = soff;
        soff += int64_t(F) * 3 * (M / 2 + 1);
        r.group_off[q] = groups;
        const int per = 4096 / M;  // frames transformed together by one 256-thread CTA
        r.n_groups[q] = (F + per - 1) / per;
        for (int32_t f = 0, gi = 0; f < F; f += per, ++gi) p->loss.items.push_back({j, q, f, groups + gi});
        groups += r.n_groups[q];
      }
      p->loss.rows.push_back(r);
    }
    p->loss.frame_floats = foff;
    p->loss.spec_float2s = soff;
    p->loss.n_groups_total = groups;
  }

  // ---- workspace layout (every region 256-byte aligned)
  {
    WsLayout& w = p->ws;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    w.nodes = take(sizeof(NodeDev) * n);
    w.node_ext = take(sizeof(int4_) * n);
    w.csr_ptr = take(4 * size_t(n + 1));
    w.csr_src = take(4 * size_t(std::max(n_e, 1)));
    w.tcsr_ptr = take(4 * size_t(n + 1));
    w.tcsr_dst = take(4 * size_t(std::max(n_e, 1)));
    w.items = take(sizeof(int4_) * std::max<size_t>(p->items.size(), 1));
    w.csr_row = take(8 * size_t(std::max(n_e, 1)));
    w.tcsr_row = take(8 * size_t(std::max(n_e, 1)));
    w.in1_begin = take(4 * size_t(n));
    w.out1_begin = take(4 * size_t(n));
    w.twiddle = take(sizeof(float2_) * TWIDDLE_N);
    w.ptw = take(sizeof(float2_) * fft::PTW_TOTAL);
    w.eq_cos = take(4 * p->eq_cos.size());
    w.eq_hann = take(4 * p->eq_hann.size());
    w.eq_band = take(4 * p->eq_band.size());
    w.rv_band = take(4 * p->rv_band.size());
    w.rv_win = take(4 * p->rv_win.size());
    w.rv_cs = take(sizeof(float2_) * p->rv_cs.size());
    size_t nrow = std::max<size_t>(p->loss.rows.size(), 1);
    w.loss_rows = take(sizeof(LossRow) * nrow);
    w.loss_items = take(sizeof(int4_) * std::max<size_t>(p->loss.items.size(), 1));
    w.tables_end = o;
    // cleared at the start of every render / backprop
    w.status = take(16);
    w.tickets = take(4 * size_t(2 * (N + 2)));
    w.flags = take(8 * std::max<size_t>(p->items.size(), 1));   // look-back words of small compressor steps
    w.flags_bytes = o - w.status;
    w.eq_spec = take(4 * size_t(std::max(p->n_eq, 1)) * (p->eq_fft / 2 + 4));   // 16-byte aligned rows
    w.eq_aux = take(4 * size_t(std::max(p->n_eq, 1)) * 1024);
    w.eq_bandpart = take(4 * size_t(std::max(p->n_eq, 1)) * 16 * 8);
    w.comp_carry = take(4 * size_t(std::max(p->n_comp_chunks, 1)));
    w.dl_aux = take(4 * size_t(std::max(p->n_delay, 1)) * 2 * p->dl_taps * (DL_FIR + 1));
    w.dl_spec = take(8 * size_t(std::max(p->n_dl_slots, 1)) * DL_M);
    w.dl_R = take(8 * size_t(std::max(p->n_delay, 1)) * p->dl_P * DL_M);
    w.dl_r = take(4 * size_t(std::max(p->n_delay, 1)) * 2 * p->dl_P * DL_B);
    const size_t nr = size_t(std::max(p->n_reverb, 1));
    const size_t rbins = size_t(p->rv_n / 2 + 1);
    w.rv_U = take(8 * size_t(2) * p->rv_f * rbins);
    w.rv_fr = take(8 * nr * p->rv_f * p->rv_n);
    w.rv_h = take(4 * nr * 2 * RV_HLEN);
    w.rv_H = take(8 * nr * RV_P * DL_M);
    w.rv_Y = take(8 * nr * size_t(std::max(p->rv_nbmax, 1)) * DL_M);
    w.rv_R = take(8 * nr * RV_P * DL_M);
    w.rv_r = take(4 * nr * 2 * RV_HLEN);
    w.rv_mm = take(8 * nr * p->rv_f * 2 * rbins);
    w.rv_lm = take(4 * nr * 4 * size_t(RV_BINS));
    w.rv_dot = take(4 * nr * size_t(RV_P));
    w.partial = take(16 * size_t(std::max(p->n_partials, 1)));
    w.eq_partial = take(8 * size_t(std::max(p->n_eq_runs, 1)) * (p->eq_fft / 2 + 1));
    w.eq_uspec = take(8 * size_t(std::max<int64_t>(p->n_eq_blocks, 1)) * p->eq_fft);
    w.eq_ola = take(4 * size_t(std::max<int64_t>(p->n_eq_blocks, 1)) * 4 * size_t(std::max(p->eq_H, 1)));
    w.loss_part = take(32 * size_t(std::max(p->loss.n_groups_total, 1)));
    w.loss_stats = take(32 * nrow * N_RES);
    w.loss_rowloss = take(4 * nrow);
    w.loss_frames = take(4 * size_t(std::max<int64_t>(p->loss.frame_floats, 1)));
    w.loss_spec = take(8 * size_t(std::max<int64_t>(p->loss.spec_float2s, 1)));
    {
      int64_t fl = 0;
      for (int t = 0; t < GRAFX_N_TYPES; ++t) {
        p->dgrad_off[t] = fl;
        if (p->source_batch > 1) fl += int64_t(p->n_rows_union[t]) * p->pcols[t];
      }
      w.dgrad = take(4 * size_t(std::max<int64_t>(fl, 1)));
    }
    w.bal = take(4 * size_t(std::max<int64_t>(p->bal_floats, 1)));
    w.U = take(4 * size_t(std::max<int64_t>(u_floats, 1)));
    w.A = take(4 * size_t(std::max<int64_t>(a_floats, 1)));
    w.total = o;
  }
  return GRAFX_OK;
}

}  // namespace grafx
