// Host-side plan: the render data of Algorithm 1 (schedule, reordering, index maps)
// plus the device work lists and workspace layout for the sm_103a kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/grafx.h"
#include "devtypes.h"

struct grafx_graph {
  std::vector<int32_t> types;
  std::vector<std::pair<int32_t, int32_t>> edges;
  std::vector<std::pair<int32_t, int32_t>> ports;   // per edge: (output of src, input of dst)
};

namespace grafx {

// Inputs M and outputs N of a node type (Eq. 1a).
inline int type_inputs(int t) {
  return t == GRAFX_T_IN ? 0 : (t == GRAFX_T_MERGE || t == GRAFX_T_SIDECHAIN) ? 2 : 1;
}
inline int type_outputs(int t) { return t == GRAFX_T_SPLIT ? 2 : 1; }

// status helpers (thread-local last error)
int fail(int code, const std::string& msg);
void clear_error();
const char* last_error_cstr();

struct Schedule {
  std::vector<int32_t> string;              // type string t_0..t_N
  std::vector<std::vector<int32_t>> steps;  // V_0..V_N, original ids ascending
};

// Graph rules of Sec. 2 "Definitions"; returns GRAFX_OK or an error code (message set).
int validate(const std::vector<int32_t>& types, const std::vector<std::pair<int32_t, int32_t>>& edges);
// Type schedules of Sec. 2 "Type scheduling".
int make_schedule(const std::vector<int32_t>& types, const std::vector<std::pair<int32_t, int32_t>>& edges,
                  int method, int beam_width, int n_threads, Schedule* out);

struct StepInfo {
  int32_t type;
  int32_t node_begin, node_end;    // new ids [begin, end)
  int32_t fitem_begin, fitem_count;  // forward work items (global index)
  int32_t bitem_begin, bitem_count;  // backward work items (global index)
  int32_t dsub_begin[5], dsub_count[5];  // delay backward sub-lists: adjoint, spectra, acc, lags, grads
  // 1: gain/imager step whose every node feeds exactly one node of the next step (also
  // gain/imager, each with that single input): the two steps run as one fused kernel;
  // 2: gain step whose every node is the single input of one EQ node of the next step,
  // and feeds only it: the EQ forward applies the gain on load (backward unfused);
  // 3: mix step whose every node is the single input of one output node of the next
  // step: one forward kernel writes both rows (outputs have no backward step)
  int32_t fuse_next = 0;
  // every in-edge of the step's nodes comes from an input node: without requested source
  // adjoints the step's input adjoints have no reader
  int32_t in_from_sources = 0;
};

// Byte offsets of the regions inside the caller's workspace.
struct WsLayout {
  size_t nodes, node_ext, csr_ptr, csr_src, tcsr_ptr, tcsr_dst, items;
  size_t csr_row, tcsr_row, in1_begin, out1_begin;
  size_t twiddle, ptw, eq_cos, eq_hann, eq_band, rv_win, rv_cs;
  size_t loss_rows, loss_items;
  size_t tables_end;                           // [0, tables_end) is uploaded at bind time
  size_t status, tickets, flags, flags_bytes;  // flags_bytes covers status+tickets+flags (cleared per call)
  size_t eq_spec, eq_aux, eq_bandpart, comp_carry, partial, eq_partial;
  size_t eq_uspec, eq_ola;                     // EQ input block spectra (forward), adjoint heads/tails
  size_t dl_aux, dl_spec, dl_R, dl_r;
  size_t rv_band, rv_U, rv_fr, rv_h, rv_H, rv_Y, rv_R, rv_r, rv_mm;
  size_t rv_lm, rv_dot;                        // per reverb node: band-interpolated H0/Hd, h.r partials
  size_t loss_part, loss_stats, loss_rowloss, loss_frames, loss_spec;
  size_t dgrad;                                // per-copy parameter gradients (source batch)
  size_t bal;                                  // ballistic scratch rows
  size_t U, A;
  size_t total;
};

struct LossPlan {
  // per output row j
  std::vector<LossRow> rows;
  // work items (row, resolution, first frame, statistics group)
  std::vector<int4_> items;
  int64_t frame_floats = 0;  // total floats in the frame buffer
  int64_t spec_float2s = 0;  // total float2 in the spectrum cache (forward -> backward)
  int32_t n_groups_total = 0;
  bool ok = false;           // every output row is long enough (>= 2048 samples)
};

struct Plan {
  grafx_plan_opts opts;
  int32_t n_graphs = 0;
  std::vector<int64_t> L, pitch;         // per graph
  std::vector<int32_t> types;            // union, original ids
  std::vector<std::pair<int32_t, int32_t>> edges;
  std::vector<std::pair<int32_t, int32_t>> ports;   // per edge (output k of src, input l of dst)
  // per new id: first in-edge of input 1 and first consumer edge of output 1 (the ends
  // of the nodes' edge ranges when they have a single input / output)
  std::vector<int32_t> in1_begin, out1_begin;
  // per edge in CSR order: the source's output row; per edge in consumer-CSR order: the
  // consumer's input-adjoint row (row references: NodeKind << 60 | float offset)
  std::vector<int64_t> csr_row, tcsr_row;
  std::vector<int32_t> node_graph;       // original id -> graph
  Schedule sched;
  std::vector<int32_t> step_ptr, sigma, csr_ptr, csr_src, tcsr_ptr, tcsr_dst, param_row;
  std::vector<int32_t> new_types;
  std::vector<NodeDev> nodes;            // new ids
  // per node: x = first partial slot (gain/imager/compressor) or first EQ run,
  // y = number of slots / runs, z = EQ spectrum index or first compressor chunk id
  std::vector<int4_> node_ext;
  std::vector<StepInfo> steps;           // index 1..N (steps[0] unused: inputs)
  std::vector<int4_> items;              // all work items, forward lists then backward lists
  int32_t n_type_rows[GRAFX_N_TYPES] = {0};
  int32_t n_eq = 0, n_comp_chunks = 0, n_partials = 0, n_eq_runs = 0;
  int64_t n_eq_blocks = 0;               // overlap-save blocks of all EQ nodes
  int32_t n_fitems = 0, in_bitem_begin = 0, in_bitem_count = 0;
  int32_t n_delay = 0, n_dl_slots = 0, n_reverb = 0, rv_nbmax = 0, dl_nbmax = 0;
  int32_t n_bal = 0;                     // ballistic nodes
  int64_t bal_floats = 0;                // their scratch (mid, envelope, adjoint, coefficient per sample)
  double dl_taylor[9] = {0};
  int32_t eq_taps = 1023, eq_H = 511, eq_fft = 4096, eq_step = 0;  // eq_step: outputs per block
  int32_t comp_chunk = 2048;
  // processor layouts (grafx_plan_opts eq_params, delay_layout, reverb_layout)
  int32_t eq_logmag = 0;
  int32_t dl_taps = DL_TAPS, dl_nd = DL_NFFT, dl_slot = 0, dl_P = 10;
  int32_t rv_paper = 0, rv_n = RV_N, rv_hop = RV_HOP, rv_f = RV_F;
  int32_t pcols[GRAFX_N_TYPES] = {0};    // columns of P[t]
  // source-level batch: B copies of the graphs (copy-major); n_type_rows counts one copy
  int32_t source_batch = 1, graphs_per_copy = 0;
  int32_t n_rows_union[GRAFX_N_TYPES] = {0};
  int64_t dgrad_off[GRAFX_N_TYPES] = {0};  // float offsets of the per-copy gradient tables (B > 1)
  std::vector<int32_t> grad_row;         // per new id: row of the per-copy gradient table
  int32_t ckpt_steps = 0;                // signal checkpointing: steps per segment (0 = off)
  std::vector<int32_t> seg_ptr;          // first step of each segment, then N + 1
  int64_t src_elems = 0, out_elems = 0, node_samples = 0;
  std::vector<int64_t> src_graph_off, out_graph_off;
  std::vector<int32_t> outputs_new;      // new ids of output rows in order
  LossPlan loss;
  WsLayout ws;
  // host tables
  std::vector<float2_> twiddle, ptw;
  std::vector<float> eq_cos, eq_hann, eq_band, rv_band, rv_win;
  std::vector<float2_> rv_cs;            // (cos, sin)(2 pi j / rv_n): the reverb's frame DFTs
  // bindings
  char* dev_ws = nullptr;
  const float* params[GRAFX_N_TYPES] = {nullptr};
  const float* rv_noise = nullptr;
  int64_t param_rows[GRAFX_N_TYPES] = {0};
  int32_t last_launches = 0;
  // side stream (cudaStream_t) and events (cudaEvent_t) for work off the critical path:
  // parameter-only designs in the forward, parameter-gradient finalizers in the backward
  void* side = nullptr;
  std::vector<void*> events;             // [0] fork, [1] join, [2 + k] forward step k, [2 + N + 1 + k] backward step k
};

int build_plan(const std::vector<const grafx_graph*>& graphs, const int64_t* lengths,
               const grafx_plan_opts& opts, Plan* p);

// Twiddle table exp(-2 pi i m / TWIDDLE_N) and the per-pass FFT twiddle tables (fft.cuh)
void fill_fft_tables(std::vector<float2_>& twiddle, std::vector<float2_>& ptw);

inline int64_t pitch_of(int64_t L) { return (L + 3) & ~int64_t(3); }

}  // namespace grafx

struct grafx_plan : public grafx::Plan {};
