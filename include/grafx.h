/*
 * grafx.h - C ABI of the B300 (sm_103a) GRAFX graph renderer.
 *
 * The library renders audio-processing graphs (arxiv 2408.03204, "GRAFX"):
 * directed acyclic graphs of stereo processors, forward and backward.  The calls
 * follow the paper's problem statement and its Fig. 2a usage: build a graph
 * (GRAFX(), add, add_serial_chain, connect), compute the render data
 * (compute_render_data: the ScheduleBatchedProcessing, OptimizeNodeOrder, Reorder
 * and GetReadWriteIndex steps of Algorithm 1), bind parameters, render (its Initialize
 * step, then per schedule step Gather, Aggregate, Process and Store) and
 * backpropagate.
 *
 * Conventions
 *  - Every call returns an int status: GRAFX_OK (0) or a GRAFX_E* code.  On error
 *    grafx_last_error() returns a message for the calling thread.
 *  - Handles (grafx_graph, grafx_plan) are opaque and owned by the library; they
 *    are freed with the matching *_destroy call.
 *  - Device memory is owned by the caller.  The library allocates no device memory
 *    in any call of this header; the caller passes a workspace of
 *    grafx_plan_info.ws_bytes bytes (256-byte aligned) and binds it once.
 *  - Streams are passed as void* and must be a cudaStream_t (NULL = legacy default
 *    stream).  Device work is asynchronous on that stream; a plan must be used on
 *    one stream at a time.  Device-side failures (a bounded wait that expired, an
 *    index out of range) set a status word in the workspace that
 *    grafx_sync_status() reports.
 *  - Signals are float32 stereo rows laid out [channel][pitch] with
 *    pitch = grafx_pitch(L) = L rounded up to a multiple of 4.  Samples at and past
 *    L inside a row are padding: ignored on input, written as 0 on output.
 *  - Node type ids: see GRAFX_T_*.  Parameter widths per type (columns of P[t]):
 *    gain 2, imager 1, compressor 4, noisegate 4, sidechain 4, ballistic 5, split and merge none;
 *    eq 8, delay 176, reverb 50 in the
 *    compact layouts, eq (eq_taps+1)/2, delay 880, reverb 768 in the paper's
 *    (grafx_plan_opts, grafx_plan_info.param_cols, grafx_bind_params).
 */
#ifndef GRAFX_H
#define GRAFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  GRAFX_OK = 0,
  GRAFX_EINVAL = 1,    /* bad argument or graph rule broken (Sec. 2 Definitions) */
  GRAFX_ECYCLE = 2,    /* graph has a cycle (Sec. 2: feedback loops are not allowed) */
  GRAFX_ESHAPE = 3,    /* size / length / parameter-table shape mismatch */
  GRAFX_ETYPE = 4,     /* unknown or unsupported node type */
  GRAFX_ENOMEM = 5,    /* host allocation failed */
  GRAFX_ECUDA = 6,     /* a CUDA runtime call failed */
  GRAFX_ETIMEOUT = 7,  /* a bounded device-side wait expired (reported by grafx_sync_status) */
  GRAFX_ESTATE = 8     /* call out of order (e.g. render before bind_workspace) */
};

/* ---------------------------------------------------------------- node types
 * Letters of the paper (Fig. 1 and Fig. 2b legends).  in/out are the graph inputs
 * and outputs; mix is an identity node whose input is the sum of its in-edges. */
enum {
  GRAFX_T_IN = 0, GRAFX_T_OUT = 1, GRAFX_T_MIX = 2, GRAFX_T_GAIN = 3, GRAFX_T_IMAGER = 4,
  GRAFX_T_EQ = 5, GRAFX_T_COMP = 6, GRAFX_T_DELAY = 7, GRAFX_T_REVERB = 8, GRAFX_T_GATE = 9,
  /* multi-port processors (Sec. 2 Definitions, Eq. 1a with M inputs and N outputs):
   * SPLIT: 1 input, 2 outputs (port 0 = (m, m), port 1 = (s, s), m = (l + r)/2,
   *        s = (l - r)/2); MERGE: 2 inputs (0 = mid path, 1 = side path), 1 output
   *        (u0_l + u1_l, u0_r - u1_r), the inverse of SPLIT; SIDECHAIN: the compressor
   *        of Eq. 8-12 with 2 inputs (0 = main, 1 = key): the envelope follows the key,
   *        the gain applies to the main input. */
  GRAFX_T_SPLIT = 10, GRAFX_T_MERGE = 11, GRAFX_T_SIDECHAIN = 12,
  /* the compressor with attack/release ballistics (Eq. 8 with alpha[n] = alpha_attack while
   * the envelope rises, alpha_release while it falls; the recursion is sample-serial) */
  GRAFX_T_BALLISTIC = 13,
  GRAFX_N_TYPES = 14
};

/* Inputs M and outputs N of a node type (GRAFX_EINVAL for an unknown type): sources
 * 0 x 1, SPLIT 1 x 2, MERGE and SIDECHAIN 2 x 1, every other type 1 x 1. */
int grafx_type_ports(int32_t type, int32_t* n_inputs, int32_t* n_outputs);

/* ---------------------------------------------------------------- schedules (Sec. 2 "Type scheduling") */
enum {
  GRAFX_SCHED_BEAM = 0,       /* beam search keeping beam_width partial schedules */
  GRAFX_SCHED_GREEDY = 1,     /* type with the most computable nodes; ties -> smallest type id */
  GRAFX_SCHED_OPTIMAL = 2,    /* exhaustive shortest schedule; tiny graphs only (<= 28 processing nodes) */
  GRAFX_SCHED_ONE_BY_ONE = 3  /* one processing node per step (the paper's baseline) */
};

typedef struct grafx_graph grafx_graph;
typedef struct grafx_plan grafx_plan;

/* Message for the last failed call on this thread ("" if none).  Owned by the
 * library; valid until the next call on this thread. */
const char* grafx_last_error(void);

/* L rounded up to a multiple of 4: the channel stride of every signal row. */
int64_t grafx_pitch(int64_t L);

/* ---------------------------------------------------------------- graph building
 * Sec. 2 "Graph representations" and Fig. 2a: a mutable graph G = (V, E).  Node ids
 * are assigned in insertion order from 0.  Edges are SISO "cables" (Eq. 1b): the
 * input of a node is the sum of the outputs of its in-edges; repeated edges add
 * the same signal again.  Rules are checked when a plan is created: inputs have no
 * in-edges, every other node has at least one, outputs have no out-edges, there is
 * at least one output, and there is no cycle. */
int grafx_graph_create(grafx_graph** out);
int grafx_graph_destroy(grafx_graph* g);
/* Append a node of `type` (GRAFX_T_*); its id is written to *id_out. */
int grafx_graph_add(grafx_graph* g, int32_t type, int32_t* id_out);
/* Append n nodes of types[0..n) connected in series; first/last ids are returned. */
int grafx_graph_add_serial_chain(grafx_graph* g, const int32_t* types, int32_t n,
                                 int32_t* first_id, int32_t* last_id);
/* Append the edge src -> dst (ids must exist): output 0 of src to input 0 of dst. */
int grafx_graph_connect(grafx_graph* g, int32_t src, int32_t dst);
/* Append the edge from output `src_port` of src to input `dst_port` of dst: the edge
 * type t_ij = (k, l) of Sec. 2 (the edge type tensor T_E).  Input l of a node is the
 * sum of the signals on its edges into l; an input with no edge reads zeros.  Ports
 * are checked against grafx_type_ports when a plan is created (GRAFX_EINVAL). */
int grafx_graph_connect_ports(grafx_graph* g, int32_t src, int32_t dst, int32_t src_port, int32_t dst_port);
int grafx_graph_size(const grafx_graph* g, int32_t* n_nodes, int32_t* n_edges);

/* ---------------------------------------------------------------- planning
 * compute_render_data: the ScheduleBatchedProcessing, OptimizeNodeOrder, Reorder and
 * GetReadWriteIndex steps of Algorithm 1, on the host.  Several graphs may be
 * planned together; they are treated as one disconnected graph (graph-level
 * parallelism, Sec. 2 "Batched processing"), each with its own signal length.
 * Node ids of the union are the per-graph ids offset by the node counts of the
 * graphs before it; the k-th input of the union reads source row k, the j-th
 * output writes output row j, and the l-th node of type t in the union owns row l
 * of that type's parameter table. */
typedef struct {
  int32_t schedule;       /* GRAFX_SCHED_*; default BEAM */
  int32_t beam_width;     /* default 32 (the paper's Sec. 4 setting) */
  int32_t eq_taps;        /* odd FIR length N of the zero-phase EQ (Eq. 4); default 1023 */
  int32_t sample_rate;    /* Hz, for the EQ band centres; default 44100 */
  int32_t n_threads;      /* host threads for planning; 0 = hardware concurrency */
  int32_t eq_fft;         /* EQ block FFT size (1024..8192, at least 2 eq_taps + 2); 0 = default */
  int32_t comp_chunk;     /* compressor scan chunk (1024, 2048 or 4096 samples); 0 = default */
  int32_t checkpoint_steps; /* signal checkpointing: 0 = off (every node row kept from the
                             * forward to the backward pass); k > 0 = the schedule steps are
                             * cut into segments of k steps, only rows read by a later
                             * segment are kept, the other rows of all segments share one
                             * scratch region, and grafx_backprop recomputes the forward of
                             * every segment but the last before running its backward
                             * (smaller workspace, one extra forward of steps 1..N-k). */
  int32_t eq_params;      /* GRAFX_EQ_*: what a row of P[eq] holds (default BANDS) */
  int32_t delay_layout;   /* GRAFX_DELAY_*: taps of the multitap delay (default COMPACT) */
  int32_t reverb_layout;  /* GRAFX_REVERB_*: STFT and masks of the reverb (default COMPACT) */
  int32_t source_batch;   /* source-level batch B (Sec. 2 "Batched processing"): 0 or 1 = none;
                           * B > 1 renders the graphs B times on B source sets with the same
                           * parameters.  Sources and outputs are [B][the rows of one pass]
                           * (copy-major); parameter tables keep the rows of one pass and
                           * their gradients are summed over the B copies in copy order. */
  int32_t reserved[4];
} grafx_plan_opts;

/* Processor settings (Sec. 3).  The COMPACT layouts are small parameter sets for
 * fitting and batching; the PAPER layouts are the paper's own settings. */
enum {
  GRAFX_EQ_BANDS = 0,     /* 8 band gains in dB, interpolated in log2 frequency onto the
                           * (eq_taps+1)/2 log-magnitudes: 8 columns */
  GRAFX_EQ_LOGMAG = 1     /* the (eq_taps+1)/2 natural-log magnitudes p_e[k] of Eq. 4
                           * themselves (eq_taps = 2047 -> 1024 columns, the paper's EQ) */
};
enum {
  GRAFX_DELAY_COMPACT = 0, /* 4 taps per channel, each delay anywhere in [0, 32768)
                            * samples (surrogate length N_d = 32768): 176 columns */
  GRAFX_DELAY_SLOTS = 1    /* the paper's 2 s delay: 20 taps per channel, tap m in its own
                            * 100 ms slot [m S, m S + S), S = sample_rate / 10, surrogate
                            * length N_d = S: 880 columns */
};
enum {
  GRAFX_REVERB_COMPACT = 0, /* STFT 1024 / hop 256, masks from 12 log-spaced bands, dry and
                             * wet gains: 50 columns */
  GRAFX_REVERB_PAPER = 1    /* STFT 384 / hop 192, masks from 192 log-magnitudes per filter
                             * (bins 0..191; the Nyquist bin is dropped), wet output only:
                             * 768 columns */
};

void grafx_plan_opts_default(grafx_plan_opts* o);

/* graphs[0..n_graphs) with lengths[g] samples each (1 <= L <= 2^24).  The graphs
 * are copied; they may be destroyed after this call.  Errors: EINVAL, ECYCLE,
 * ETYPE, ESHAPE (graphs with delay or reverb nodes are limited to 2^19 samples). */
int grafx_plan_create(const grafx_graph* const* graphs, int32_t n_graphs, const int64_t* lengths,
                      const grafx_plan_opts* opts, grafx_plan** out);
int grafx_plan_destroy(grafx_plan* p);

typedef struct {
  int32_t n_graphs, n_nodes, n_edges;
  int32_t n_steps;            /* N: the schedule is V_0..V_N */
  int32_t n_inputs, n_outputs;
  int32_t n_type_rows[GRAFX_N_TYPES];  /* |V_t| per type */
  int64_t src_elems;          /* floats in the source buffer: sum_g K_g * 2 * pitch_g */
  int64_t out_elems;          /* floats in the output buffer: sum_g |O_g| * 2 * pitch_g */
  int64_t node_samples;       /* sum over processing (non-input) nodes of L */
  size_t ws_bytes;            /* device workspace bytes (render + backprop + loss) */
  int32_t eq_fft, comp_chunk; /* the tile sizes in use */
  int32_t param_cols[GRAFX_N_TYPES];  /* columns of P[t] under the plan's layouts (0: none) */
  int32_t source_batch;       /* B (1 without a source batch); n_graphs, n_nodes, n_edges,
                               * n_inputs, n_outputs, src_elems, out_elems and node_samples
                               * count all B copies, n_type_rows one copy */
  int32_t fused_pairs;        /* schedule steps k fused with step k+1: every node of k+1 has one
                               * input, a node of k whose only consumer it is, and the types are
                               * gain/imager then gain/imager (forward and backward fused), gain
                               * then EQ (the EQ forward applies the gain on load) or mix then
                               * output (one forward kernel writes both rows).  A render or
                               * backprop whose step range holds both steps runs them as one
                               * kernel (same results, bit for bit; the intermediate rows are
                               * written forward, the intermediate adjoint rows of a gain/imager
                               * pair are not); never with checkpointing */
} grafx_plan_info_t;

int grafx_plan_info(const grafx_plan* p, grafx_plan_info_t* info);

/* Copy the plan's host index maps out (for checking them bit for bit).  Any pointer
 * may be NULL.  Sizes: type_string N+1, step_ptr N+2, sigma |V| (original id of the
 * union -> new id), csr_ptr |V|+1, csr_src |E| (in-edges by (dst, src) in new ids:
 * I^G / I^A), tcsr_ptr |V|+1, tcsr_dst |E| (consumers by (src, dst)), param_row |V|
 * (row of P[t] owned by each new id: I^P). */
int grafx_plan_export(const grafx_plan* p, int32_t* type_string, int32_t* step_ptr,
                      int32_t* sigma, int32_t* csr_ptr, int32_t* csr_src,
                      int32_t* tcsr_ptr, int32_t* tcsr_dst, int32_t* param_row);
/* Copy the work items of schedule step `step` (1..N) out: the forward ones (backward = 0)
 * or the backward ones (backward = 1), each 4 int32 (new node id, then three fields whose
 * meaning is per processor type: for the compressor, noisegate and sidechain the chunk
 * index, the chunk's global id and (backward) its partial slot), in launch order, into
 * items (host, 4 * capacity int32; may be NULL).  *count receives the step's item count;
 * GRAFX_ESHAPE if it exceeds capacity (items is then not written).  For checking the
 * planner's orders; the render never needs it. */
int grafx_plan_step_items(const grafx_plan* p, int32_t step, int32_t backward, int32_t* items, int32_t capacity,
                          int32_t* count);

/* ---------------------------------------------------------------- device binding
 * Bind a caller-owned device workspace of at least info.ws_bytes bytes (256-byte
 * aligned) and upload the plan's tables into it.  Blocks until the upload is done.
 * The workspace holds the intermediate tensor U (Algorithm 1) and the adjoints, so
 * it must stay untouched between a render and the backprop that follows it.  The first
 * binding in a process also sets the kernels' attributes and launch shapes (shared-
 * memory limits, resident CTAs per SM); call it outside any stream capture. */
int grafx_plan_bind_workspace(grafx_plan* p, void* dev_ws, size_t bytes, void* stream);

/* Bind the parameter table P[type]: a device float32 array [rows][cols], row-major,
 * rows = |V_type| in the union's original node order (Sec. 2: the l-th row belongs
 * to the l-th node of that type), cols = the type's width.  The pointer is kept and
 * read at every render/backprop, so values may change in place between calls.
 * Physical units: gain [ln g_l, ln g_r] (Eq. 2); imager [p_s] (Eq. 3); eq 8 band
 * gains in dB at 20*1000^((b+0.5)/8) Hz (Eq. 4, log-frequency interpolation);
 * compressor [alpha, T, W, R] with T, W in natural-log energy (Eq. 8-12), W > 0;
 * delay 176 = [channel l, r][tap 0..3][Re z, Im z, 20 log-magnitudes of its 39-tap
 * zero-phase FIR] (Eq. 14-15): the forward pass delays by round(32768 (-arg z)/2pi)
 * mod 32768 samples, the backward pass takes the z-gradient of the surrogate of Eq. 15;
 * reverb 50 = [mid, side][H0 (12 bands), Hd (12 bands)] natural-log magnitudes and
 * per-frame decays of the noise masks (Eq. 7), then q_dry, q_wet (log gains):
 * y = e^{q_dry} u + e^{q_wet} (h * u) with the 88200-tap IR h of Eq. 6-7;
 * noisegate [alpha, T, W, R] like the compressor, with the gate curve of Eq. 13
 * (unchanged above T + W, expansion by R below T - W, a quadratic knee between);
 * sidechain [alpha, T, W, R] as the compressor, the envelope taken from input 1;
 * ballistic [alpha_attack, alpha_release, T, W, R]: the compressor with the coefficient
 * of Eq. 8 switched per sample by whether the envelope rises (x[n] > g[n-1]).
 * Paper layouts: eq (eq_taps+1)/2 = the log-magnitudes p_e[k] of Eq. 4 (GRAFX_EQ_LOGMAG);
 * delay 880 = [channel][tap 0..19][Re z, Im z, 20 log-magnitudes], tap m delayed by
 * m S + (round(S (-arg z)/2pi) mod S), S = sample_rate/10, the surrogate of Eq. 15 of
 * length S placed at the slot (GRAFX_DELAY_SLOTS); reverb 768 = [mid, side][H0 (192),
 * Hd (192)] per-bin log-magnitudes of the masks on bins 0..191 of the 384-point STFT
 * (hop 192), the Nyquist bin masked to 0, y = h * u (GRAFX_REVERB_PAPER).
 * cols must equal grafx_plan_info.param_cols[type]; otherwise GRAFX_ESHAPE. */
int grafx_bind_params(grafx_plan* p, int32_t type, const float* dev, int64_t rows, int64_t cols);

/* Bind the two noise buffers of the filtered-noise reverb (Sec. 3 "Reverb", Eq. 6-7):
 * device float32 [2][88200] (mid, side; 2 s at 44.1 kHz), shared by every reverb node;
 * kept by pointer.  Required when the plan has reverb nodes. */
int grafx_bind_reverb_noise(grafx_plan* p, const float* dev, int64_t n);

/* ---------------------------------------------------------------- render / backprop
 * grafx_render: the render of Algorithm 1 (Initialize; per schedule step Gather,
 * Aggregate, Process, Store).  sources: device float32 holding, graph after
 * graph, K_g rows of [2][pitch_g] (src_elems floats).  out: device float32 of
 * out_elems floats, the rows of the output nodes (Y_N).  Input rows are read in
 * place (U = S (+) 0 without a copy); output rows are written in place. */
int grafx_render(grafx_plan* p, const float* sources, float* out, void* stream);

/* Reverse-mode pass of the last render (same sources, workspace untouched).
 * d_out: dLoss/dY, laid out like `out`.  d_params[t] (t < GRAFX_N_TYPES): device
 * float32 [rows][cols] like P[t], overwritten with dLoss/dP[t]; NULL entries (and
 * types without parameters) are skipped, but every bound type with a non-NULL
 * entry is written completely.  d_sources: NULL or a buffer like `sources`,
 * overwritten with dLoss/dS. */
int grafx_backprop(grafx_plan* p, const float* sources, const float* d_out,
                   float* const* d_params, float* d_sources, void* stream);

/* Run only the schedule steps k in [first, last) of the render (1 <= first <= last <= N+1),
 * in order; grafx_render is first = 1, last = N+1.  Used to time or re-run individual
 * steps (Algorithm 1 iterations). */
int grafx_render_steps(grafx_plan* p, const float* sources, float* out, int32_t first, int32_t last,
                       void* stream);
/* Backward over the steps k in [first, last) in reverse order (0 <= first <= last <= N+1);
 * k = 0 stands for the source adjoints (written only if d_sources is not NULL).
 * Without checkpointing grafx_backprop is first = 0, last = N+1.  With checkpointing
 * the node rows of a step are valid only while its segment is the one rendered last,
 * so a range must lie in that segment (grafx_backprop orders this itself).  With a
 * source batch (B > 1) only the whole range first = 0, last = N+1 is accepted (the
 * gradients of the copies are summed after the last step); otherwise GRAFX_ESTATE. */
int grafx_backprop_steps(grafx_plan* p, const float* sources, const float* d_out, float* const* d_params,
                         float* d_sources, int32_t first, int32_t last, void* stream);

/* ---------------------------------------------------------------- loss
 * Multi-resolution STFT magnitude loss between the output rows and a target laid
 * out like `out` (the paper fits a rendered mix to a target, Sec. 4 Example usage;
 * the loss itself is not specified there).  Per row and resolution M in
 * {512, 1024, 2048}, hop M/4, periodic Hann, frames at f*hop with no padding, per
 * channel: ||(|Y|-|T|)||_F / ||T||_F + mean|ln(|Y|+1e-7) - ln(|T|+1e-7)| over bins
 * 0..M/2; averaged over the 6 (resolution, channel) pairs and summed over rows.
 * Every output length must be >= 2048.  loss: device float32 scalar (written). */
int grafx_mrstft_forward(grafx_plan* p, const float* out, const float* target, float* loss,
                         void* stream);
/* dLoss/dout into d_out (laid out like out; overwritten).  Uses the statistics and
 * the per-bin spectra that the last grafx_mrstft_forward on the same plan stored in the
 * workspace, which must have been run on the same out and target. */
int grafx_mrstft_backward(grafx_plan* p, const float* out, const float* target, float* d_out,
                          void* stream);

/* ---------------------------------------------------------------- status
 * Synchronise `stream` and report device-side failures recorded since the last
 * call (GRAFX_ETIMEOUT for an expired bounded wait, GRAFX_EINVAL for an index that
 * a device bounds check rejected), then clear them. */
int grafx_sync_status(grafx_plan* p, void* stream);

/* Number of kernel launches issued by the most recent grafx_render / grafx_backprop /
 * grafx_mrstft_* call on this plan (for launch accounting). */
int grafx_last_launch_count(const grafx_plan* p, int32_t* n);

/* ---------------------------------------------------------------- one fit step as a CUDA graph
 * Batched rendering replays a fixed launch sequence per plan (Sec. 2 "Batched
 * processing": the schedule and index maps are computed once), so a whole step --
 * render, loss, loss gradient and backprop, with the buffers given here -- is
 * recorded once into a CUDA graph and replayed with one launch.  The buffers and the
 * bound parameters are baked in: replays read their current contents.  d_params and
 * d_sources follow grafx_backprop.  Create runs no kernel itself (it captures on
 * `stream`, which must not be the legacy NULL stream: EINVAL); the graph is owned by the library until grafx_step_graph_destroy. */
typedef struct grafx_step_graph grafx_step_graph;
int grafx_step_graph_create(grafx_plan* p, const float* sources, float* out, const float* target, float* loss,
                            float* d_out, float* const* d_params, float* d_sources, void* stream,
                            grafx_step_graph** out_graph);
int grafx_step_graph_launch(grafx_step_graph* g, void* stream);
/* Number of kernels one replay launches. */
int grafx_step_graph_launches(const grafx_step_graph* g, int32_t* n);
int grafx_step_graph_destroy(grafx_step_graph* g);

/* ---------------------------------------------------------------- fitting (Adam)
 * Gradient descent on every processor's parameters (Abstract; Sec. 4 "Example usage").
 * The optimiser works on unconstrained theta; the processors see p = map(theta),
 * element-wise by a per-column code (codes[i % cols]):
 *   0 identity; 1 alpha = 0.9 + 0.0999 sigmoid(theta); 2 softplus(theta);
 *   3 1 + softplus(theta); 4 -softplus(theta); 5 attack coefficient
 *   0.5 + 0.4999 sigmoid(theta); 6, 7 a multitap delay tap's Re z and Im z (identity
 *   maps; a 6 must be followed by a 7 in the same row).
 * A (6, 7) pair is updated together (Sec. 3 "Multitap delay", after Eq. 15: the paper
 * normalises the surrogate's z-gradient and pulls z towards the unit circle): its
 * gradient 2-vector is scaled to unit length (zero stays zero) and the gradient of the
 * penalty 1e-2 (|z| - 1)^2 at the old z is added before the Adam moments.
 * grafx_adam_step: one Adam update (bias-corrected, step >= 1) of n elements, in place:
 * theta, m, v (device float32, m and v zero before step 1) and param (written with
 * map(theta_new)); grad_param = dLoss/dp from grafx_backprop at the old param.
 * codes: device int8[cols].  Asynchronous on `stream`. */
int grafx_adam_step(float* theta, float* m, float* v, const float* grad_param, float* param,
                    const int8_t* codes, int32_t cols, int64_t n, int32_t step, float lr, float beta1,
                    float beta2, float eps, void* stream);
/* grafx_adam_step with the step number read from device memory (*step, int32, >= 1;
 * values below 1 count as 1), so that a captured fit step can advance its own counter.
 * The bias corrections are computed in double precision like grafx_adam_step's. */
int grafx_adam_step_dev(float* theta, float* m, float* v, const float* grad_param, float* param,
                        const int8_t* codes, int32_t cols, int64_t n, const int32_t* step, float lr, float beta1,
                        float beta2, float eps, void* stream);
/* theta = inverse map of param (to start a fit from physical parameters). */
int grafx_params_to_theta(const float* param, const int8_t* codes, int32_t cols, int64_t n, float* theta,
                          void* stream);

/* ---------------------------------------------------------------- failure detection
 * The paper has no counterpart; this exists so that the bounded device waits can be
 * tested without hanging a GPU.  One warp polls the device word *flag at most `limit`
 * times (1 <= limit <= 4194304, each poll followed by a short sleep), exactly like a
 * look-back of the compressor scan: if the word's upper half is nonzero, *value = the
 * float in its lower half; otherwise the wait expires, ST_TIMEOUT (1) is OR-ed into the
 * device word *status and *value = 0.  Asynchronous on `stream`. */
int grafx_selftest_bounded_wait(const unsigned long long* flag, uint32_t* status, int32_t limit, float* value,
                                void* stream);

/* ---------------------------------------------------------------- learned warm-start
 * The paper motivates estimating processor parameters with a trained network
 * (Sec. 1) and leaves the estimator open; this is the library's own: it predicts the
 * unconstrained parameters theta of every processor node (the variables of
 * grafx_adam_step) from audio, as a starting point for the gradient fit.
 *
 * Node inputs: after grafx_render(p, sources, out) (typically with neutral
 * parameters), writes u_v (Eq. 1b: the sum of the node's in-edge sources) of the n
 * nodes `ids` (host int32, ids in the plan's union numbering: graph g's node j is
 * j + the node counts of graphs 0..g-1) into device rows dst[i][2][dst_pitch]
 * (dst_pitch a multiple of 4 and >= the node's length; samples past the length are
 * 0).  Input nodes are rejected (GRAFX_EINVAL), and so are plans with checkpointing
 * (GRAFX_ESTATE: their scratch rows do not outlive a segment).  Asynchronous on `stream`. */
int grafx_node_inputs(grafx_plan* p, const float* sources, const float* out, const int32_t* ids, int32_t n,
                      float* dst, int64_t dst_pitch, void* stream);

/* Network (weights: one flat device float32 buffer, layout below, owned by the caller):
 *   features  [B][256][32]: log-mel (frames 2048, hop 512, no padding, periodic Hann,
 *             power, 128 HTK-mel triangles over 0..fs/2, ln(mel + 1e-5), frames
 *             average-pooled to 32) of the node input (channels 0..127) and of the
 *             target mix (128..255);
 *   encoder   4 x conv1d (kernel 5, zero padding 2) 256->128->128->128->128, bias,
 *             exact GELU; mean over the 32 frames;
 *   heads     per type (gain, imager, EQ, compressor, delay, reverb) an MLP
 *             128->288->288->N_t (N_t = 2, 1, 8, 4, 176, 50), GELU, GELU, linear.
 *   weights   conv{l}.w [Cout][Cin][5], conv{l}.b for l = 0..3, then per head in that
 *             type order w1 [288][128], b1, w2 [288][288], b2, w3 [N_t][288], b3.
 * Every matrix product runs on the tensor cores (tcgen05, accumulator in tensor memory)
 * with BF16 operands (rounded to nearest even from float32) and float32 accumulation.
 *
 * A net handle holds host tables only; its device workspace (caller-owned, 256-byte
 * aligned, grafx_ws_workspace_bytes for up to max_rows log-mel rows of up to
 * max_len samples) is attached by grafx_ws_bind, which uploads the constant tables
 * (synchronous on `stream`).  Calls on one net are stream-ordered and share the
 * workspace: grafx_ws_backward must follow the grafx_ws_forward of the same batch with
 * no other forward in between. */
typedef struct grafx_wsnet grafx_wsnet;
int grafx_ws_create(int32_t max_batch, int32_t sample_rate, grafx_wsnet** out);
int grafx_ws_destroy(grafx_wsnet* n);
int grafx_ws_param_count(const grafx_wsnet* n, int64_t* count);
int grafx_ws_workspace_bytes(const grafx_wsnet* n, int32_t max_rows, int64_t max_len, size_t* bytes);
int grafx_ws_bind(grafx_wsnet* n, void* ws, size_t bytes, void* stream);
/* Log-mel features of n_rows stereo rows (device, row r at rows + r*row_stride,
 * channel stride pitch, len >= 2048 samples each) into feats[i][coff..coff+127][32]
 * for the n_samples samples (sample i takes row row_of_sample[i], a device int32 array;
 * NULL means sample i = row i; an index outside [0, n_rows) gives zero features).
 * coff is 0 (node input) or 128 (target mix).  Asynchronous on `stream`. */
int grafx_ws_logmel(grafx_wsnet* n, const float* rows, int32_t n_rows, int64_t row_stride, int64_t pitch, int64_t len,
                    const int32_t* row_of_sample, int32_t n_samples, int32_t coff, float* feats, void* stream);
/* Cross-spectral band gain of n_samples node inputs against target mixes (a reading:
 * the paper motivates a trained estimator, Sec. 1, without fixing its inputs).  Sample i
 * takes the node input u_rows + i*u_stride and the target row
 * t_rows + row_of_sample[i]*t_stride (device int32 array; an index outside [0, n_trows)
 * gives a zero target); both stereo, channel stride pitch, len >= 2048.  For the mid
 * (l + r)/2 and the side (l - r)/2 of both, per log-mel frame and pair of mel triangles
 * (64 bands), C = sum w Re(T conj(U)) and P = sum w |U|^2; per pooling slot the sums over
 * its frames give feats[i][coff + h*64 + b][t] = ln(max(C / P, 0) + 0.01) (h = 0 mid,
 * 1 side).  The sources of a mix are independent, so C / P estimates the gain of the
 * node's own path to the output in that band.  The workspace must hold
 * n_samples * 2 log-mel rows (grafx_ws_workspace_bytes).  Asynchronous on `stream`. */
int grafx_ws_xgain(grafx_wsnet* n, const float* u_rows, int32_t n_samples, int64_t u_stride, const float* t_rows,
                   int32_t n_trows, int64_t t_stride, const int32_t* row_of_sample, int64_t pitch, int64_t len,
                   int32_t coff, float* feats, void* stream);
/* Forward of a batch of B <= max_batch samples sorted by head: head_count (host
 * int32[6]) gives how many consecutive samples use each head, in the type order above
 * (their sum must be B: GRAFX_ESHAPE otherwise).  out: device [B][176]; row i holds the
 * N_t outputs of its head and zeros after them.  Asynchronous on `stream`. */
int grafx_ws_forward(grafx_wsnet* n, const float* weights, const float* feats, const int32_t* head_count, int32_t B,
                     float* out, void* stream);
/* Gradient of <d_out, out> with respect to the weights after grafx_ws_forward on the
 * same inputs; d_weights (device, param_count floats) is overwritten.  Column sums are
 * taken in a fixed order (deterministic).  Asynchronous on `stream`. */
int grafx_ws_backward(grafx_wsnet* n, const float* weights, const float* feats, const int32_t* head_count, int32_t B,
                      const float* d_out, float* d_weights, void* stream);
/* Masked mean-squared error between out and target (device [B][176]): the squared
 * error is averaged over the first n_out[i] (device int32, >= 1) columns of each row and
 * then over the rows; *loss (device float) and d_out = dloss/dout (0 in unused
 * columns).  Asynchronous on `stream`. */
int grafx_ws_mse(const float* out, const float* target, const int32_t* n_out, int32_t B, float* loss, float* d_out,
                 void* stream);
/* The network's outputs are the fit's theta standardised per head and column: row i of
 * x (device float32 [B][cols]) uses the statistics of head head[i] (device int32) in mu
 * and sd (device float32 [heads][cols]); back = 0 gives y = (x - mu) / sd (training
 * targets), back = 1 gives y = mu + sd x (predictions); columns at or past n_out[i]
 * (device int32) are written 0.  y may be x.  Asynchronous on `stream`. */
int grafx_ws_standardise(const float* x, const int32_t* head, const int32_t* n_out, const float* mu, const float* sd,
                         int32_t B, int32_t cols, int32_t back, float* y, void* stream);
/* Synchronise `stream` and report (and clear) a bounded tensor-core wait of the net's
 * products that expired since the last call: GRAFX_ETIMEOUT, else GRAFX_OK. */
int grafx_ws_sync_status(grafx_wsnet* n, void* stream);
/* The network's matrix product on its own: C = alpha A B + beta C over device float32
 * buffers with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C row-major with
 * leading dimension ldc >= N; A and B are rounded to BF16 (nearest even) and the sums
 * accumulate in float32.  M <= 8388480.  scratch (device, scratch_floats floats, may be
 * NULL) lets a product with few output tiles split K over more CTAs: the partial tiles
 * (M*N floats each) are summed in a fixed order afterwards.  Asynchronous on `stream`. */
int grafx_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak, const float* B,
                    int64_t sbk, int64_t sbn, float* C, int64_t ldc, float alpha, float beta, float* scratch,
                    int64_t scratch_floats, void* stream);

/* ---------------------------------------------------------------- allocation-free compressor
 * The paper has no counterpart to this call; it exists for callers that must not
 * allocate device memory at all, such as real-time audio callbacks and plugin hosts
 * (a device allocation can block on a device-wide synchronisation) and host
 * frameworks that hand out every byte of device memory from their own pool.
 *
 * Applies the compressor of grafx_render (same parameters [alpha, T, W, R] and the
 * same chunked scan) to one stereo row: u and y are caller-owned device float32
 * [2][pitch] rows (16-byte aligned, pitch a multiple of 4, pitch >= len), params a
 * device pointer to 4 floats.  Every sample of y at and past len, up to pitch, is
 * written as 0.  status (device, 4-byte aligned, may be NULL) is a caller-owned word
 * into which the kernel ORs GRAFX status bits: bit 0 (1) means a bounded device wait
 * expired and some chunk used a zero carry, i.e. y is wrong; the call never clears it.
 * Read it after the stream has passed the call.  With status NULL an expiry is not
 * reported.  Asynchronous on `stream`.
 *
 * It calls no allocator: its only scratch (about 17 KB of look-back words, a ticket
 * and an internal status word) is a fixed array inside the library that every GPU
 * which loads the library holds until the process exits; the part a call uses is
 * zeroed on `stream` at every call.  Hence len is limited to 4194304 samples
 * (GRAFX_ESHAPE beyond).  The first call on a device looks up that array's device
 * address (once per device, with that device current; again only if the device's
 * context was destroyed and re-created, e.g. by cudaDeviceReset), so make that first
 * call before any stream capture.  Every call shares the one array: calls whose work
 * overlaps on the GPU (different streams, or devices that alias it) race and give
 * wrong results; serialise them. */
int grafx_compressor_forward_noalloc(const float* u, int64_t len, int64_t pitch, const float* params,
                                     float* y, uint32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GRAFX_H */
