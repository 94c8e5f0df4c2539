// Launch wrappers of the step kernels (one per .cu file).  Each returns the number of
// kernels it launched.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace grafx {

int grid_size(int n_items, int per_sm);
// CTAs of `kernel` that fit on one SM at once with `threads` threads and `smem` bytes of
// dynamic shared memory (its registers and static shared memory counted), at least 1.
// A strided item loop launched with grid_size(n, resident_per_sm(...)) runs as one wave:
// with more CTAs than fit, the surplus starts only after whole CTAs of the first wave
// have finished all their items, on a partly empty GPU.  Query it after setting the
// kernel's dynamic shared-memory attribute, outside any stream capture.
int resident_per_sm(const void* kernel, int threads, size_t smem);

// elementwise types (mix/out, gain, imager)
int launch_ew_fwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s);
int launch_ew_bwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s);
// the same without the input-adjoint stores (gain/imager: partials only; mix: nothing)
int launch_ew_bwd_nostore(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s);
int launch_ew_finalize(const DevCtx& c, int node_begin, int node_end, int cols, cudaStream_t s);
// fused pair of gain/imager steps (types tv then tw) over the second step's items
int launch_ew2(bool bwd, int tv, int tw, const DevCtx& c, int item0, int n_items, cudaStream_t s);
// source batch: dst[i] = sum over the B copies of part[b n + i]
int launch_fold_copies(const float* part, float* dst, int64_t n, int B, cudaStream_t s);

// EQ: what = 0 design (a = node_begin, b = node_end), 1 forward (a = item0,
// b = n_items), 2 backward (items), 3 gradient finalize (node range)
int launch_eq(int what, const DevCtx& c, int a, int b, cudaStream_t s);  // what < 0: set kernel attributes only

// compressor, noisegate and sidechain compressor (mode 0, 1, 2): what = 0 forward,
// 1 backward (a = item0, b = n_items, ticket index), 2 gradient finalize (a = node_begin,
// b = node_end)
int launch_comp(int what, const DevCtx& c, int a, int b, int n0, int n1, int ticket, int mode, cudaStream_t s);

// delay: what = 0 design (node range), 1 forward (items), 2 input adjoint, 3 block
// spectra, 4 partition accumulation, 5 lags (inverse FFTs), 6 gradients; < 0 attributes
int launch_delay(int what, const DevCtx& c, int a, int b, cudaStream_t s);

// compressor with attack/release ballistics: forward (items + node range), backward,
// parameter-gradient finalize (node range)
int launch_bal_fwd(const DevCtx& c, int item0, int n_items, int node_begin, int node_end, cudaStream_t s);
int launch_bal_bwd(const DevCtx& c, int item0, int n_items, int node_begin, int node_end, cudaStream_t s);
int launch_bal_finalize(const DevCtx& c, int node_begin, int node_end, cudaStream_t s);

// reverb over the reverb nodes [a, b) of a step: what = 0 impulse responses, 1 forward
// convolution, 2 input adjoint, 3 parameter gradients; < 0 attributes only
int launch_reverb(int what, const DevCtx& c, int a, int b, cudaStream_t s);

// Node inputs u_v of a batch of nodes (new ids), gathered after a render into rows
// dst[first + i][2][dst_pitch] (warm-start features).
constexpr int NI_MAX = 256;
struct NodeIds {
  int32_t first;
  int32_t v[NI_MAX];
};
int launch_node_inputs(const DevCtx& c, const NodeIds& ids, int n, float* dst, int64_t dst_pitch, cudaStream_t s);

struct LossLaunch {
  const LossRow* rows;
  const int4_* items;   // (row, resolution, first frame, group)
  int n_items;
  const float* y;
  const float* tgt;
  float4* part;
  float4* stats;
  float* frames;
  float2* spec;         // spectrum cache written by the forward, read by the backward
  const float2_* tw;
  const float2_* ptw;
  int n_rows;
  int max_pitch;
  float* loss;
  float* row_loss;
  float* d_out;
};
// what = 0 forward (statistics + reduce into *loss), 2 backward (frames + overlap-add into d_out)
int launch_loss(int what, const LossLaunch& L, cudaStream_t s);  // what < 0: set kernel attributes only

}  // namespace grafx
