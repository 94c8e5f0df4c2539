// Device context and helpers shared by the step kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/grafx.h"
#include "devtypes.h"

namespace grafx {

// Everything a step kernel needs, passed by value.  Row bases are indexed by
// NodeKind: [0] sources (or d_sources), [1] the caller's out (or d_out), [2] the
// workspace U (or adjoint A) region.
struct DevCtx {
  const NodeDev* nodes;
  const int4_* ext;
  const int32_t* csr_ptr;
  const int32_t* csr_src;
  const int32_t* tcsr_ptr;
  const int32_t* tcsr_dst;
  const int64_t* csr_row;     // per in-edge (CSR order): the source's output-port row (REF_SHIFT)
  const int64_t* tcsr_row;    // per consumer edge: the consumer's input-port adjoint row
  const int32_t* in1_begin;   // per node: first in-edge of input 1 (= csr_ptr[v+1] with one input)
  const int32_t* out1_begin;  // per node: first consumer edge of output 1
  const int4_* items;
  const float2_* tw;    // exp(-2 pi i m / 8192), m < 8192 (window tables)
  const float2_* ptw;   // FFT pass twiddle tables (fft.cuh)
  const float* eq_cos;
  const float* eq_hann;
  const float* eq_band;
  uint32_t* status;
  int32_t* tickets;
  unsigned long long* flags;
  float* eq_spec;
  float* eq_aux;       // per EQ node: 1024 floats (taps in the forward, gradient fold in the backward)
  float* eq_bandpart;  // per EQ node: chunk partials of the band gradient (16 x 8 floats)
  float2* eq_uspec;    // per EQ block: the forward's spectrum of its input window (M bins)
  float* eq_ola;       // per EQ block: input-adjoint head and tail [2][2 ch][H] (overlap-add)
  float* comp_carry;   // per compressor chunk: the envelope state entering it (forward)
  float* dl_aux;        // per delay node: [channel][tap][39 taps, delay] (2 dl_taps 40 floats)
  float2* dl_spec;      // block spectra of the lag correlation
  float2* dl_R;         // per delay node and lag partition: accumulated spectra
  float* dl_r;          // per delay node and channel: lags r[n], n from -DL_B (dl_P DL_B each)
  float dl_taylor[9];   // Taylor coefficients of sum_k k q^k near q = 1
  const float* rv_noise;  // reverb noise [2][RV_LEN] (mid, side)
  const float* rv_band;   // [RV_BINS][RV_BANDS] band interpolation (compact layout)
  const float* rv_win;    // [rv_n] periodic Hann window of the reverb STFT
  const float2_* rv_cs;   // [rv_n] (cos, sin)(2 pi j / rv_n): direct frame DFTs (paper layout)
  float2* rv_U;           // noise STFT [2][rv_f][rv_n/2+1]
  float2* rv_fr;          // per reverb node: IR frames [rv_f][rv_n] (mid, side)
  float* rv_h;            // per reverb node: h_l, h_r [2][RV_HLEN]
  float2* rv_H;           // per reverb node: partition spectra [RV_P][DL_M]
  float2* rv_Y;           // per reverb node: block spectra [rv_nbmax][DL_M]
  float2* rv_R;           // per reverb node: lag partition spectra [RV_P][DL_M]
  float* rv_r;            // per reverb node: lags [2][RV_HLEN]
  float2* rv_mm;          // per reverb node: mask-gradient terms [rv_f][2][rv_n/2+1]
  float* rv_lm;           // per reverb node (compact layout): [mid, side][H0, Hd][RV_BINS]
  float* rv_dot;          // per reverb node: sum_n h_x[n] r_x[n] over each lag partition
  int32_t rv_nbmax;
  float* bal;            // per ballistic node: mid, envelope, envelope-adjoint and coefficient rows
  int32_t bal_maxlen;    // the longest signal of the plan (grids of the ballistic chunk kernels)
  float4* partial;
  float2* eq_partial;
  float* ybase[3];
  float* abase[3];
  const float* params;  // P[t] of the launched step's type
  const float* params2; // fused elementwise pairs: P[t] of the first step's type
  float* dparams;       // dLoss/dP[t] (finalize kernels)
  int32_t pcols;
  int32_t eq_taps, eq_H, eq_Hal, eq_fft, eq_step;
  int32_t comp_chunk;
  float sample_rate;
  // processor layouts
  int32_t eq_logmag;                        // P[eq] rows hold the (eq_taps+1)/2 log-magnitudes
  int32_t dl_taps, dl_nd, dl_slot, dl_P;    // delay taps per channel, surrogate length, slot width, lag partitions
  int32_t dl_nbmax;                         // most B-sample blocks of any delay node's signal
  int32_t rv_paper, rv_n, rv_hop, rv_f;     // reverb: paper layout, STFT size, hop, frames
};

// cp.async of 16 bytes into shared memory; the bytes past src_bytes (all 16 when
// src_bytes = 0, nothing read) are written as zeros.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ const float* yrow(const DevCtx& c, const NodeDev& n) {
  return c.ybase[n.kind] + n.off_y;
}
__device__ __forceinline__ float* yrow_w(const DevCtx& c, const NodeDev& n) {
  return c.ybase[n.kind] + n.off_y;
}
__device__ __forceinline__ const float* arow(const DevCtx& c, const NodeDev& n) {
  return c.abase[n.kind] + n.off_a;
}
__device__ __forceinline__ float* arow_w(const DevCtx& c, const NodeDev& n) {
  return c.abase[n.kind] + n.off_a;
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Keep only the samples of quad [t, t+4) that are < len (row padding reads as 0).
__device__ __forceinline__ float4 mask4(float4 v, int t, int len) {
  if (t + 4 <= len) return v;
  if (t + 0 >= len) v.x = 0.f;
  if (t + 1 >= len) v.y = 0.f;
  if (t + 2 >= len) v.z = 0.f;
  if (t + 3 >= len) v.w = 0.f;
  return v;
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
// Plain (coherent) load for rows written earlier in the same launch sequence.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// The row an in-edge e reads (the source's output port k) and the adjoint row a consumer
// edge e reads (the consumer's input-port-l adjoint), from the planner's row references.
__device__ __forceinline__ const float* in_row(const DevCtx& c, int e) {
  const int64_t r = c.csr_row[e];
  return c.ybase[r >> REF_SHIFT] + (r & REF_MASK);
}
__device__ __forceinline__ const float* out_adj_row(const DevCtx& c, int e) {
  const int64_t r = c.tcsr_row[e];
  return c.abase[r >> REF_SHIFT] + (r & REF_MASK);
}

// u_v: sum over the in-edges of v (Eq. 1b; I^G gather + I^A aggregate of Algorithm 1)
// of the quad [t, t+4) of channel ch, in CSR order.  t must be a multiple of 4.
// (Single-input nodes: every in-edge enters input 0.)
__device__ __forceinline__ float4 gather_in(const DevCtx& c, int v, int ch, int t, int len, int pitch) {
  float4 acc = f4zero();
  const int e1 = c.csr_ptr[v + 1];
  for (int e = c.csr_ptr[v]; e < e1; ++e) acc = f4add(acc, ld4(in_row(c, e) + ch * pitch + t));
  return mask4(acc, t, len);
}

// ybar_v: sum over the consumers w of v of their input adjoints (transposed CSR).
// (Single-output nodes: every consumer edge leaves output 0.)
__device__ __forceinline__ float4 gather_out_adj(const DevCtx& c, int v, int ch, int t, int len, int pitch) {
  float4 acc = f4zero();
  const int e1 = c.tcsr_ptr[v + 1];
  for (int e = c.tcsr_ptr[v]; e < e1; ++e) acc = f4add(acc, ld4(out_adj_row(c, e) + ch * pitch + t));
  return mask4(acc, t, len);
}

__device__ __forceinline__ void set_status(const DevCtx& c, uint32_t bits) { atomicOr(c.status, bits); }

// Block-wide sum of up to 4 values (blockDim.x multiple of 32, <= 1024).  Result
// valid in thread 0.  Uses `sh` of at least 4*32 floats.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* sh) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i * 32 + warp] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float x = lane < nw ? sh[i * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[i] = x;
    }
  }
}

}  // namespace grafx
