// Zero-phase FIR equalizer (Eq. 4-5): design, overlap-save block-FFT convolution,
// and the adjoint.
//
// Design (one CTA per node): 8 band gains (dB) -> K = (N+1)/2 log-magnitudes by the
// fixed band matrix -> A_k = exp(.) -> h0[n] = (A_0 + 2 sum_k A_k cos(2 pi k n/N))/N
// for n in [0, H] (even, so only half is computed) -> h = Hann * h0 -> the M-point
// spectrum of h placed circularly (real and even), scaled by 1/M for the inverse.
//
// Convolution (one CTA per block): block j covers the window [ws, ws+M) with
// ws = -Hal + j*S (Hal = H rounded up to 4 so loads are float4-aligned) and writes
// the S valid outputs [ws+H, ws+H+S).  Left and right are packed as l + i r in one
// complex FFT; the filter spectrum is real, so one forward and one inverse transform
// serve both channels.  The gather of predecessors is fused into the window load.
//
// The forward keeps every block's input spectrum U[k] (the first transform's result).
//
// Backward (one CTA per run of consecutive blocks): ybar restricted to the block's output
// range [H, H+S) is transformed once.  The tap gradient dL/dh[m] = sum_t ybar[t] u[t-m]
// is accumulated in the frequency domain (every t lies in one block's range and t - m in
// that block's window): with the packed spectra Zy = Yl + i Yr and Zu = Ul + i Ur of
// real signals, P[k] = sum_blocks Zy[k] conj(Zu[k]) is accumulated over all M bins and
// Yl conj(Ul) + Yr conj(Ur) = (P[k] + conj(P[M-k])) / 2 written once per run for
// k <= M/2; a finalize kernel sums the runs of a node, inverts, and chains through Hann,
// the cosine sum, exp and the band matrix.  The input adjoint (the correlation of ybar with h, h even) is assembled by
// overlap-add: the inverse of Ybarc[k] Hspec[k] is the block's contribution on window
// positions [0, S + 2H); its own range [H, H+S) goes to the adjoint row, its head
// [0, H) belongs to the previous block's [S, S+H) and its tail [S+H, S+2H) to the next
// block's [H, 2H) (S >= 2H: only the two neighbours, into disjoint parts).  Inside a run
// the CTA adds the previous block's tail (kept in shared memory) before storing and its
// head into the stored previous block; across runs the head and tail go to a scratch and
// k_eq_ola adds them.  Two transforms per block instead of three (ybar window, centred
// u, inverse).
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {

constexpr float LN10_20 = 0.11512925464970229f;  // ln(10)/20

// A_k for k < K into smem A: exp(p_e[k]) when the row holds the log-magnitudes
// themselves (the paper's parameter), else exp(ln10/20 * sum_b B[k][b] band_dB[b]).
__device__ void eq_magnitudes(const DevCtx& c, const NodeDev& nd, float* A, int K) {
  if (c.eq_logmag) {
    const float* lm = c.params + size_t(nd.prow) * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) A[k] = expf(lm[k]);
    return;
  }
  const float* bands = c.params + nd.prow * 8;
  float b[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) b[i] = bands[i];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float* row = c.eq_band + k * 8;
    float db = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) db += row[i] * b[i];
    A[k] = expf(LN10_20 * db);
  }
}

constexpr int EQ_CHUNK = 64;  // taps (or bins) per CTA of the cosine-sum kernels

// Row stride of the filter spectra (M/2+1 real bins): a multiple of 4 floats so that
// every row starts 16-byte aligned (staged with cp.async).
__host__ __device__ constexpr int eq_spec_stride(int M) { return M / 2 + 4; }

constexpr int EQ_SPLIT = 4;    // lanes sharing one cosine sum (adjacent lanes of a warp)

// The filter design of one EQ node in one CTA (M/16 threads): A_k, then the even taps
// h[n] = Hann[n] (A_0 + 2 sum_{k>=1} A_k cos(2 pi k n / N)) / N for n in [0, H] (Eq. 4;
// the cosine indexed exactly by (k n) mod N), placed circularly (real, even) and scaled
// by 1/M, then the block spectrum by the FFT.  Parameter only: it runs on the side stream
// from the start of the render.
template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_design(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  __shared__ float A[1024];
  __shared__ float cs[2048];
  __shared__ float hs[1024];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int N = c.eq_taps, H = c.eq_H, K = (N + 1) / 2;
  eq_magnitudes(c, nd, A, K);
  for (int i = threadIdx.x; i < N; i += blockDim.x) cs[i] = c.eq_cos[i];
  __syncthreads();
  for (int n = threadIdx.x; n <= H; n += blockDim.x) {
    float s0 = 0.f, s1 = 0.f;   // two interleaved partial sums (odd and even k)
    int idx = n % N;            // (k n) mod N for k = 1
    const int step = (2 * n) % N;
    int idx2 = (2 * n) % N;     // k = 2
    int k = 1;
    for (; k + 1 < K; k += 2) {
      s0 += A[k] * cs[idx];
      s1 += A[k + 1] * cs[idx2];
      idx += step;
      if (idx >= N) idx -= N;
      idx2 += step;
      if (idx2 >= N) idx2 -= N;
    }
    if (k < K) s0 += A[k] * cs[idx];
    hs[n] = c.eq_hann[n] * (A[0] + 2.f * (s0 + s1)) / float(N);
  }
  __syncthreads();
  const float inv_m = 1.f / float(M);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const int a = m <= M / 2 ? m : M - m;    // circular position -> |tap index|
    buf[fft::pad(m)] = make_float2(a <= H ? hs[a] * inv_m : 0.f, 0.f);
  }
  __syncthreads();
  fft::forward<M>(buf, c.ptw, threadIdx.x, true);
  float* spec = c.eq_spec + size_t(c.ext[v].z) * eq_spec_stride(M);
  for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) spec[k] = buf[fft::pad(k)].x;
}

// Thread tid's share of the packed window [ws, ws+M): v[m] = (l, r) at p = tid + T m,
// gathered over the in-edges (u) or over the consumers' adjoints (ybar); zero outside
// [0, len) and, with `centre`, outside the block's output range [H, H+S).
template <int M, bool ADJ>
__device__ __forceinline__ void eq_load_regs(const DevCtx& c, int v, const NodeDev& nd, int ws, float2 (&x)[16],
                                             bool centre, int H, int S) {
  constexpr int T = M / 16;
#pragma unroll
  for (int m = 0; m < 16; ++m) x[m] = make_float2(0.f, 0.f);
  const int e0 = ADJ ? c.tcsr_ptr[v] : c.csr_ptr[v];
  const int e1 = ADJ ? c.tcsr_ptr[v + 1] : c.csr_ptr[v + 1];
  for (int e = e0; e < e1; ++e) {
    const float* row = ADJ ? out_adj_row(c, e) : in_row(c, e);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int p = threadIdx.x + T * m;
      const int t = ws + p;
      const bool in = t >= 0 && t < nd.len && (!centre || (p >= H && p < H + S));
      if (in) {
        x[m].x += row[t];
        x[m].y += row[nd.pitch + t];
      }
    }
  }
}

// conj(X[k] * Hspec[k]) for the thread's bins k = tid + T m (the conjugation makes the
// next forward transform an inverse; Hspec is real, even and scaled by 1/M).
template <int M>
__device__ __forceinline__ void eq_apply_regs(float2 (&x)[16], const float* spec) {
  constexpr int T = M / 16;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = threadIdx.x + T * m;
    const float hk = __ldg(spec + (k <= M / 2 ? k : M - k));
    x[m] = make_float2(x[m].x * hk, -x[m].y * hk);
  }
}

// Write the block's valid outputs p in [H, H+S) from the (conjugated) inverse result.
template <int M>
__device__ __forceinline__ void eq_store_regs(float* row, const NodeDev& nd, int ws, const float2 (&x)[16], int H,
                                              int S) {
  constexpr int T = M / 16;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int p = threadIdx.x + T * m;
    const int t = ws + p;
    if (p >= H && p < H + S && t >= 0 && t < nd.pitch) {
      const bool in = t < nd.len;
      row[t] = in ? x[m].x : 0.f;
      row[nd.pitch + t] = in ? -x[m].y : 0.f;
    }
  }
}

// PRO: the EQ node's single input is a gain node fused into this step (the planner's
// fuse_next = 2): the window is gathered over the gain's inputs and scaled by its gains
// (c.params2) on load, and the block's output range [H, H+S) of the gain's row is stored
// here (every sample once), so the row stays valid for every reader.
template <int M, bool PRO>
__global__ void __launch_bounds__(M / 16, 3 * 4096 / M) k_eq_fwd(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  float2* b0 = smem2;   // one FFT buffer (three CTAs per SM)
  // this size's FFT pass twiddles, staged once per CTA (the CTA loops over many blocks)
  float2_* stw = reinterpret_cast<float2_*>(smem2 + fft::Padded<M>::size);
  for (int i = threadIdx.x; i < fft::ptw_size(M); i += blockDim.x) stw[i] = c.ptw[fft::ptw_base(M) + i];
  const int H = c.eq_H, S = c.eq_step, Hal = c.eq_Hal;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const int ws = -Hal + w.y * S;
    const float* spec = c.eq_spec + size_t(w.z) * eq_spec_stride(M);
    float2 x[16];
    if constexpr (PRO) {
      const int gv = c.csr_src[c.csr_ptr[v]];   // the gain node
      const NodeDev ng = c.nodes[gv];
      eq_load_regs<M, false>(c, gv, ng, ws, x, false, H, S);
      const float gl = expf(c.params2[ng.prow * 2]), gr = expf(c.params2[ng.prow * 2 + 1]);
      float* yg = yrow_w(c, ng);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        x[m] = make_float2(__fmul_rn(gl, x[m].x), __fmul_rn(gr, x[m].y));   // as the gain kernel rounds
        const int p = threadIdx.x + (M / 16) * m, t = ws + p;
        if (p >= H && p < H + S && t >= 0 && t < ng.pitch) {
          yg[t] = t < ng.len ? x[m].x : 0.f;
          yg[ng.pitch + t] = t < ng.len ? x[m].y : 0.f;
        }
      }
    } else {
      eq_load_regs<M, false>(c, v, nd, ws, x, false, H, S);
    }
    __syncthreads();   // the previous transform's readers of b0 are done (and stw is staged)
    fft::forward_regs_1buf_tw<M>(x, b0, stw, threadIdx.x);
    float2* us = c.eq_uspec + size_t(w.w) * M;   // kept for the backward
#pragma unroll
    for (int m = 0; m < 16; ++m) us[threadIdx.x + (M / 16) * m] = x[m];
    eq_apply_regs<M>(x, spec);
    __syncthreads();
    fft::forward_regs_1buf_tw<M>(x, b0, stw, threadIdx.x);
    eq_store_regs<M>(yrow_w(c, nd), nd, ws, x, H, S);
  }
}

template <int M>
__global__ void __launch_bounds__(M / 16, 3 * 4096 / M) k_eq_bwd(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  constexpr int T = M / 16;
  float2* b0 = smem2;                              // one FFT buffer (three CTAs per SM)
  float2* X = smem2 + fft::Padded<M>::size;        // the block's input spectrum (unpadded)
  float* tl = reinterpret_cast<float*>(X + M);     // the previous block's tail [l, r][H]
  const int H = c.eq_H, S = c.eq_step, Hal = c.eq_Hal;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const int4_ e = c.ext[v];
    const float* spec = c.eq_spec + size_t(e.z) * eq_spec_stride(M);
    float2 acc[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) acc[m] = make_float2(0.f, 0.f);
    for (int j = w.y; j < w.y + w.z; ++j) {
      const int ws = -Hal + j * S;
      const size_t g = size_t(e.w) + j;
      __syncthreads();  // previous block's readers of b0/b1/X are done
      // the forward's spectrum of this block's window, in flight under the ybar load and
      // transform
      const float2* us = c.eq_uspec + g * M;
      for (int i = threadIdx.x; i < M / 2; i += T) cp_async16(X + 2 * i, us + 2 * i, 16);
      cp_async_commit();
      float2 x[16];
      eq_load_regs<M, true>(c, v, nd, ws, x, true, H, S);
      fft::forward_regs_1buf<M>(x, b0, c.ptw, threadIdx.x);
      cp_async_wait_all();
      __syncthreads();
      // P[k] += Zy[k] conj(Zu[k])
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float2 a = x[m], b = X[threadIdx.x + T * m];
        acc[m].x += a.x * b.x + a.y * b.y;
        acc[m].y += a.y * b.x - a.x * b.y;
      }
      // input adjoint: this block's share of the correlation with the even filter;
      // x[m] = (l, -r) at window position p = tid + T m
      eq_apply_regs<M>(x, spec);
      fft::forward_regs_1buf<M>(x, b0, c.ptw, threadIdx.x);   // every thread passed the barrier after the first
      const bool first = j == w.y, last = j == w.y + w.z - 1;
      if (!first)   // the previous block's tail falls on [H, 2H)
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int p = threadIdx.x + T * m;
          if (p >= H && p < 2 * H) {
            x[m].x += tl[p - H];
            x[m].y -= tl[H + p - H];
          }
        }
      __syncthreads();   // every thread has read tl before it is rewritten below
      float* row = arow_w(c, nd);
      eq_store_regs<M>(row, nd, ws, x, H, S);
      float* hd = c.eq_ola + g * 4 * H;   // run boundaries: [head, tail][l, r][H]
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int p = threadIdx.x + T * m;
        if (p < H) {   // head: the previous block's [S, S+H)
          const int t = ws + p;
          if (!first) {
            if (t >= 0 && t < nd.len) {   // stored by this CTA before the block's first barrier
              row[t] += x[m].x;
              row[nd.pitch + t] -= x[m].y;
            }
          } else if (j > 0) {
            hd[p] = x[m].x;
            hd[H + p] = -x[m].y;
          }
        } else if (p >= S + H && p < S + 2 * H) {   // tail: the next block's [H, 2H)
          const int q = p - (S + H);
          if (!last) {
            tl[q] = x[m].x;
            tl[H + q] = -x[m].y;
          } else {
            hd[2 * H + q] = x[m].x;
            hd[3 * H + q] = -x[m].y;
          }
        }
      }
    }
    // the run's both-channel sum (P[k] + conj(P[M-k])) / 2 for k <= M/2 (P[M-k] is held by
    // thread T - tid: exchanged through b0 once per run)
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; ++m) b0[fft::pad(threadIdx.x + T * m)] = acc[m];
    __syncthreads();
    float2* out = c.eq_partial + size_t(w.w) * (M / 2 + 1);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int k = threadIdx.x + T * m;
      if (k <= M / 2) {
        const float2 y = b0[fft::pad((M - k) & (M - 1))];
        out[k] = make_float2(0.5f * (acc[m].x + y.x), 0.5f * (acc[m].y - y.y));
      }
    }
  }
}

// Overlap-add of the input adjoint across runs (after k_eq_bwd): into a run's first
// block j0 goes block j0-1's tail (its window positions [S+H, S+2H) = j0's [H, 2H)), into
// its last block j1 block j1+1's head (its [0, H) = j1's [S, S+H)), for samples inside
// [0, len); one CTA per run.
__global__ void __launch_bounds__(256) k_eq_ola(DevCtx c, int item0, int n_items) {
  const int H = c.eq_H, S = c.eq_step, Hal = c.eq_Hal;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const int nb = (nd.len + Hal - H + S - 1) / S;
    const size_t base = size_t(c.ext[v].w);
    float* row = arow_w(c, nd);
    const int j0 = w.y, j1 = w.y + w.z - 1;
    for (int i = threadIdx.x; i < 2 * H; i += blockDim.x) {
      const bool left = i < H;
      const int q = left ? i : i - H;
      const int j = left ? j0 : j1, src = left ? j0 - 1 : j1 + 1;
      const int t = -Hal + j * S + (left ? H + q : S + q);
      if (src < 0 || src >= nb || t < 0 || t >= nd.len) continue;
      const float* part = c.eq_ola + (base + src) * 4 * H + (left ? 2 * H : 0);
      row[t] += part[q];
      row[nd.pitch + t] += part[H + q];
    }
  }
}

// Sum the runs of a node's tap-gradient spectrum, invert it, and fold the even
// symmetry through the window: s[n] = Hann[n] (hbar[n] + hbar[-n]) (s[0] = Hann[0] hbar[0]).
template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_gradfft(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  const int v = node_begin + blockIdx.x;
  const int4_ e = c.ext[v];
  const int H = c.eq_H;
  for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) {
    float2 r = make_float2(0.f, 0.f);
    for (int q = 0; q < e.y; ++q) {
      float2 x = c.eq_partial[size_t(e.x + q) * (M / 2 + 1) + k];
      r.x += x.x;
      r.y += x.y;
    }
    buf[fft::pad(k)] = make_float2(r.x, -r.y);    // conjugated: the forward FFT inverts
    if (k > 0 && k < M / 2) buf[fft::pad(M - k)] = r;
  }
  __syncthreads();
  fft::forward<M>(buf, c.ptw, threadIdx.x, true);
  const float inv_m = 1.f / float(M);
  float* s = c.eq_aux + size_t(e.z) * 1024;
  for (int n = threadIdx.x; n <= H; n += blockDim.x) {
    float hp = buf[fft::pad(n)].x * inv_m;
    float hm = buf[fft::pad((M - n) & (M - 1))].x * inv_m;
    s[n] = c.eq_hann[n] * (n == 0 ? hp : hp + hm);
  }
}

// dL/dp_k = A_k (c_k/N) sum_n s[n] cos(2 pi k n / N) for one chunk of k, then this
// chunk's share of the band-matrix product (with log-magnitude rows, dL/dp_k is the
// gradient itself and is stored directly); grid (EQ nodes of the step, chunks).
__global__ void __launch_bounds__(EQ_CHUNK * EQ_SPLIT) k_eq_gradbands(DevCtx c, int node_begin) {
  __shared__ float A[1024];
  __shared__ float sv[1024];
  __shared__ float cs[2048];
  __shared__ float red[8 * 32];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int N = c.eq_taps, H = c.eq_H, K = (N + 1) / 2;
  const int z = c.ext[v].z;
  eq_magnitudes(c, nd, A, K);
  for (int i = threadIdx.x; i < N; i += blockDim.x) cs[i] = c.eq_cos[i];
  for (int i = threadIdx.x; i <= H; i += blockDim.x) sv[i] = c.eq_aux[size_t(z) * 1024 + i];
  __syncthreads();
  const int k = blockIdx.y * EQ_CHUNK + threadIdx.x / EQ_SPLIT, part = threadIdx.x % EQ_SPLIT;
  float acc = 0.f;
  if (k < K) {
    const int step = (EQ_SPLIT * k) % N;
    int idx = ((1 + part) * k) % N;  // (k n) mod N
    for (int n = 1 + part; n <= H; n += EQ_SPLIT) {
      acc += sv[n] * cs[idx];
      idx += step;
      if (idx >= N) idx -= N;
    }
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (k < K && part == 0) {
    const float pk = A[k] * (sv[0] + acc) * (k == 0 ? 1.f : 2.f) / float(N);
    if (c.eq_logmag) {   // the row is p_e itself: dL/dp_e[k], no band matrix
      c.dparams[size_t(nd.grow) * K + k] = pk;
    } else {
      const float* row = c.eq_band + k * 8;
#pragma unroll
      for (int b = 0; b < 8; ++b) bsum[b] = row[b] * pk;
    }
  }
  if (c.eq_logmag) return;   // uniform over the launch: no thread reaches the block sums
  float lo[4] = {bsum[0], bsum[1], bsum[2], bsum[3]}, hi[4] = {bsum[4], bsum[5], bsum[6], bsum[7]};
  block_sum<4>(lo, red);
  block_sum<4>(hi, red + 4 * 32);
  if (threadIdx.x == 0) {
    float* d = c.eq_bandpart + (size_t(z) * gridDim.y + blockIdx.y) * 8;
    for (int b = 0; b < 4; ++b) {
      d[b] = lo[b];
      d[b + 4] = hi[b];
    }
  }
}

// Sum the chunks' band partials in order: dL/d(band dB).
__global__ void k_eq_gradout(DevCtx c, int node_begin, int node_end, int n_chunks) {
  const int v = node_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= node_end) return;
  const int z = c.ext[v].z;
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int q = 0; q < n_chunks; ++q)
    for (int b = 0; b < 8; ++b) s[b] += c.eq_bandpart[(size_t(z) * n_chunks + q) * 8 + b];
  float* d = c.dparams + c.nodes[v].grow * 8;
  for (int b = 0; b < 8; ++b) d[b] = LN10_20 * s[b];
}

template <int M>
static int eq_launch(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  constexpr int T = M / 16;
  static bool init = false;
  const size_t s1 = sizeof(float2) * fft::Padded<M>::size;
  const size_t sf = s1 + sizeof(float2_) * fft::ptw_size(M);   // one FFT buffer + pass twiddles
  // one FFT buffer, the kept spectrum, the previous block's tail (2H floats, H <= M/4)
  const size_t sb = s1 + sizeof(float2) * M + sizeof(float) * M / 2;
  if (!init) {
    cudaFuncSetAttribute(k_eq_design<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s1));
    cudaFuncSetAttribute(k_eq_gradfft<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s1));
    cudaFuncSetAttribute(k_eq_fwd<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sf));
    cudaFuncSetAttribute(k_eq_fwd<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sf));
    cudaFuncSetAttribute(k_eq_bwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sb));
    init = true;
  }
  if (what < 0) return 0;  // attributes only (before a stream capture)
  const int chunks_k = ((c.eq_taps + 1) / 2 + EQ_CHUNK - 1) / EQ_CHUNK;
  switch (what) {
    case 0:
      k_eq_design<M><<<b - a, T, s1, s>>>(c, a);
      return 1;
    case 1:
    case 4:   // 4: with the fused gain prologue
      if (what == 4) k_eq_fwd<M, true><<<grid_size(b, (228 * 1024) / int(sf + 1024)), T, sf, s>>>(c, a, b);
      else k_eq_fwd<M, false><<<grid_size(b, (228 * 1024) / int(sf + 1024)), T, sf, s>>>(c, a, b);
      return 1;
    case 2:
      k_eq_bwd<M><<<grid_size(b, (228 * 1024) / int(sb + 1024)), T, sb, s>>>(c, a, b);
      k_eq_ola<<<grid_size(b, 8), 256, 0, s>>>(c, a, b);
      return 2;
    case 3:
      k_eq_gradfft<M><<<b - a, T, s1, s>>>(c, a);
      k_eq_gradbands<<<dim3(b - a, chunks_k), EQ_CHUNK * EQ_SPLIT, 0, s>>>(c, a);
      if (c.eq_logmag) return 2;
      k_eq_gradout<<<(b - a + 63) / 64, 64, 0, s>>>(c, a, b, chunks_k);
      return 3;
  }
  return 0;
}

// what: 0 design(node range), 1 fwd(items), 2 bwd(items), 3 finalize(node range),
// 4 fwd(items) with the fused gain prologue
int launch_eq(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  if (what >= 0 && (b <= 0 || ((what == 0 || what == 3) && b <= a))) return 0;   // what 4: fwd + gain prologue
  switch (c.eq_fft) {
    case 1024: return eq_launch<1024>(what, c, a, b, s);
    case 2048: return eq_launch<2048>(what, c, a, b, s);
    case 4096: return eq_launch<4096>(what, c, a, b, s);
    default: return eq_launch<8192>(what, c, a, b, s);
  }
}

}  // namespace grafx
