// Filtered-noise reverb (Sec. 3 "Reverb", Eq. 6-7).
//
// Impulse response per node (forward): the STFT of the two noise buffers (mid, side;
// periodic Hann, centred frames; computed once per render) is multiplied by the
// masks M_x[k, m] = exp(H0_x[k] + m Hd_x[k]), inverted frame by frame, windowed and
// overlap-added, divided by sum w^2, and turned into left/right as (mid +- side)/2.
// Two layouts: compact (FFT 1024, hop 256, H0/Hd interpolated from 12 log-spaced
// bands, y = e^{q_dry} u + e^{q_wet} (h * u); the frames go through the 1024-point
// shared-memory FFT with mid + i side packed in one complex transform) and the
// paper's (FFT 384, hop 192, H0/Hd given per bin for bins 0..191 with the Nyquist
// bin dropped, y = h * u; 384 is not a power of two: its frames go through the 3 x 128
// mixed-radix transform of fft.cuh, five frames per CTA).
// Convolution: 22 partitions of 4096 taps by overlap-save with 8192-point spectra:
// Y_b = sum_p H_p X_{b-1-p} per channel (u windows of 2B samples from the delay's
// spectrum kernel), one inverse per block.
// Backward: the input adjoint correlates ybar with h through the same partitions
// (Ubar_b = sum_p conj(H_p) Ybar_{b+p} on 2B windows of ybar); the lags
// r_x[n] = sum_t ybar[t] u[t - n] come from R_p = sum_b X_{b-p-1} conj(Ybar_b) on
// B blocks of ybar; dL/dh = e^{q_wet} r is pushed back through the overlap-add, the
// per-frame inverse transform (its adjoint is a forward transform with the one-sided
// weights c_k/N), the masks and (compact) the band matrix; dq_dry = e^{q_dry} sum_x r_x[0]
// and dq_wet = e^{q_wet} sum_x sum_n h_x[n] r_x[n].
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {


// Split a packed spectrum Z of a + i b (a, b real) at bin k into A[k], B[k].
__device__ __forceinline__ void rv_split(float2 z, float2 zm, float2* a, float2* b) {
  *a = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
  *b = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
}

// M_x[k, m] (Eq. 7) of both channels at bin k and frame m of reverb node ri.
__device__ __forceinline__ void rv_masks(const DevCtx& c, const float* q, int ri, int k, int m, float* M) {
  if (c.rv_paper) {   // per-bin log-magnitudes on bins 0..K-1; the Nyquist bin K is dropped
    const int K = c.rv_n / 2;
#pragma unroll
    for (int x = 0; x < 2; ++x) M[x] = k < K ? expf(q[x * 2 * K + k] + float(m) * q[x * 2 * K + K + k]) : 0.f;
    return;
  }
  const float* lm = c.rv_lm + size_t(ri) * 4 * RV_BINS;   // k_rv_bands
#pragma unroll
  for (int x = 0; x < 2; ++x) M[x] = expf(lm[(2 * x) * RV_BINS + k] + float(m) * lm[(2 * x + 1) * RV_BINS + k]);
}

// Compact layout: H0_x[k] and Hd_x[k] interpolated from the 12 bands once per node (they
// do not depend on the frame); grid (reverb nodes of the step).
__global__ void __launch_bounds__(256) k_rv_bands(DevCtx c, int node_begin) {
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  float* lm = c.rv_lm + size_t(ri) * 4 * RV_BINS;
  for (int k = threadIdx.x; k < RV_BINS; k += blockDim.x) {
    const float* row = c.rv_band + k * RV_BANDS;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      float h0 = 0.f, hd = 0.f;
      for (int b = 0; b < RV_BANDS; ++b) {
        h0 += row[b] * q[x * 24 + b];
        hd += row[b] * q[x * 24 + 12 + b];
      }
      lm[(2 * x) * RV_BINS + k] = h0;
      lm[(2 * x + 1) * RV_BINS + k] = hd;
    }
  }
}

// U_x[m][k], k <= 512, of both noise buffers (packed mid + i side per frame).
__global__ void __launch_bounds__(RV_N / 16) k_rv_noise_stft(DevCtx c) {
  __shared__ float2 buf[fft::Padded<RV_N>::size];
  const int m = blockIdx.x;
  for (int j = threadIdx.x; j < RV_N; j += blockDim.x) {
    const int t = m * RV_HOP + j - RV_N / 2;   // centred frame
    const float w = c.rv_win[j];
    buf[fft::pad(j)] = t >= 0 && t < RV_LEN ? make_float2(w * c.rv_noise[t], w * c.rv_noise[RV_LEN + t]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft::forward<RV_N>(buf, c.ptw, threadIdx.x, true);
  for (int k = threadIdx.x; k <= RV_N / 2; k += blockDim.x) {
    float2 a, b;
    rv_split(buf[fft::pad(k)], buf[fft::pad((RV_N - k) & (RV_N - 1))], &a, &b);
    c.rv_U[size_t(m) * RV_BINS + k] = a;
    c.rv_U[size_t(RV_F + m) * RV_BINS + k] = b;
  }
}

// Masked noise frame m of one node, inverted and windowed: (mid, side) per sample.
__global__ void __launch_bounds__(RV_N / 16) k_rv_ir_frames(DevCtx c, int node_begin) {
  __shared__ float2 buf[fft::Padded<RV_N>::size];
  const int m = blockIdx.x, v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  for (int k = threadIdx.x; k <= RV_N / 2; k += blockDim.x) {
    float M[2];
    rv_masks(c, q, ri, k, m, M);
    float2 hm = c.rv_U[size_t(m) * RV_BINS + k], hs = c.rv_U[size_t(RV_F + m) * RV_BINS + k];
    hm = make_float2(hm.x * M[0], hm.y * M[0]);
    hs = make_float2(hs.x * M[1], hs.y * M[1]);
    if (k == 0 || k == RV_N / 2) hm.y = hs.y = 0.f;   // real DC / Nyquist (one-sided inverse)
    // W = Hm + i Hs at k, conj(Hm) + i conj(Hs) at N - k; stored conjugated for the inverse
    const float2 wk = make_float2(hm.x - hs.y, hm.y + hs.x);
    buf[fft::pad(k)] = make_float2(wk.x, -wk.y);
    if (k > 0 && k < RV_N / 2) {
      const float2 wm = make_float2(hm.x + hs.y, -hm.y + hs.x);
      buf[fft::pad(RV_N - k)] = make_float2(wm.x, -wm.y);
    }
  }
  __syncthreads();
  fft::forward<RV_N>(buf, c.ptw, threadIdx.x, true);
  float2* fr = c.rv_fr + (size_t(ri) * RV_F + m) * RV_N;
  const float inv = 1.f / float(RV_N);
  for (int j = threadIdx.x; j < RV_N; j += blockDim.x) {
    const float2 z = buf[fft::pad(j)];
    const float w = c.rv_win[j] * inv;
    fr[j] = make_float2(w * z.x, -w * z.y);   // conj of the result: (mid, side)
  }
}

// Paper layout (N = 384): frames per CTA of the 384-point transforms, the shared tables.
constexpr int RV_FPC = 5;
constexpr int RV_FS = 3 * fft::R128;   // floats2 per frame buffer
struct Rv384Smem {
  float2 buf[RV_FPC * RV_FS];
  float2_ cs[RV_PN];     // (cos, sin)(2 pi j / 384)
  float2_ tw[7 * 16];    // W_128^{r k} at [(r-1) 16 + k]
};
__device__ __forceinline__ void rv384_tables(const DevCtx& c, Rv384Smem& sm) {
  for (int j = threadIdx.x; j < RV_PN; j += blockDim.x) sm.cs[j] = c.rv_cs[j];
  for (int i = threadIdx.x; i < 7 * 16; i += blockDim.x) {
    const float2_ e = c.rv_cs[(3 * (i / 16 + 1) * (i % 16)) % RV_PN];
    sm.tw[i] = float2_{e.x, -e.y};
  }
}

// Paper layout: U_x[m][k], k <= N/2, of both noise buffers: the windowed centred frames
// (mid + i side) through the 384-point transform, split per channel; five frames per CTA.
__global__ void __launch_bounds__(128) k_rv_noise_384(DevCtx c) {
  __shared__ Rv384Smem sm;
  const int N = RV_PN, bins = N / 2 + 1, m0 = blockIdx.x * RV_FPC, nf = min(RV_FPC, c.rv_f - m0);
  rv384_tables(c, sm);
  for (int i = threadIdx.x; i < RV_FPC * N; i += blockDim.x) {
    const int f = i / N, j = i % N;
    const int t = (m0 + f) * c.rv_hop + j - N / 2;
    const float w = c.rv_win[j];
    const bool in = f < nf && t >= 0 && t < RV_LEN;
    sm.buf[f * RV_FS + fft::in384(j)] = in ? make_float2(w * c.rv_noise[t], w * c.rv_noise[RV_LEN + t]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft::forward384<RV_FPC>(sm.buf, sm.cs, sm.tw);
  for (int i = threadIdx.x; i < nf * bins; i += blockDim.x) {
    const int f = i / bins, k = i % bins, m = m0 + f;
    const float2* fb = sm.buf + f * RV_FS;
    float2 am, as;
    rv_split(fb[fft::out384(k)], fb[fft::out384((N - k) % N)], &am, &as);
    c.rv_U[size_t(m) * bins + k] = am;
    c.rv_U[size_t(c.rv_f + m) * bins + k] = as;
  }
}

// Paper layout: masked noise frames of one node, inverted and windowed: (mid, side) per
// sample.  The masked spectra of both channels (Nyquist dropped: M = 0 there) are packed
// as one Hermitian-extended spectrum Hm + i Hs, conjugated, transformed forward and
// conjugated back (the inverse); five frames per CTA.
__global__ void __launch_bounds__(128) k_rv_ir_frames_384(DevCtx c, int node_begin) {
  __shared__ Rv384Smem sm;
  const int N = RV_PN, K = N / 2, bins = K + 1;
  const int m0 = blockIdx.x * RV_FPC, nf = min(RV_FPC, c.rv_f - m0), v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  rv384_tables(c, sm);
  for (int i = threadIdx.x; i < RV_FPC * bins; i += blockDim.x) {
    const int f = i / bins, k = i % bins, m = m0 + f;
    float2* fb = sm.buf + f * RV_FS;
    float2 hm = make_float2(0.f, 0.f), hs = hm;
    if (f < nf) {
      float M[2];
      rv_masks(c, q, ri, k, m, M);
      hm = c.rv_U[size_t(m) * bins + k];
      hs = c.rv_U[size_t(c.rv_f + m) * bins + k];
      hm = make_float2(hm.x * M[0], hm.y * M[0]);
      hs = make_float2(hs.x * M[1], hs.y * M[1]);
    }
    if (k == 0 || k == K) hm.y = hs.y = 0.f;   // real DC / Nyquist (one-sided inverse)
    // W = Hm + i Hs at k, conj(Hm) + i conj(Hs) at N - k; stored conjugated
    fb[fft::in384(k)] = make_float2(hm.x - hs.y, -(hm.y + hs.x));
    if (k > 0 && k < K) fb[fft::in384(N - k)] = make_float2(hm.x + hs.y, hm.y - hs.x);
  }
  __syncthreads();
  fft::forward384<RV_FPC>(sm.buf, sm.cs, sm.tw);
  const float inv = 1.f / float(N);
  for (int i = threadIdx.x; i < nf * N; i += blockDim.x) {
    const int f = i / N, j = i % N;
    const float2 z = sm.buf[f * RV_FS + fft::out384(j)];
    const float w = c.rv_win[j] * inv;
    c.rv_fr[(size_t(ri) * c.rv_f + m0 + f) * N + j] = make_float2(w * z.x, -w * z.y);   // conj: (mid, side)
  }
}

// Window envelope at sample n and the frames covering it (frame m starts at
// m hop - N/2 in signal coordinates; np = n + N/2 in padded coordinates).
__device__ __forceinline__ float rv_ola_norm(const DevCtx& c, int n, int* m0, int* m1) {
  const int N = c.rv_n, hop = c.rv_hop;
  const int np = n + N / 2;
  const int hi = min(c.rv_f - 1, np / hop);
  const int lo = np - N + 1 <= 0 ? 0 : (np - N + 1 + hop - 1) / hop;
  float D = 0.f;
  for (int m = lo; m <= hi; ++m) {
    const float w = c.rv_win[np - m * hop];
    D += w * w;
  }
  *m0 = lo;
  *m1 = hi;
  return D;
}

// h_l, h_r of one node (overlap-add / sum w^2, mid/side -> left/right), zero past RV_LEN.
__global__ void k_rv_ir_ola(DevCtx c, int node_begin) {
  const int v = node_begin + blockIdx.y;
  const int ri = c.ext[v].z;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= RV_HLEN) return;
  float hl = 0.f, hr = 0.f;
  if (n < RV_LEN) {
    int lo, hi;
    const float D = rv_ola_norm(c, n, &lo, &hi);
    if (D > 1e-8f) {
      float sm = 0.f, ss = 0.f;
      const int N = c.rv_n;
      const float2* fr = c.rv_fr + size_t(ri) * c.rv_f * N;
      for (int m = lo; m <= hi; ++m) {
        const float2 z = fr[size_t(m) * N + n + N / 2 - m * c.rv_hop];
        sm += z.x;
        ss += z.y;
      }
      sm /= D;
      ss /= D;
      hl = 0.5f * (sm + ss);
      hr = 0.5f * (sm - ss);
    }
  }
  c.rv_h[(size_t(ri) * 2) * RV_HLEN + n] = hl;
  c.rv_h[(size_t(ri) * 2 + 1) * RV_HLEN + n] = hr;
}

// Partition spectra H_p = FFT([h_l + i h_r over [pB, pB+B), zeros]).
__global__ void __launch_bounds__(DL_M / 16) k_rv_hspec(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  const int p = blockIdx.x, v = node_begin + blockIdx.y;
  const int ri = c.ext[v].z;
  const float* hl = c.rv_h + (size_t(ri) * 2) * RV_HLEN + p * DL_B;
  const float* hr = hl + RV_HLEN;
  for (int i = threadIdx.x; i < DL_M; i += blockDim.x)
    buf[fft::pad(i)] = i < DL_B ? make_float2(hl[i], hr[i]) : make_float2(0.f, 0.f);
  __syncthreads();
  fft::forward<DL_M>(buf, c.ptw, threadIdx.x, true);
  float2* out = c.rv_H + (size_t(ri) * RV_P + p) * DL_M;
  for (int k = threadIdx.x; k < DL_M; k += blockDim.x) out[k] = buf[fft::pad(k)];
}

// Load the channel-split spectra of `count` slots for DL_CHUNK bins into smem
// ([slot][bin][2 ch]).
__device__ __forceinline__ void rv_load_split(const float2* base, int count, int k0, float2* dst) {
  for (int i = threadIdx.x; i < count * DL_CHUNK; i += blockDim.x) {
    const int s = i / DL_CHUNK, kk = i % DL_CHUNK, k = k0 + kk, km = (DL_M - k) & (DL_M - 1);
    const float2* spec = base + size_t(s) * DL_M;
    float2 a, b;
    rv_split(spec[k], spec[km], &a, &b);
    dst[(size_t(s) * DL_CHUNK + kk) * 2] = a;
    dst[(size_t(s) * DL_CHUNK + kk) * 2 + 1] = b;
  }
}

__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b, bool conj_a) {
  const float ay = conj_a ? -a.y : a.y;
  return make_float2(acc.x + a.x * b.x - ay * b.y, acc.y + a.x * b.y + ay * b.x);
}

// Packed spectrum l + i r of two real signals from their bin-k spectra A_l, A_r, at k
// and (0 < k < M/2) at M - k, where each real signal's spectrum is the conjugate:
// Z[k] = A_l + i A_r, Z[M-k] = conj(A_l) + i conj(A_r).
__device__ __forceinline__ void rv_store_sym(float2* Z, int k, float2 al, float2 ar) {
  Z[k] = make_float2(al.x - ar.y, al.y + ar.x);
  if (k > 0 && k < DL_M / 2) Z[DL_M - k] = make_float2(al.x + ar.y, ar.x - al.y);
}

constexpr int RV_NBO = 4;   // output blocks per warp pass (forward, adjoint)
constexpr int RV_PCH = 6;   // partitions per warp (lags): 4 chunks x 6 >= RV_P, two block halves
static_assert(4 * RV_PCH >= RV_P, "lag chunks must cover the partitions");

// what = 0: forward Y_b = sum_p H_p X_{b-1-p}; 1: input adjoint
// Ubar_b = sum_p conj(H_p) Ybarwin_{b+p}; 2: lags R_p = sum_b X_{b-p-1} conj(Ybarblk_b).
// The products of two real signals' spectra are conjugate-symmetric, so only bins
// 0..M/2 are computed and bin M - k is written from bin k: grid (DL_M / 2 / DL_CHUNK + 1,
// reverb nodes), 256 threads: bin kk = tid % 32, lane group g.
template <int WHAT>
__global__ void __launch_bounds__(256) k_rv_acc(DevCtx c, int node_begin) {
  extern __shared__ float2 sm[];
  const int v = node_begin + blockIdx.y, k0 = blockIdx.x * DL_CHUNK;
  const int4_ e = c.ext[v];
  const int ri = e.z, nb = e.w, nw = nb + RV_P;
  const int kk = threadIdx.x % DL_CHUNK, g = threadIdx.x / DL_CHUNK, ng = blockDim.x / DL_CHUNK;
  // slots: [0, nw) u windows from -RV_P; [nw, nw + nb) ybar blocks; [nw + nb, 2 nw + nb) ybar windows from 0
  const float2* spec = c.dl_spec + size_t(e.x) * DL_M;
  float2* Hs = sm;                                        // [RV_P][chunk][2]
  float2* S = WHAT == 2 ? sm : sm + size_t(RV_P) * DL_CHUNK * 2;
  if (WHAT != 2) rv_load_split(c.rv_H + size_t(ri) * RV_P * DL_M, RV_P, k0, Hs);
  if (WHAT == 0) rv_load_split(spec, nw, k0, S);
  if (WHAT == 1) rv_load_split(spec + size_t(nw + nb) * DL_M, nw, k0, S);
  if (WHAT == 2) {
    rv_load_split(spec, nw, k0, S);
    rv_load_split(spec + size_t(nw) * DL_M, nb, k0, S + size_t(nw) * DL_CHUNK * 2);
  }
  __syncthreads();
  const int k = k0 + kk;
  if (WHAT == 0 || WHAT == 1) {
    // RV_NBO consecutive output blocks per warp pass: each staged slot is read once and
    // feeds every output it reaches (u = i - p forward, u = i + p adjoint; the partition
    // spectra stay in shared memory)
    for (int b0 = g * RV_NBO; b0 < nb; b0 += ng * RV_NBO) {
      float2 acc[RV_NBO][2];
#pragma unroll
      for (int i = 0; i < RV_NBO; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
      constexpr int U0 = WHAT == 0 ? -(RV_P - 1) : 0, U1 = WHAT == 0 ? RV_NBO : RV_NBO + RV_P - 1;
#pragma unroll 1
      for (int u = U0; u < U1; ++u) {
        // forward: slot b - 1 - p + RV_P with p = i - u; adjoint: slot b + p with p = u - i
        const int sl = WHAT == 0 ? b0 - 1 + RV_P + u : b0 + u;
        if (sl >= nw) continue;
        const float2 xl = S[(size_t(sl) * DL_CHUNK + kk) * 2], xr = S[(size_t(sl) * DL_CHUNK + kk) * 2 + 1];
#pragma unroll
        for (int i = 0; i < RV_NBO; ++i) {
          const int p = WHAT == 0 ? i - u : u - i;
          if (p >= 0 && p < RV_P) {
            const float2 hl = Hs[(size_t(p) * DL_CHUNK + kk) * 2], hr = Hs[(size_t(p) * DL_CHUNK + kk) * 2 + 1];
            acc[i][0] = cmac(acc[i][0], hl, xl, WHAT == 1);
            acc[i][1] = cmac(acc[i][1], hr, xr, WHAT == 1);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RV_NBO; ++i) {
        const int b = b0 + i;
        if (b < nb && k <= DL_M / 2)
          rv_store_sym(c.rv_Y + (size_t(ri) * c.rv_nbmax + b) * DL_M, k, acc[i][0], acc[i][1]);
      }
    }
  } else {
    // warp g: partitions [p0, p0 + RV_PCH) over half h of the blocks, the X slots of
    // those partitions in a register window that slides by one slot per block; the two
    // halves are added in shared memory (fixed order)
    const float2* X = S;
    const float2* Yb = S + size_t(nw) * DL_CHUNK * 2;
    const int pc = g % (ng / 2), h = g / (ng / 2), p0 = pc * RV_PCH;
    const int bs = h == 0 ? 0 : nb / 2, be = h == 0 ? nb / 2 : nb;
    auto ldx = [&](int sl, float2& l, float2& r) {
      l = r = make_float2(0.f, 0.f);
      if (sl >= 0 && sl < nw) {
        l = X[(size_t(sl) * DL_CHUNK + kk) * 2];
        r = X[(size_t(sl) * DL_CHUNK + kk) * 2 + 1];
      }
    };
    float2 acc[RV_PCH][2], wl[RV_PCH], wr[RV_PCH];
#pragma unroll
    for (int j = 0; j < RV_PCH; ++j) {
      acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
      wl[j] = wr[j] = make_float2(0.f, 0.f);
    }
    // window slot of partition p0 + j at block b: b - 1 + RV_P - p0 - j
#pragma unroll
    for (int j = 0; j + 1 < RV_PCH; ++j) ldx(bs - 1 + RV_P - p0 - (j + 1), wl[j], wr[j]);
    for (int b = bs; b < be; ++b) {
#pragma unroll
      for (int j = RV_PCH - 1; j > 0; --j) {
        wl[j] = wl[j - 1];
        wr[j] = wr[j - 1];
      }
      ldx(b - 1 + RV_P - p0, wl[0], wr[0]);
      const float2 yl = Yb[(size_t(b) * DL_CHUNK + kk) * 2], yr = Yb[(size_t(b) * DL_CHUNK + kk) * 2 + 1];
#pragma unroll
      for (int j = 0; j < RV_PCH; ++j) {
        acc[j][0] = cmac(acc[j][0], yl, wl[j], true);   // x conj(y) = conj(y) x
        acc[j][1] = cmac(acc[j][1], yr, wr[j], true);
      }
    }
    __syncthreads();   // the staged spectra are no longer read: reuse them for the halves
    float2* red = sm;  // [pc][j][kk][2]
    if (h == 1)
#pragma unroll
      for (int j = 0; j < RV_PCH; ++j) {
        red[((size_t(pc) * RV_PCH + j) * DL_CHUNK + kk) * 2] = acc[j][0];
        red[((size_t(pc) * RV_PCH + j) * DL_CHUNK + kk) * 2 + 1] = acc[j][1];
      }
    __syncthreads();
    if (h == 0)
#pragma unroll
      for (int j = 0; j < RV_PCH; ++j) {
        const int p = p0 + j;
        if (p < RV_P) {
          const float2 ol = red[((size_t(pc) * RV_PCH + j) * DL_CHUNK + kk) * 2];
          const float2 orr = red[((size_t(pc) * RV_PCH + j) * DL_CHUNK + kk) * 2 + 1];
          const float2 al = make_float2(acc[j][0].x + ol.x, acc[j][0].y + ol.y);
          const float2 ar = make_float2(acc[j][1].x + orr.x, acc[j][1].y + orr.y);
          if (k <= DL_M / 2) rv_store_sym(c.rv_R + (size_t(ri) * RV_P + p) * DL_M, k, al, ar);
        }
      }
  }
}

// Inverse of a packed block spectrum; what = 0: forward output block b (samples
// [B, 2B) of the circular result are the linear convolution), 1: input adjoint block
// b (samples [0, B) are the correlation), 2: lags of partition p (IDFT[B - nu]).
template <int WHAT>
__global__ void __launch_bounds__(DL_M / 16) k_rv_inv(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  const int b = blockIdx.x, v = node_begin + blockIdx.y;
  const int4_ e = c.ext[v];
  const int ri = e.z, nb = e.w;
  if (WHAT != 2 && b >= nb) return;
  const NodeDev nd = c.nodes[v];
  const float2* Z = WHAT == 2 ? c.rv_R + (size_t(ri) * RV_P + b) * DL_M : c.rv_Y + (size_t(ri) * c.rv_nbmax + b) * DL_M;
  for (int k = threadIdx.x; k < DL_M; k += blockDim.x) {
    const float2 z = Z[k];
    buf[fft::pad(k)] = make_float2(z.x, -z.y);
  }
  __syncthreads();
  fft::forward<DL_M>(buf, c.ptw, threadIdx.x, true);
  const float inv = 1.f / float(DL_M);
  if (WHAT == 2) {
    // the lags of partition b, and (compact layout) this partition's sum_x sum_n h_x r_x
    // for dq_wet, reduced in a fixed order
    const float* hl = c.rv_h + (size_t(ri) * 2) * RV_HLEN;
    float acc[1] = {0.f};
    for (int nu = threadIdx.x; nu < DL_B; nu += blockDim.x) {
      const float2 z = buf[fft::pad((DL_B - nu) & (DL_M - 1))];
      const int n = b * DL_B + nu;
      const float rl = z.x * inv, rr = -z.y * inv;
      c.rv_r[(size_t(ri) * 2) * RV_HLEN + n] = rl;
      c.rv_r[(size_t(ri) * 2 + 1) * RV_HLEN + n] = rr;
      if (n < RV_LEN) acc[0] += hl[n] * rl + hl[RV_HLEN + n] * rr;
    }
    if (!c.rv_paper) {
      __syncthreads();   // buf is reused as the reduction scratch
      block_sum<1>(acc, reinterpret_cast<float*>(buf));
      if (threadIdx.x == 0) c.rv_dot[size_t(ri) * RV_P + b] = acc[0];
    }
    return;
  }
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  const bool dry = !c.rv_paper;   // the paper's reverb is wet only
  const float a_dry = dry ? expf(q[48]) : 0.f, a_wet = dry ? expf(q[49]) : 1.f;
  float* row = WHAT == 0 ? yrow_w(c, nd) : arow_w(c, nd);
  const int e0 = WHAT == 0 ? c.csr_ptr[v] : c.tcsr_ptr[v];
  const int e1 = WHAT == 0 ? c.csr_ptr[v + 1] : c.tcsr_ptr[v + 1];
  for (int j = threadIdx.x; j < DL_B; j += blockDim.x) {
    const int t = b * DL_B + j;
    if (t >= nd.pitch) continue;
    const float2 z = buf[fft::pad(WHAT == 0 ? DL_B + j : j)];
    float dl = 0.f, dr = 0.f;
    if (dry && t < nd.len)
      for (int ed = e0; ed < e1; ++ed) {
        const float* r = WHAT == 0 ? in_row(c, ed) : out_adj_row(c, ed);
        dl += r[t];
        dr += r[nd.pitch + t];
      }
    const bool in = t < nd.len;
    row[t] = in ? a_dry * dl + a_wet * z.x * inv : 0.f;
    row[nd.pitch + t] = in ? a_dry * dr - a_wet * z.y * inv : 0.f;
  }
}

// Adjoint of the IR synthesis for frame m of one node: per channel and bin, the mask
// gradient times the mask, M dL/dM, and m M dL/dM.
__global__ void __launch_bounds__(RV_N / 16) k_rv_gfr(DevCtx c, int node_begin) {
  __shared__ float2 buf[fft::Padded<RV_N>::size];
  const int m = blockIdx.x, v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  const float a_wet = expf(q[49]);
  const float* rl = c.rv_r + (size_t(ri) * 2) * RV_HLEN;
  const float* rr = rl + RV_HLEN;
  for (int j = threadIdx.x; j < RV_N; j += blockDim.x) {
    const int n = m * RV_HOP + j - RV_N / 2;   // centred frame
    float gm = 0.f, gs = 0.f;
    if (n >= 0 && n < RV_LEN) {
      int lo, hi;
      const float D = rv_ola_norm(c, n, &lo, &hi);
      if (D > 1e-8f) {
        const float hbl = a_wet * rl[n], hbr = a_wet * rr[n];
        const float w = c.rv_win[j] / D;
        gm = w * 0.5f * (hbl + hbr);
        gs = w * 0.5f * (hbl - hbr);
      }
    }
    buf[fft::pad(j)] = make_float2(gm, gs);
  }
  __syncthreads();
  fft::forward<RV_N>(buf, c.ptw, threadIdx.x, true);
  float2* out = c.rv_mm + (size_t(ri) * RV_F + m) * 2 * RV_BINS;
  for (int k = threadIdx.x; k <= RV_N / 2; k += blockDim.x) {
    float2 A[2];
    rv_split(buf[fft::pad(k)], buf[fft::pad((RV_N - k) & (RV_N - 1))], &A[0], &A[1]);
    const float ck = (k == 0 || k == RV_N / 2 ? 1.f : 2.f) / float(RV_N);
    float M[2];
    rv_masks(c, q, ri, k, m, M);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const float2 U = c.rv_U[size_t(x * RV_F + m) * RV_BINS + k];
      const float mbar = ck * (A[x].x * U.x + A[x].y * U.y);
      const float mm = M[x] * mbar;
      out[x * RV_BINS + k] = make_float2(mm, float(m) * mm);
    }
  }
}

// Paper layout: the adjoint of the IR synthesis for the frames of one node (the adjoint
// of the one-sided inverse is a forward transform with weights c_k/N): the frame
// adjoints (mid + i side) through the 384-point transform, split per channel; per
// channel and bin, M dL/dM and m M dL/dM.  Five frames per CTA.
__global__ void __launch_bounds__(128) k_rv_gfr_384(DevCtx c, int node_begin) {
  __shared__ Rv384Smem sm;
  const int N = RV_PN, K = N / 2, bins = K + 1;
  const int m0 = blockIdx.x * RV_FPC, nf = min(RV_FPC, c.rv_f - m0), v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  const float* rl = c.rv_r + (size_t(ri) * 2) * RV_HLEN;
  const float* rr = rl + RV_HLEN;
  rv384_tables(c, sm);
  for (int i = threadIdx.x; i < RV_FPC * N; i += blockDim.x) {
    const int f = i / N, j = i % N;
    const int n = (m0 + f) * c.rv_hop + j - N / 2;   // centred frame
    float gm = 0.f, gs = 0.f;
    if (f < nf && n >= 0 && n < RV_LEN) {
      int lo, hi;
      const float D = rv_ola_norm(c, n, &lo, &hi);
      if (D > 1e-8f) {
        const float w = c.rv_win[j] / D;
        gm = w * 0.5f * (rl[n] + rr[n]);
        gs = w * 0.5f * (rl[n] - rr[n]);
      }
    }
    sm.buf[f * RV_FS + fft::in384(j)] = make_float2(gm, gs);
  }
  __syncthreads();
  fft::forward384<RV_FPC>(sm.buf, sm.cs, sm.tw);
  for (int i = threadIdx.x; i < nf * bins; i += blockDim.x) {
    const int f = i / bins, k = i % bins, m = m0 + f;
    const float2* fb = sm.buf + f * RV_FS;
    float2 A[2];
    rv_split(fb[fft::out384(k)], fb[fft::out384((N - k) % N)], &A[0], &A[1]);
    const float ck = (k == 0 || k == K ? 1.f : 2.f) / float(N);
    float M[2];
    rv_masks(c, q, ri, k, m, M);
    float2* out = c.rv_mm + (size_t(ri) * c.rv_f + m) * 2 * bins;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const float2 U = c.rv_U[size_t(x * c.rv_f + m) * bins + k];
      const float mm = M[x] * ck * (A[x].x * U.x + A[x].y * U.y);
      out[x * bins + k] = make_float2(mm, float(m) * mm);
    }
  }
}

// Mask-gradient terms summed over frames, (channel, bin) items in parallel: a CTA takes
// 32 items of one node and eight frame groups, added in a fixed order.  Paper layout:
// the sums are the per-bin H0 and Hd gradients (written out); compact: they replace
// frame 0's row of the terms, for k_rv_grad (every frame of these items has been read
// by then, and no other CTA touches them).
__global__ void __launch_bounds__(256) k_rv_msum(DevCtx c, int node_begin) {
  __shared__ float2 red[8][32];
  const int v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z, bins = c.rv_n / 2 + 1;
  const int lane = threadIdx.x & 31, fg = threadIdx.x >> 5, i = blockIdx.x * 32 + lane;
  float2* mm = c.rv_mm + size_t(ri) * c.rv_f * 2 * bins;
  float2 t = make_float2(0.f, 0.f);
  if (i < 2 * bins)
    for (int m = fg; m < c.rv_f; m += 8) {
      const float2 z = mm[size_t(m) * 2 * bins + i];
      t.x += z.x;
      t.y += z.y;
    }
  red[fg][lane] = t;
  __syncthreads();
  if (fg != 0 || i >= 2 * bins) return;
#pragma unroll
  for (int g = 1; g < 8; ++g) t = make_float2(t.x + red[g][lane].x, t.y + red[g][lane].y);
  if (c.rv_paper) {   // uniform over the launch
    const int K = bins - 1, x = i / bins, k = i % bins;
    float* out = c.dparams + size_t(nd.grow) * c.pcols;
    if (k < K) {   // the Nyquist bin carries no parameter
      out[x * 2 * K + k] = t.x;
      out[x * 2 * K + K + k] = t.y;
    }
  } else {
    mm[i] = t;
  }
}

// Compact layout: the frame sums (frame 0's row after k_rv_msum) through the band
// matrix, then dq_dry and dq_wet.
__global__ void __launch_bounds__(256) k_rv_grad(DevCtx c, int node_begin) {
  __shared__ float g0[2][RV_BINS], gd[2][RV_BINS];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int ri = c.ext[v].z, bins = c.rv_n / 2 + 1;
  const float* q = c.params + size_t(nd.prow) * c.pcols;
  float* out = c.dparams + size_t(nd.grow) * c.pcols;
  const float2* mm = c.rv_mm + size_t(ri) * c.rv_f * 2 * bins;
  for (int i = threadIdx.x; i < 2 * bins; i += blockDim.x) {
    const float2 z = mm[i];
    g0[i / bins][i % bins] = z.x;
    gd[i / bins][i % bins] = z.y;
  }
  __syncthreads();
  if (threadIdx.x < 48) {
    const int x = threadIdx.x / 24, r = threadIdx.x % 24, b = r % 12;
    const float* src = r < 12 ? g0[x] : gd[x];
    float s = 0.f;
    for (int k = 0; k < RV_BINS; ++k) s += c.rv_band[k * RV_BANDS + b] * src[k];
    out[threadIdx.x] = s;
  }
  const float* rl = c.rv_r + (size_t(ri) * 2) * RV_HLEN;
  if (threadIdx.x == 0) {   // sum_x sum_n h_x[n] r_x[n] from the lag kernel's partition partials
    float dot = 0.f;
    for (int b = 0; b < RV_P; ++b) dot += c.rv_dot[size_t(ri) * RV_P + b];
    out[48] = expf(q[48]) * (rl[0] + rl[RV_HLEN]);
    out[49] = expf(q[49]) * dot;
  }
}

int launch_reverb(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  static bool init = false;
  const size_t sm_fft = sizeof(float2) * fft::Padded<DL_M>::size;
  const int nbm = c.rv_nbmax;
  const size_t sm0 = sizeof(float2) * 2 * DL_CHUNK * size_t(RV_P + nbm + RV_P);
  const size_t sm2 = sizeof(float2) * 2 * DL_CHUNK * size_t(nbm + RV_P + nbm);
  if (!init) {
    cudaFuncSetAttribute(k_rv_hspec, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    cudaFuncSetAttribute(k_rv_inv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    cudaFuncSetAttribute(k_rv_inv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    cudaFuncSetAttribute(k_rv_inv<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    const int maxsm = int(sizeof(float2) * 2 * DL_CHUNK * size_t(2 * DL_MAX_BLOCKS + RV_P + RV_P));
    cudaFuncSetAttribute(k_rv_acc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
    cudaFuncSetAttribute(k_rv_acc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
    cudaFuncSetAttribute(k_rv_acc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
    init = true;
  }
  if (what < 0 || b <= a) return 0;
  const int n = b - a;   // reverb nodes of the step: [a, b)
  const dim3 chunks(DL_M / 2 / DL_CHUNK + 1, n);   // bins 0..M/2 (conjugate symmetry)
  switch (what) {
    case 0:  // impulse responses and their partition spectra
      if (c.rv_paper) {
        const int fg = (c.rv_f + RV_FPC - 1) / RV_FPC;
        k_rv_noise_384<<<fg, 128, 0, s>>>(c);
        k_rv_ir_frames_384<<<dim3(fg, n), 128, 0, s>>>(c, a);
      } else {
        k_rv_noise_stft<<<RV_F, RV_N / 16, 0, s>>>(c);
        k_rv_bands<<<n, 256, 0, s>>>(c, a);
        k_rv_ir_frames<<<dim3(RV_F, n), RV_N / 16, 0, s>>>(c, a);
      }
      k_rv_ir_ola<<<dim3((RV_HLEN + 255) / 256, n), 256, 0, s>>>(c, a);
      k_rv_hspec<<<dim3(RV_P, n), DL_M / 16, sm_fft, s>>>(c, a);
      return c.rv_paper ? 4 : 5;
    case 1:  // forward convolution (after the u window spectra)
      k_rv_acc<0><<<chunks, 256, sm0, s>>>(c, a);
      k_rv_inv<0><<<dim3(nbm, n), DL_M / 16, sm_fft, s>>>(c, a);
      return 2;
    case 2:  // input adjoint (after the ybar spectra)
      k_rv_acc<1><<<chunks, 256, sm0, s>>>(c, a);
      k_rv_inv<1><<<dim3(nbm, n), DL_M / 16, sm_fft, s>>>(c, a);
      return 2;
    case 3:  // parameter gradients
      k_rv_acc<2><<<chunks, 256, sm2, s>>>(c, a);
      k_rv_inv<2><<<dim3(RV_P, n), DL_M / 16, sm_fft, s>>>(c, a);
      if (c.rv_paper)
        k_rv_gfr_384<<<dim3((c.rv_f + RV_FPC - 1) / RV_FPC, n), 128, 0, s>>>(c, a);
      else
        k_rv_gfr<<<dim3(RV_F, n), RV_N / 16, 0, s>>>(c, a);
      k_rv_msum<<<dim3((2 * (c.rv_n / 2 + 1) + 31) / 32, n), 256, 0, s>>>(c, a);
      if (c.rv_paper) return 4;
      k_rv_grad<<<n, 256, 0, s>>>(c, a);
      return 5;
  }
  return 0;
}

}  // namespace grafx
