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
// Backward (one CTA per run of consecutive blocks): the input adjoint is the same
// centred convolution applied to ybar (h is even); the tap gradient
// dL/dh[m] = sum_t ybar[t] u[t-m] is accumulated in the frequency domain as
// sum_blocks Ybar[k] conj(Ucentre[k]) (both channels combined from the packed
// spectra) and written once per run; a finalize kernel sums the runs of a node,
// inverts, and chains through Hann, the cosine sum, exp and the band matrix.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {

constexpr float LN10_20 = 0.11512925464970229f;  // ln(10)/20

// A_k = exp(ln10/20 * sum_b B[k][b] band_dB[b]) for k < K, into smem A.
__device__ void eq_magnitudes(const DevCtx& c, const NodeDev& nd, float* A, int K) {
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

template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_design(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;                                     // Padded<M>
  float* A = reinterpret_cast<float*>(buf + fft::Padded<M>::size);  // K floats
  float* h = A + 1024;                                     // H+1 floats
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int N = c.eq_taps, H = c.eq_H, K = (N + 1) / 2;
  eq_magnitudes(c, nd, A, K);
  __syncthreads();
  for (int n = threadIdx.x; n <= H; n += blockDim.x) {
    float s = 0.f;
    int idx = 0;                       // (k * n) mod N
    for (int k = 1; k < K; ++k) {
      idx += n;
      if (idx >= N) idx -= N;
      s += A[k] * c.eq_cos[idx];
    }
    h[n] = c.eq_hann[n] * (A[0] + 2.f * s) / float(N);
  }
  __syncthreads();
  const float inv_m = 1.f / float(M);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    int a = m <= M / 2 ? m : M - m;    // circular position -> |tap index|
    buf[fft::pad(m)] = make_float2(a <= H ? h[a] * inv_m : 0.f, 0.f);
  }
  __syncthreads();
  fft::forward<M>(buf, c.tw, threadIdx.x, true);
  float* spec = c.eq_spec + size_t(c.ext[v].z) * (M / 2 + 1);
  for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) spec[k] = buf[fft::pad(k)].x;
}

// Load the packed window [ws, ws+M) of u (gathered) or of ybar (gathered over the
// consumers), zero outside [0, len).  With `centre`, samples outside the block's
// output range [ws+H, ws+H+S) are zeroed too.
template <int M, bool ADJ>
__device__ __forceinline__ void eq_load(const DevCtx& c, int v, const NodeDev& nd, int ws, float2* buf,
                                        bool centre, int H, int S) {
  for (int q = threadIdx.x; q < M / 4; q += blockDim.x) {
    const int t = ws + 4 * q;
    float4 l = f4zero(), r = f4zero();
    if (t >= 0 && t < nd.len) {
      if (ADJ) {
        l = gather_out_adj(c, v, 0, t, nd.len, nd.pitch);
        r = gather_out_adj(c, v, 1, t, nd.len, nd.pitch);
      } else {
        l = gather_in(c, v, 0, t, nd.len, nd.pitch);
        r = gather_in(c, v, 1, t, nd.len, nd.pitch);
      }
    }
    float lv[4] = {l.x, l.y, l.z, l.w}, rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int p = 4 * q + i;
      bool keep = !centre || (p >= H && p < H + S);
      buf[fft::pad(p)] = keep ? make_float2(lv[i], rv[i]) : make_float2(0.f, 0.f);
    }
  }
}

// conj(Z[k] * Hspec[k]) in place (the conjugation turns the next forward FFT into
// an inverse; Hspec is real, even, and already scaled by 1/M).
template <int M>
__device__ __forceinline__ void eq_apply(float2* buf, const float* spec) {
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    float hk = spec[k <= M / 2 ? k : M - k];
    float2 z = buf[fft::pad(k)];
    buf[fft::pad(k)] = make_float2(z.x * hk, -z.y * hk);
  }
}

// Write the S valid outputs of the block (conj of the inverse result), zero padding.
template <int M>
__device__ __forceinline__ void eq_store(float* row, const NodeDev& nd, int ws, const float2* buf, int H, int S) {
  for (int p = H + threadIdx.x; p < H + S; p += blockDim.x) {
    const int t = ws + p;
    if (t < 0 || t >= nd.pitch) continue;
    float2 z = buf[fft::pad(p)];
    bool in = t < nd.len;
    row[t] = in ? z.x : 0.f;
    row[nd.pitch + t] = in ? -z.y : 0.f;
  }
}

template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_fwd(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  const int H = c.eq_H, S = c.eq_step, Hal = c.eq_Hal;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const int ws = -Hal + w.y * S;
    const float* spec = c.eq_spec + size_t(w.z) * (M / 2 + 1);
    eq_load<M, false>(c, v, nd, ws, buf, false, H, S);
    __syncthreads();
    fft::forward<M>(buf, c.tw, threadIdx.x, true);
    eq_apply<M>(buf, spec);
    __syncthreads();
    fft::forward<M>(buf, c.tw, threadIdx.x, true);
    eq_store<M>(yrow_w(c, nd), nd, ws, buf, H, S);
    __syncthreads();
  }
}

template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_bwd(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  float2* by = smem2;                            // ybar window -> its spectrum
  float2* bx = smem2 + fft::Padded<M>::size;     // centred u -> spectrum; then ubar
  constexpr int T = M / 16;
  constexpr int NK = (M / 2 + 1 + T - 1) / T;    // accumulator bins per thread
  const int H = c.eq_H, S = c.eq_step, Hal = c.eq_Hal;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const float* spec = c.eq_spec + size_t(c.ext[v].z) * (M / 2 + 1);
    float2 acc[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int j = w.y; j < w.y + w.z; ++j) {
      const int ws = -Hal + j * S;
      eq_load<M, true>(c, v, nd, ws, by, false, H, S);
      eq_load<M, false>(c, v, nd, ws, bx, true, H, S);
      __syncthreads();
      fft::forward<M>(by, c.tw, threadIdx.x, true);
      fft::forward<M>(bx, c.tw, threadIdx.x, true);
      // sum_x Ybar_x[k] conj(U_x[k]) from the packed spectra
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        int k = threadIdx.x + i * T;
        if (k <= M / 2) {
          int km = (M - k) & (M - 1);
          float2 a = by[fft::pad(k)], b = bx[fft::pad(k)];
          float2 a2 = by[fft::pad(km)], b2 = bx[fft::pad(km)];
          // a conj(b) + conj(a2) b2
          float re = a.x * b.x + a.y * b.y + a2.x * b2.x + a2.y * b2.y;
          float im = a.y * b.x - a.x * b.y + a2.x * b2.y - a2.y * b2.x;
          acc[i].x += 0.5f * re;
          acc[i].y += 0.5f * im;
        }
      }
      __syncthreads();
      // input adjoint: conj(Ybar * H) -> forward FFT -> conj
      for (int k = threadIdx.x; k < M; k += blockDim.x) {
        float hk = spec[k <= M / 2 ? k : M - k];
        float2 z = by[fft::pad(k)];
        bx[fft::pad(k)] = make_float2(z.x * hk, -z.y * hk);
      }
      __syncthreads();
      fft::forward<M>(bx, c.tw, threadIdx.x, true);
      eq_store<M>(arow_w(c, nd), nd, ws, bx, H, S);
      __syncthreads();
    }
    float2* out = c.eq_partial + size_t(w.w) * (M / 2 + 1);
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      int k = threadIdx.x + i * T;
      if (k <= M / 2) out[k] = acc[i];
    }
  }
}

template <int M>
__global__ void __launch_bounds__(M / 16) k_eq_finalize(DevCtx c, int node_begin) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  float* A = reinterpret_cast<float*>(buf + fft::Padded<M>::size);  // K
  float* s = A + 1024;                                               // H+1
  __shared__ float red[8 * 32];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int4_ e = c.ext[v];
  const int N = c.eq_taps, H = c.eq_H, K = (N + 1) / 2;
  // Hermitian spectrum of r'[m] = dL/dh[m]; conjugated for the inverse
  for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) {
    float2 r = make_float2(0.f, 0.f);
    for (int q = 0; q < e.y; ++q) {
      float2 x = c.eq_partial[size_t(e.x + q) * (M / 2 + 1) + k];
      r.x += x.x;
      r.y += x.y;
    }
    buf[fft::pad(k)] = make_float2(r.x, -r.y);
    if (k > 0 && k < M / 2) buf[fft::pad(M - k)] = r;
  }
  eq_magnitudes(c, nd, A, K);
  __syncthreads();
  fft::forward<M>(buf, c.tw, threadIdx.x, true);
  // hbar[m] = Re(result)/M at m mod M; fold the even symmetry: s[n] = v[n](hbar[n] + hbar[-n])
  const float inv_m = 1.f / float(M);
  for (int n = threadIdx.x; n <= H; n += blockDim.x) {
    float hp = buf[fft::pad(n)].x * inv_m;
    float hm = buf[fft::pad((M - n) & (M - 1))].x * inv_m;
    s[n] = c.eq_hann[n] * (n == 0 ? hp : hp + hm);
  }
  __syncthreads();
  // dL/dp_k = A_k * (c_k/N) sum_n s[n] cos(2 pi k n / N); then the band matrix
  float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float acc = s[0];
    int idx = 0;
    for (int n = 1; n <= H; ++n) {
      idx += k;
      if (idx >= N) idx -= N;
      acc += s[n] * c.eq_cos[idx];
    }
    float pk = A[k] * acc * (k == 0 ? 1.f : 2.f) / float(N);
    const float* row = c.eq_band + k * 8;
#pragma unroll
    for (int b = 0; b < 8; ++b) bsum[b] += row[b] * pk;
  }
  // block reduce 8 values (two passes of 4)
  float lo[4] = {bsum[0], bsum[1], bsum[2], bsum[3]}, hi[4] = {bsum[4], bsum[5], bsum[6], bsum[7]};
  block_sum<4>(lo, red);
  block_sum<4>(hi, red + 4 * 32);
  if (threadIdx.x == 0) {
    float* d = c.dparams + nd.prow * 8;
    for (int b = 0; b < 4; ++b) {
      d[b] = LN10_20 * lo[b];
      d[b + 4] = LN10_20 * hi[b];
    }
  }
}

template <int M>
static size_t design_smem() { return sizeof(float2) * fft::Padded<M>::size + sizeof(float) * (1024 + 1024 + 4); }

template <int M>
static int eq_launch(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  constexpr int T = M / 16;
  static bool init = false;
  const size_t s1 = sizeof(float2) * fft::Padded<M>::size;
  if (!init) {
    cudaFuncSetAttribute(k_eq_design<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(design_smem<M>()));
    cudaFuncSetAttribute(k_eq_fwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s1));
    cudaFuncSetAttribute(k_eq_bwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(2 * s1));
    cudaFuncSetAttribute(k_eq_finalize<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(design_smem<M>()));
    init = true;
  }
  switch (what) {
    case 0: k_eq_design<M><<<b - a, T, design_smem<M>(), s>>>(c, a); break;
    case 1: k_eq_fwd<M><<<grid_size(b, (228 * 1024) / int(s1 + 1024)), T, s1, s>>>(c, a, b); break;
    case 2: k_eq_bwd<M><<<grid_size(b, (228 * 1024) / int(2 * s1 + 1024)), T, 2 * s1, s>>>(c, a, b); break;
    case 3: k_eq_finalize<M><<<b - a, T, design_smem<M>(), s>>>(c, a); break;
  }
  return 1;
}

// what: 0 design(node range), 1 fwd(items), 2 bwd(items), 3 finalize(node range)
int launch_eq(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  if (b <= 0 || (what == 0 || what == 3) && b <= a) return 0;
  switch (c.eq_fft) {
    case 1024: return eq_launch<1024>(what, c, a, b, s);
    case 2048: return eq_launch<2048>(what, c, a, b, s);
    case 4096: return eq_launch<4096>(what, c, a, b, s);
    default: return eq_launch<8192>(what, c, a, b, s);
  }
}

}  // namespace grafx
