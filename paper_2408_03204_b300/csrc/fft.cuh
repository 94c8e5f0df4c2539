// Shared-memory complex FFT for the block convolutions and the STFT loss.
//
// Stockham auto-sort formulation: M = 16^a * r points, one radix-16 pass per factor
// 16 and one final radix-r pass (r in {2, 4, 8, 16}).  A transform is run by
// T = M/16 threads; thread `tid` owns M/(16 T) = 1 radix-16 butterfly per pass (or
// 16/r radix-r butterflies in the last pass), so every pass is: load the
// butterfly inputs from shared memory into registers, barrier, apply the
// twiddles W_{Ns R}^{r k} and an in-register DFT_R, write to the auto-sorted
// positions, barrier.  Shared-memory indices are padded (i + i/16) so that the
// stride-16 writes of the first pass are free of bank conflicts.
//
// Twiddles come from per-pass tables (ptw_*) built on the host in double precision.  The forward transform uses exp(-2 pi i k n / M); an inverse is
// obtained by conjugating the input and the output.
//
// The pass bodies are __host__ __device__ so that a CPU harness can run the same
// arithmetic thread by thread.
#pragma once
#include "devtypes.h"

#ifdef __CUDACC__
#define GX_HD __host__ __device__ __forceinline__
#else
#define GX_HD inline
struct float2 { float x, y; };
inline float2 make_float2(float x, float y) { return float2{x, y}; }
#endif

namespace grafx {
namespace fft {

GX_HD int pad(int i) { return i + (i >> 4); }
template <int M> struct Padded { static constexpr int size = M + M / 16; };

GX_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
GX_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
GX_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
GX_HD float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
GX_HD float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

// exp(-2 pi i m / 16) for the in-register radix-16 twiddles (m = n2*k1 <= 9)
GX_HD float2 w16(int m) {
  const float c = 0.92387953251128674f, s = 0.38268343236508978f, h = 0.70710678118654752f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c, -s);
    case 2: return make_float2(h, -h);
    case 3: return make_float2(s, -c);
    case 4: return make_float2(0.f, -1.f);
    case 6: return make_float2(-h, -h);
    default: return make_float2(-c, s);  // m = 9
  }
}
GX_HD float2 w8(int m) {
  const float h = 0.70710678118654752f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(h, -h);
    case 2: return make_float2(0.f, -1.f);
    default: return make_float2(-h, -h);  // m = 3
  }
}

GX_HD void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
// forward 4-point DFT of (x0, x1, x2, x3) in place
GX_HD void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_mi(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <int R> struct Dft;
template <> struct Dft<2> {
  GX_HD static void run(float2* v) { dft2(v[0], v[1]); }
};
template <> struct Dft<4> {
  GX_HD static void run(float2* v) { dft4(v[0], v[1], v[2], v[3]); }
};
// 8 = 4 x 2: inner DFT4 over n1 of x[2 n1 + n2], twiddle W8^(n2 k1), outer DFT2;
// output X[k1 + 4 k2]
template <> struct Dft<8> {
  GX_HD static void run(float2* v) {
    float2 a[2][4];
#pragma unroll
    for (int n2 = 0; n2 < 2; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[2 * n1 + n2];
      dft4(a[n2][0], a[n2][1], a[n2][2], a[n2][3]);
    }
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[1][k1] = cmul(a[1][k1], w8(k1));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 p = a[0][k1], q = a[1][k1];
      dft2(p, q);
      v[k1] = p;
      v[k1 + 4] = q;
    }
  }
};
// 16 = 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle W16^(n2 k1), outer DFT4
template <> struct Dft<16> {
  GX_HD static void run(float2* v) {
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[4 * n1 + n2];
      dft4(a[n2][0], a[n2][1], a[n2][2], a[n2][3]);
    }
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) a[n2][k1] = cmul(a[n2][k1], w16(n2 * k1));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 x0 = a[0][k1], x1 = a[1][k1], x2 = a[2][k1], x3 = a[3][k1];
      dft4(x0, x1, x2, x3);
      v[k1] = x0;
      v[k1 + 4] = x1;
      v[k1 + 8] = x2;
      v[k1 + 12] = x3;
    }
  }
};

// Pass geometry: pass p (p = 0..npass-1) merges Ns = 16^p points into 16^p * R_p with
// R_p = 16, except the last pass of an M that is not a power of 16 (radix M / 16^n16).
GX_HD constexpr int geo_n16(int M) { return M >= 4096 ? 3 : M >= 256 ? 2 : 1; }
// (iterative, so that device code inlines and folds them instead of calling a recursion)
GX_HD constexpr int ipow16(int p) {
  int r = 1;
  for (int i = 0; i < p; ++i) r *= 16;
  return r;
}
GX_HD constexpr int geo_last(int M) { return M / ipow16(geo_n16(M)); }
GX_HD constexpr int geo_npass(int M) { return geo_n16(M) + (geo_last(M) > 1 ? 1 : 0); }
GX_HD constexpr int pass_radix(int M, int p) { return (p == geo_npass(M) - 1 && geo_last(M) > 1) ? geo_last(M) : 16; }

// Pass twiddle tables: for every pass p >= 1 of an M-point transform, the entries
// W_{Ns R}^{r k} = exp(-2 pi i r k / (Ns R)) for r in [1, R), k in [0, Ns), stored at
// [(r-1) Ns + k] so that the threads of a warp (consecutive k) read consecutive
// entries.  The tables of M = 512, 1024, ..., 8192 are concatenated in that order.
GX_HD constexpr int ptw_pass_size(int M, int p) { return p == 0 ? 0 : (pass_radix(M, p) - 1) * ipow16(p); }
GX_HD constexpr int ptw_pass_off(int M, int p) {
  int o = 0;
  for (int q = 0; q < p; ++q) o += ptw_pass_size(M, q);
  return o;
}
GX_HD constexpr int ptw_size(int M) { return ptw_pass_off(M, geo_npass(M)); }
GX_HD constexpr int ptw_base(int M) {
  int o = 0;
  for (int m = 512; m < M; m *= 2) o += ptw_size(m);
  return o;
}
constexpr int PTW_TOTAL = ptw_base(8192) + ptw_size(8192);

// Pass geometry of an M-point transform.
template <int M> struct Geo {
  static constexpr int T = M / 16;  // threads per transform
  static constexpr int n16 = (M >= 65536) ? 4 : (M >= 4096) ? 3 : (M >= 256) ? 2 : 1;
  static constexpr int last = M / (n16 == 3 ? 4096 : n16 == 2 ? 256 : 16);  // radix of the final pass (1 = none)
  static constexpr int npass = n16 + (last > 1 ? 1 : 0);
};

// Phase 1 of a pass: read the butterfly inputs of thread `tid`.
template <int M, int R>
GX_HD void pass_load(const float2* buf, int tid, float2 (*v)[R]) {
  constexpr int T = M / 16, BPT = 16 / R;
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    int j = tid + b * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = buf[pad(j + r * (M / R))];
  }
}

// Phase 2 of a pass: twiddle, DFT_R, auto-sorted store.  Ns = points already merged;
// tw = this pass's twiddle table (see ptw_pass_off).
template <int M, int R>
GX_HD void pass_store(float2* buf, const float2_* tw, int tid, int Ns, float2 (*v)[R]) {
  constexpr int T = M / 16, BPT = 16 / R;
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    int j = tid + b * T;
    int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2_ w = tw[(r - 1) * Ns + k];
        v[b][r] = cmul(v[b][r], make_float2(w.x, w.y));
      }
    }
    Dft<R>::run(v[b]);
    int out = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad(out + r * Ns)] = v[b][r];
  }
}

// Twiddle + DFT_R of the butterflies of thread `tid` in the pass that has merged Ns
// points, without storing; results stay in v[b][r] (output position
// (j - k) R + k + r Ns for butterfly j = tid + b T, k = j mod Ns).
template <int M, int R>
GX_HD void pass_compute(const float2_* tw, int tid, int Ns, float2 (*v)[R]) {
  constexpr int T = M / 16, BPT = 16 / R;
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    int j = tid + b * T;
    int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2_ w = tw[(r - 1) * Ns + k];
        v[b][r] = cmul(v[b][r], make_float2(w.x, w.y));
      }
    }
    Dft<R>::run(v[b]);
  }
}

// 384-point transform (the paper reverb's STFT size), 384 = 3 x 128.  With j = 128 j1 + j2
// and k = k1 + 3 k2:
//   X[k1 + 3 k2] = sum_{j2} W_128^{j2 k2} W_384^{j2 k1} sum_{j1} x[128 j1 + j2] W_3^{j1 k1},
// i.e. a radix-3 stage over the three rows x[128 j1 + .] with the twiddles W_384^{j2 k1},
// then a 128-point Stockham transform of each row (a radix-16 pass, then a radix-8 pass
// with the table W_128^{r k} at [(r-1) 16 + k], r < 8, k < 16).  Layout: three padded
// rows of 128 points, row r at r * R128; x[j] enters at in384(j), X[k] leaves at out384(k).
constexpr int R128 = Padded<128>::size;
GX_HD int in384(int j) { return (j >> 7) * R128 + pad(j & 127); }
GX_HD int out384(int k) { return (k % 3) * R128 + pad(k / 3); }

// The radix-3 stage for column j2 (< 128), in place.  cs[m] = (cos, sin)(2 pi m / 384).
GX_HD void r3_stage384(float2* buf, int j2, const float2_* cs) {
  const float s3 = 0.86602540378443865f;   // sin(2 pi / 3)
  float2* a = buf + pad(j2);
  const float2 x0 = a[0], x1 = a[R128], x2 = a[2 * R128];
  const float2 t = cadd(x1, x2), d = csub(x1, x2);
  const float2 h = make_float2(x0.x - 0.5f * t.x, x0.y - 0.5f * t.y);
  float2 y1 = make_float2(h.x + s3 * d.y, h.y - s3 * d.x);   // x0 + x1 W_3 + x2 W_3^2
  float2 y2 = make_float2(h.x - s3 * d.y, h.y + s3 * d.x);   // x0 + x1 W_3^2 + x2 W_3^4
  const float2_ w1 = cs[j2], w2 = cs[2 * j2];                // W_384^m = (cos, -sin)
  y1 = cmul(y1, make_float2(w1.x, -w1.y));
  y2 = cmul(y2, make_float2(w2.x, -w2.y));
  a[0] = cadd(x0, t);
  a[R128] = y1;
  a[2 * R128] = y2;
}

#ifdef __CUDACC__
// Full forward transform of one M-point padded buffer by threads tid in [0, M/16).
// Every thread of the CTA must call it (it contains __syncthreads); threads with
// tid >= M/16 pass `active = false`.  The caller synchronises before the first pass.
// ptw: the concatenated pass twiddle tables (PTW_TOTAL entries).
template <int M>
__device__ __forceinline__ void forward(float2* buf, const float2_* __restrict__ ptw, int tid, bool active) {
  const float2_* tw = ptw + ptw_base(M);
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < Geo<M>::n16; ++p) {
    float2 v[1][16];
    if (active) pass_load<M, 16>(buf, tid, v);
    __syncthreads();
    if (active) pass_store<M, 16>(buf, tw + ptw_pass_off(M, p), tid, Ns, v);
    __syncthreads();
    Ns *= 16;
  }
  if constexpr (Geo<M>::last > 1) {
    constexpr int R = Geo<M>::last;
    float2 v[16 / R][R];
    if (active) pass_load<M, R>(buf, tid, v);
    __syncthreads();
    if (active) pass_store<M, R>(buf, tw + ptw_pass_off(M, Geo<M>::n16), tid, Ns, v);
    __syncthreads();
  }
}

// Forward 384-point transforms of F frames (frame f at buf + f * 3 * R128, layout
// in384 -> out384) by a CTA of at least 24 F threads; every thread calls it (barriers).
// The caller synchronises before it; tw128: W_128^{r k} at [(r-1) 16 + k].
template <int F>
__device__ __forceinline__ void forward384(float2* buf, const float2_* cs, const float2_* tw128) {
  for (int i = threadIdx.x; i < F * 128; i += blockDim.x) r3_stage384(buf + (i >> 7) * 3 * R128, i & 127, cs);
  __syncthreads();
  const int t = threadIdx.x;
  const bool act = t < 24 * F;
  float2* rb = buf + (act ? (t / 24) * 3 * R128 + ((t >> 3) % 3) * R128 : 0);
  const int t8 = t & 7;
  {
    float2 v[1][16];
    if (act) pass_load<128, 16>(rb, t8, v);
    __syncthreads();
    if (act) pass_store<128, 16>(rb, tw128, t8, 1, v);
    __syncthreads();
  }
  {
    float2 v[2][8];
    if (act) pass_load<128, 8>(rb, t8, v);
    __syncthreads();
    if (act) pass_store<128, 8>(rb, tw128, t8, 16, v);
    __syncthreads();
  }
}

// Forward transform with the data in registers on both ends: on entry thread tid holds
// x[tid + T m] in v[m] (m < 16, T = M/16); on exit it holds X[tid + T m].  Stockham's
// first pass reads exactly that layout and its last pass writes it, so only the inner
// passes go through shared memory, alternating between b0 and b1 (one barrier per
// pass).  The caller guarantees that no thread still reads b0 when this is entered;
// on exit other threads may still read the buffer of the last inner pass: b1 when the
// pass count is odd, b0 when it is even.
// tw: this size's pass tables (ptw + ptw_base(M)), in global or shared memory.
template <int M>
__device__ __forceinline__ void forward_regs_tw(float2 (&v)[16], float2* b0, float2* b1, const float2_* tw, int tid) {
  constexpr int n16 = Geo<M>::n16, last = Geo<M>::last;
  constexpr int npass = n16 + (last > 1 ? 1 : 0);
  float2* bufs[2] = {b0, b1};
  // pass 1: radix 16, Ns = 1, from registers
  {
    float2(*w)[16] = reinterpret_cast<float2(*)[16]>(v);
    Dft<16>::run(w[0]);
#pragma unroll
    for (int r = 0; r < 16; ++r) b0[pad(tid * 16 + r)] = v[r];
  }
  __syncthreads();
  int Ns = 16;
  int cur = 0;
#pragma unroll
  for (int p = 1; p < npass; ++p) {
    const bool is_last = (p == npass - 1);
    const int R = (is_last && last > 1) ? last : 16;
    if (R == 16) {
      float2 w[1][16];
      pass_load<M, 16>(bufs[cur], tid, w);
      pass_compute<M, 16>(tw + ptw_pass_off(M, p), tid, Ns, w);
      if (is_last) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = w[0][r];
      } else {
        const int j = tid, k = j & (Ns - 1), out = (j - k) * 16 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) bufs[cur ^ 1][pad(out + r * Ns)] = w[0][r];
      }
    } else if constexpr (last > 1 && last < 16) {
      constexpr int RL = last, BPT = 16 / RL;
      float2 w[BPT][RL];
      pass_load<M, RL>(bufs[cur], tid, w);
      pass_compute<M, RL>(tw + ptw_pass_off(M, p), tid, Ns, w);
#pragma unroll
      for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) v[b + r * BPT] = w[b][r];
    }
    if (!is_last) {
      __syncthreads();
      cur ^= 1;
      Ns *= 16;
    }
  }
}
template <int M>
__device__ __forceinline__ void forward_regs(float2 (&v)[16], float2* b0, float2* b1,
                                             const float2_* __restrict__ ptw, int tid) {
  forward_regs_tw<M>(v, b0, b1, ptw + ptw_base(M), tid);
}

// forward_regs with one shared buffer: the same register layouts on entry (x[tid + T m])
// and exit (X[tid + T m]), every inner pass reading the whole buffer into registers,
// a barrier, then writing it back.  The caller guarantees that no thread still reads buf
// when this is entered; on exit other threads may still read it.  All threads of the
// CTA call it (barriers); ptw: the concatenated pass tables.
template <int M>
__device__ __forceinline__ void forward_regs_1buf_tw(float2 (&v)[16], float2* buf, const float2_* tw, int tid) {
  constexpr int n16 = Geo<M>::n16, last = Geo<M>::last;
  constexpr int npass = n16 + (last > 1 ? 1 : 0);
  {  // pass 1: radix 16, Ns = 1, from registers
    float2(*w)[16] = reinterpret_cast<float2(*)[16]>(v);
    Dft<16>::run(w[0]);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[pad(tid * 16 + r)] = v[r];
  }
  __syncthreads();
  int Ns = 16;
#pragma unroll
  for (int p = 1; p < npass; ++p) {
    const bool is_last = (p == npass - 1);
    const int R = (is_last && last > 1) ? last : 16;
    if (R == 16) {
      float2 w[1][16];
      pass_load<M, 16>(buf, tid, w);
      if (!is_last) __syncthreads();   // every thread has read before any writes
      pass_compute<M, 16>(tw + ptw_pass_off(M, p), tid, Ns, w);
      if (is_last) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = w[0][r];
      } else {
        const int j = tid, k = j & (Ns - 1), out = (j - k) * 16 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[pad(out + r * Ns)] = w[0][r];
        __syncthreads();
      }
    } else if constexpr (last > 1 && last < 16) {
      constexpr int RL = last, BPT = 16 / RL;
      float2 w[BPT][RL];
      pass_load<M, RL>(buf, tid, w);
      pass_compute<M, RL>(tw + ptw_pass_off(M, p), tid, Ns, w);
#pragma unroll
      for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) v[b + r * BPT] = w[b][r];
    }
    if (!is_last) Ns *= 16;
  }
}
// tw of forward_regs_1buf_tw: this size's pass tables (ptw + ptw_base(M)), in global or
// shared memory
template <int M>
__device__ __forceinline__ void forward_regs_1buf(float2 (&v)[16], float2* buf, const float2_* __restrict__ ptw,
                                                  int tid) {
  forward_regs_1buf_tw<M>(v, buf, ptw + ptw_base(M), tid);
}
#endif

}  // namespace fft
}  // namespace grafx
