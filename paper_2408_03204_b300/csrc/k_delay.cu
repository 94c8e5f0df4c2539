// Multitap delay (Sec. 3 "Multitap delay", Eq. 14-15).
//
// Per channel x and tap m: a 39-tap zero-phase FIR c_{x,m} built like the equalizer
// from 20 log-magnitudes, and a complex z_{x,m} whose phase gives the integer delay
// d = m S + (round(N_d (-arg z) / 2 pi) mod N_d).  Compact layout: 4 taps, S = 0,
// N_d = 32768.  Slot layout (the paper's 2 s effect): 20 taps, tap m in its own 100 ms
// slot, S = N_d = fs / 10.  Forward (exact, as the paper's straight-through estimator
// prescribes): y_x[t] = sum_m sum_j c[j] u_x[t - d_m - j], a sparse FIR run from
// shared-memory windows, two taps' windows staged at a time.  Backward:
//   * input adjoint: the transposed sparse FIR over ybar;
//   * FIR taps: dL/dc_m[j] = r_x[d_m + j] with r_x[n] = sum_t ybar_x[t] u_x[t - n];
//   * z (surrogate of Eq. 15 placed at the slot, s[n] = Re{(1/N_d) sum_k z^k w^{k(n - m S)}}):
//     with g[n] = sum_j c[j] r_x[m S + n + j] = dL/ds[m S + n] over n in [0, N_d),
//     Q = sum_n g[n] phi[n], phi[n] = (1/N_d) sum_k k z^{k-1} w^{kn}, and
//     dL/dRe z = Re Q, dL/dIm z = -Im Q.  phi has the closed form
//     F(q)/(N_d z), q = z w^n, F(q) = sum_k k q^k = (-a (1 + (N_d - 1) z^N) - b) / a^2
//     with a = 1 - q and b = z^N - 1 evaluated without cancellation; within
//     |N_d ln q| < 1/2 (the lag next to the delay) F uses its Taylor series in
//     t = N_d ln q instead.
// The correlation r over the lags [-19, reach + 19), reach = (M - 1) S + N_d, is a
// partitioned frequency-domain accumulation: 8192-point spectra of 2B-sample windows
// of u and of B-sample blocks of ybar (B = 4096, both channels packed as l + i r),
// R_p = sum_b X_{b-p} conj(Ybar_b) per lag partition p (P partitions of B lags from
// -B), one inverse FFT per partition.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {

// The row feeding node v (forward) or the adjoint row of its only consumer (adjoint)
// when there is exactly one, else nullptr (the window is then summed over the edges).
template <bool ADJ>
__device__ __forceinline__ const float* dl_single_row(const DevCtx& c, int v) {
  const int e0 = ADJ ? c.tcsr_ptr[v] : c.csr_ptr[v];
  const int e1 = ADJ ? c.tcsr_ptr[v + 1] : c.csr_ptr[v + 1];
  if (e1 - e0 != 1) return nullptr;
  return ADJ ? out_adj_row(c, e0) : in_row(c, e0);
}

// Shared-memory index of window element i: 4 floats of padding after every 16, so that
// the float4 reads of threads 16 elements apart (20 floats in shared memory: 8 lanes per
// 32 banks) do not collide, and a thread's reads sit at fixed offsets from its first.
__device__ __forceinline__ int dl_pidx(int i) { return i + ((i >> 4) << 2); }

// Window of one tap for a tile of one channel summed over several rows (padded layout).
template <bool ADJ>
__device__ __forceinline__ void dl_window_sum(const DevCtx& c, int v, const NodeDev& nd, int ch, int start,
                                              float* win, int n) {
  const int e0 = ADJ ? c.tcsr_ptr[v] : c.csr_ptr[v];
  const int e1 = ADJ ? c.tcsr_ptr[v + 1] : c.csr_ptr[v + 1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int t = start + i;
    float s = 0.f;
    if (t >= 0 && t < nd.len)
      for (int e = e0; e < e1; ++e) s += (ADJ ? out_adj_row(c, e) : in_row(c, e))[ch * nd.pitch + t];
    win[dl_pidx(i)] = s;
  }
}

constexpr int DL_GROUP = 2;                  // taps whose windows are staged together
constexpr int DL_OPT = 16;                   // consecutive outputs per thread
constexpr int DL_FT = DL_TILE / DL_OPT;      // threads of the FIR kernels
constexpr int DL_SH = DL_FIR + 3;            // taps of the shifted filters (alignment shift 0..3)
constexpr int DL_XL = (DL_OPT + DL_SH - 1 + 3) & ~3;   // window floats a thread reads (15 float4)
constexpr int DL_WL = DL_OPT * (DL_FT - 1) + DL_XL;     // window floats staged (16-byte groups)
constexpr int DL_WP = DL_WL + ((DL_WL + 15) / 16) * 4;  // padded window floats
static_assert(DL_OPT % 16 == 0, "a thread's window starts on a padding segment");
static_assert(DL_WL % 4 == 0 && DL_WL >= DL_TILE + DL_SH - 1, "window covers the tile");

// Forward (ADJ = false) or input adjoint (ADJ = true) of the sparse FIR for one
// (node, tile, channel) item; DL_FT threads x DL_OPT consecutive outputs.  A tap's window
// starts at s = t0 -+ d - H, which has any alignment; it is staged from s0 = s rounded down
// to a multiple of 4 with 16-byte copies (zero-filled outside the signal), and the
// misalignment o = s - s0 moves into the filter instead: the tap's 39 coefficients are
// placed in a 42-tap filter at offset 3 - o (forward) or o (adjoint), so every thread runs
// the same unrolled loop over aligned float4 reads.  The windows of a group of DL_GROUP
// taps are staged while the previous group is computed (cp.async from a single source
// row; a sum over several rows is staged synchronously), double-buffered, with 4 floats of
// padding after every 16 so that the threads' float4 reads (16 floats apart) fall in
// distinct banks.
template <bool ADJ>
__global__ void __launch_bounds__(DL_FT) k_delay_fir(DevCtx c, int item0, int n_items) {
  __shared__ __align__(16) float win[2][DL_GROUP][DL_WP];
  __shared__ __align__(16) float taps[DL_SLOT_TAPS][DL_SH + 2];   // rows of 44: float4 reads
  __shared__ int wst[DL_SLOT_TAPS];                                // aligned window starts
  constexpr int H = (DL_FIR - 1) / 2;
  const int ntap = c.dl_taps;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t0 = w.y, ch = w.z;
    const NodeDev nd = c.nodes[v];
    const float* aux = c.dl_aux + size_t(c.ext[v].z) * 2 * ntap * (DL_FIR + 1) + size_t(ch) * ntap * (DL_FIR + 1);
    const float* single = dl_single_row<ADJ>(c, v);
    __syncthreads();   // readers of the previous item's taps and windows are done
    for (int m = threadIdx.x; m < ntap; m += blockDim.x) {
      const int d = int(aux[m * (DL_FIR + 1) + DL_FIR]);
      const int st = ADJ ? t0 + d - H : t0 - d - H;     // window start (forward: u[t0 - d - H + k])
      wst[m] = st - (((st % 4) + 4) % 4);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ntap * (DL_SH + 2); i += blockDim.x) {
      const int m = i / (DL_SH + 2), jp = i % (DL_SH + 2);
      const int d = int(aux[m * (DL_FIR + 1) + DL_FIR]);
      const int o = (ADJ ? t0 + d - H : t0 - d - H) - wst[m];
      const int j = ADJ ? jp - o : jp - (3 - o);       // the original tap index at shifted position jp
      taps[m][jp] = (jp < DL_SH && j >= 0 && j < DL_FIR) ? aux[m * (DL_FIR + 1) + j] : 0.f;
    }
    __syncthreads();
    // window k of tap m: u[s0 + k] (forward) or ybar[s0 + k] (adjoint), s0 = wst[m]
    auto stage = [&](int g0, int buf) {
      const int ng = min(DL_GROUP, ntap - g0);
      for (int m = 0; m < ng; ++m) {
        const int s0 = wst[g0 + m];
        if (single) {
          const float* row = single + size_t(ch) * nd.pitch;
          if (s0 >= 0 && s0 + DL_WL <= nd.len) {   // the whole window inside the signal
            for (int q = threadIdx.x; q < DL_WL / 4; q += blockDim.x)
              cp_async16(&win[buf][m][dl_pidx(4 * q)], row + s0 + 4 * q, 16);
          } else {
            for (int q = threadIdx.x; q < DL_WL / 4; q += blockDim.x) {
              const int t = s0 + 4 * q;   // a multiple of 4: the quad lies wholly before 0 or starts inside
              const int nbytes = (t < 0 || t >= nd.len) ? 0 : 4 * min(4, nd.len - t);
              cp_async16(&win[buf][m][dl_pidx(4 * q)], nbytes ? row + t : row, nbytes);
            }
          }
        } else {
          dl_window_sum<ADJ>(c, v, nd, ch, s0, win[buf][m], DL_WL);
        }
      }
      cp_async_commit();
    };
    stage(0, 0);
    float acc[DL_OPT];
#pragma unroll
    for (int q = 0; q < DL_OPT; ++q) acc[q] = 0.f;
    const int i0 = DL_OPT * threadIdx.x;
    for (int g0 = 0, buf = 0; g0 < ntap; g0 += DL_GROUP, buf ^= 1) {
      if (g0 + DL_GROUP < ntap) stage(g0 + DL_GROUP, buf ^ 1);
      else cp_async_commit();   // an empty group keeps the wait count uniform
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this group's windows landed
      __syncthreads();
      const int ng = min(DL_GROUP, ntap - g0);
      for (int m = 0; m < ng; ++m) {
        float x[DL_XL];
        const float* wb = win[buf][m] + dl_pidx(i0);   // i0 starts a padding segment
#pragma unroll
        for (int k = 0; k < DL_XL / 4; ++k) {   // a float4 never crosses a padding point
          const float4 q4 = *reinterpret_cast<const float4*>(wb + dl_pidx(4 * k));
          x[4 * k] = q4.x, x[4 * k + 1] = q4.y, x[4 * k + 2] = q4.z, x[4 * k + 3] = q4.w;
        }
        const float4* t4 = reinterpret_cast<const float4*>(taps[g0 + m]);
#pragma unroll
        for (int j4 = 0; j4 < (DL_SH + 2) / 4; ++j4) {
          const float4 c4 = t4[j4];   // the same address in every lane: one broadcast
          const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int jj = 4 * j4 + r;
            if (jj < DL_SH)
#pragma unroll
              for (int q = 0; q < DL_OPT; ++q) acc[q] += cs[r] * x[q + (ADJ ? jj : DL_SH - 1 - jj)];
          }
        }
      }
      __syncthreads();   // readers of win[buf] are done before it is staged again
    }
    float* row = (ADJ ? arow_w(c, nd) : yrow_w(c, nd)) + ch * nd.pitch;
    if (t0 + i0 + DL_OPT <= nd.len) {   // t0 + i0 is a multiple of 4 (16-byte rows)
#pragma unroll
      for (int q = 0; q < DL_OPT; q += 4)
        st4(row + t0 + i0 + q, make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]));
    } else {
#pragma unroll
      for (int q = 0; q < DL_OPT; ++q) {
        const int t = t0 + i0 + q;
        if (t < nd.pitch) row[t] = t < nd.len ? acc[q] : 0.f;
      }
    }
  }
}

// cos(2 pi j / 39) and the 39-tap design's Hann v[j - H] = 0.5 (1 + cos(2 pi (j - H) / 40)).
__device__ __forceinline__ void dl_tables(float* cos39, float* hann39) {
  constexpr int H = (DL_FIR - 1) / 2;
  if (threadIdx.x < DL_FIR) {
    cos39[threadIdx.x] = cospif(2.f * float(threadIdx.x) / float(DL_FIR));
    hann39[threadIdx.x] = 0.5f * (1.f + cospif(2.f * float(int(threadIdx.x) - H) / float(DL_FIR + 1)));
  }
}

// Per delay node: the taps c_{x,m} (Eq. 4 with N = 39, K = 20; FP32 with exp and cosine
// tables, the cosine indexed exactly by (k |n|) mod 39) and the delays
// d_{x,m} = m S + (round(N_d (-arg z) / 2 pi) mod N_d).
__global__ void k_delay_design(DevCtx c, int node_begin) {
  __shared__ float A[2 * DL_SLOT_TAPS][DL_K];
  __shared__ float cos39[DL_FIR], hann39[DL_FIR];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const int ntap = c.dl_taps, Nd = c.dl_nd;
  float* aux = c.dl_aux + size_t(c.ext[v].z) * 2 * ntap * (DL_FIR + 1);
  const float* p = c.params + size_t(nd.prow) * c.pcols;
  constexpr int H = (DL_FIR - 1) / 2, K = DL_K;
  for (int i = threadIdx.x; i < 2 * ntap * K; i += blockDim.x) A[i / K][i % K] = expf(p[(i / K) * DL_ROW + 2 + i % K]);
  dl_tables(cos39, hann39);
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * ntap * DL_FIR; i += blockDim.x) {
    const int xm = i / DL_FIR, j = i % DL_FIR, an = j < H ? H - j : j - H;
    float s = 0.f;
    int idx = 0;   // (k |n|) mod 39
    for (int k = 1; k < K; ++k) {
      idx += an;
      if (idx >= DL_FIR) idx -= DL_FIR;
      s += A[xm][k] * cos39[idx];
    }
    aux[xm * (DL_FIR + 1) + j] = hann39[j] * (A[xm][0] + 2.f * s) / float(DL_FIR);
  }
  for (int xm = threadIdx.x; xm < 2 * ntap; xm += blockDim.x) {
    const float* q = p + xm * DL_ROW;
    const double ang = atan2(double(q[1]), double(q[0]));
    long long d = llrint(double(Nd) * (-ang) / (2.0 * M_PI));
    d %= Nd;
    if (d < 0) d += Nd;
    aux[xm * (DL_FIR + 1) + DL_FIR] = float(d + (long long)(xm % ntap) * c.dl_slot);
  }
}

// 8192-point spectrum of a u window (kind 0: samples [w B, w B + 2B)) or of a ybar
// block (kind 1: samples [b B, b B + B), zero-padded), both channels packed l + i r.
// Windows that hold no sample of the signal (those before its start and past its end)
// get the zero spectrum without a transform.
__global__ void __launch_bounds__(DL_M / 16, 2) k_delay_spec(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  constexpr int T = DL_M / 16;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, idx = w.y, kind = w.z;
    const NodeDev nd = c.nodes[v];
    // kind 0: u window of 2B; 1: ybar block of B (zero-padded); 2: ybar window of 2B
    const bool adj = kind != 0;
    const int start = idx * DL_B, count = kind == 1 ? DL_B : 2 * DL_B;
    float2* out = c.dl_spec + size_t(w.w) * DL_M;
    if (start + count <= 0 || start >= nd.len) {   // no sample of the signal: the zero spectrum
      for (int k = threadIdx.x; k < DL_M; k += blockDim.x) out[k] = make_float2(0.f, 0.f);
      continue;   // uniform over the CTA
    }
    const int e0 = adj ? c.tcsr_ptr[v] : c.csr_ptr[v];
    const int e1 = adj ? c.tcsr_ptr[v + 1] : c.csr_ptr[v + 1];
    const float* single = e1 - e0 == 1 ? (adj ? out_adj_row(c, e0) : in_row(c, e0)) : nullptr;
    // thread t takes samples start + t + T m (m < 16) straight into the registers of the
    // transform's first pass, all loads issued together
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int i = threadIdx.x + T * m, t = start + i;
      float l = 0.f, r = 0.f;
      if (i < count && t >= 0 && t < nd.len) {
        if (single) {
          l = single[t];
          r = single[nd.pitch + t];
        } else {
          for (int e = e0; e < e1; ++e) {
            const float* row = adj ? out_adj_row(c, e) : in_row(c, e);
            l += row[t];
            r += row[nd.pitch + t];
          }
        }
      }
      x[m] = make_float2(l, r);
    }
    __syncthreads();   // readers of buf (the previous item's last pass) are done
    fft::forward_regs_1buf<DL_M>(x, buf, c.ptw, threadIdx.x);
#pragma unroll
    for (int m = 0; m < 16; ++m) out[threadIdx.x + T * m] = x[m];
  }
}

// cp.async of 8 bytes (both addresses 8-byte aligned) into shared memory.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// R_p[k] for one node and DL_CHUNK bins, all lag partitions: per channel
// sum_b X_{b-p}[k] conj(Ybar_b[k]), packed as R_l + i R_r for the joint inverse.  The
// per-channel products of real signals' spectra are conjugate-symmetric, so the work
// items cover bins 0..M/2 and bin M - k is written from bin k.  Launched with
// DL_CHUNK * ceil(dl_P / DL_NPT) threads (one per bin and group of DL_NPT partitions;
// DL_NPT = 4 where that leaves no more unused partition slots than pairs do, else 2).
template <int DL_NPT>
__global__ void __launch_bounds__(DL_CHUNK * DL_PMAX) k_delay_acc(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 sm[];
  const int P = c.dl_P;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, k0 = w.y * DL_CHUNK;
    const int4_ e = c.ext[v];
    const int nb = e.w, nw = nb + P;
    float2* X = sm;                         // [nw][DL_CHUNK][2 ch]
    float2* Y = sm + size_t(nw) * DL_CHUNK * 2;
    __syncthreads();
    // Z[k] and Z[M - k] of every staged spectrum copied asynchronously (all of a thread's
    // copies in flight together), then split in place into the channels' spectra:
    // l = (Z[k] + conj(Z[-k]))/2, r = (Z[k] - conj(Z[-k]))/(2i).  X and Y are contiguous.
    const int n_el = (nw + nb) * DL_CHUNK;
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
      const int s = i / DL_CHUNK, kk = i % DL_CHUNK, k = k0 + kk, km = (DL_M - k) & (DL_M - 1);
      float2* dst = X + size_t(i) * 2;
      if (s < P - 1) {   // u windows w = s - P < -1 hold no sample: zero spectra, never written
        dst[0] = make_float2(0.f, 0.f);
        dst[1] = make_float2(0.f, 0.f);
      } else {
        const float2* spec = c.dl_spec + size_t(e.x + s) * DL_M;
        cp_async8(dst, spec + k);
        cp_async8(dst + 1, spec + km);
      }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
      float2* dst = X + size_t(i) * 2;
      const float2 z = dst[0], zm = dst[1];
      dst[0] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      dst[1] = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    }
    __syncthreads();
    // thread (group q, bin kk) accumulates partitions p = DL_NPT q + j, j < DL_NPT: partition
    // p0 + j at block b uses the window partition p0 used at block b - j, carried in
    // registers (one window and one ybar block read per block for DL_NPT partitions)
    const int kk = threadIdx.x % DL_CHUNK, p0 = DL_NPT * (threadIdx.x / DL_CHUNK);
    // wl[j], wr[j]: window b - p0 - j once block b has shifted it in; before block 0 they
    // hold window -p0 - 1 - j (stored at P - p0 - 1 - j; below 0 only for partitions >= P)
    float2 al[DL_NPT], ar[DL_NPT], wl[DL_NPT], wr[DL_NPT];
#pragma unroll
    for (int j = 0; j < DL_NPT; ++j) {
      al[j] = ar[j] = make_float2(0.f, 0.f);
      const int s0 = P - p0 - 1 - j;
      wl[j] = s0 >= 0 ? X[(size_t(s0) * DL_CHUNK + kk) * 2] : make_float2(0.f, 0.f);
      wr[j] = s0 >= 0 ? X[(size_t(s0) * DL_CHUNK + kk) * 2 + 1] : make_float2(0.f, 0.f);
    }
#pragma unroll 4
    for (int b = 0; b < nb; ++b) {
#pragma unroll
      for (int j = DL_NPT - 1; j > 0; --j) wl[j] = wl[j - 1], wr[j] = wr[j - 1];
      const int ws = b - p0 + P;              // window index b - p0, stored from -P
      wl[0] = X[(size_t(ws) * DL_CHUNK + kk) * 2];
      wr[0] = X[(size_t(ws) * DL_CHUNK + kk) * 2 + 1];
      const float2 yl = Y[(size_t(b) * DL_CHUNK + kk) * 2], yr = Y[(size_t(b) * DL_CHUNK + kk) * 2 + 1];
#pragma unroll
      for (int j = 0; j < DL_NPT; ++j) {
        al[j].x += wl[j].x * yl.x + wl[j].y * yl.y;
        al[j].y += wl[j].y * yl.x - wl[j].x * yl.y;
        ar[j].x += wr[j].x * yr.x + wr[j].y * yr.y;
        ar[j].y += wr[j].y * yr.x - wr[j].x * yr.y;
      }
    }
    // R_l + i R_r at k, conj(R_l) + i conj(R_r) at M - k
    const int k = k0 + kk;
    if (k <= DL_M / 2) {
#pragma unroll
      for (int j = 0; j < DL_NPT; ++j) {
        if (p0 + j >= P) break;
        float2* R = c.dl_R + (size_t(e.y) + p0 + j) * DL_M;
        R[k] = make_float2(al[j].x - ar[j].y, al[j].y + ar[j].x);
        if (k > 0 && k < DL_M / 2) R[DL_M - k] = make_float2(al[j].x + ar[j].y, ar[j].x - al[j].y);
      }
    }
  }
}

// r_x[n] for n = -B + p B + nu, nu in [0, B): r_p[nu] = IDFT(R_p)[B - nu].  The spectrum
// goes straight into the transform's registers (thread t: bins t + T m) and the lags come
// straight out of them.
__global__ void __launch_bounds__(DL_M / 16) k_delay_lags(DevCtx c, int item0, int n_items) {
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  constexpr int T = DL_M / 16;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, p = w.y;
    const int4_ e = c.ext[v];
    const float2* R = c.dl_R + (size_t(e.y) + p) * DL_M;
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const float2 z = R[threadIdx.x + T * m];
      x[m] = make_float2(z.x, -z.y);
    }
    __syncthreads();   // readers of buf (the previous item's last pass) are done
    fft::forward_regs_1buf<DL_M>(x, buf, c.ptw, threadIdx.x);
    const int nlag = c.dl_P * DL_B;
    float* rl = c.dl_r + size_t(e.z) * 2 * nlag;
    const float inv = 1.f / float(DL_M);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int k = threadIdx.x + T * m;   // conj(result) / M at bin k = (l, r) of lag B - k
      if (k >= 1 && k <= DL_B) {
        const int nu = DL_B - k;
        rl[p * DL_B + nu] = x[m].x * inv;
        rl[nlag + p * DL_B + nu] = -x[m].y * inv;
      }
    }
  }
}

struct cplx {
  float x, y;
};
__device__ __forceinline__ cplx cm(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cdv(cplx a, cplx b) {
  const float d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// Gradients of one (node, channel, tap): FIR log-magnitudes and the surrogate z.
// The phase of q = z w^n is taken relative to the tap's integer delay bin d0 (the n with
// q closest to 1): arg q / pi = delta + 2 m / N_d with m = (n - d0) mod N_d in
// (-N_d/2, N_d/2] exact in integers and delta = arg z / pi + 2 d0 / N_d (|delta| <= 1/N_d)
// formed once in double, so the lag next to the pole (m = 0, the Taylor branch) keeps
// its full precision in FP32.  Each thread runs over RUN consecutive lags with a
// register window of r for the 39-tap correlation g.
struct DlSurrogate {
  cplx zN, bz, zinv;
  float dlt, tx, npi, rf, one_m_rho;
  float rot_c, rot_s;   // cos, sin of pi / N_d: the half-angle step from one lag to the next
  int d0;
};
constexpr int DL_FAR = 80;   // lags from the pole beyond which the phasor is rotated, not recomputed

__global__ void __launch_bounds__(256) k_delay_grad(DevCtx c, int item0, int n_items) {
  __shared__ DlSurrogate sc;
  __shared__ float csh[DL_SH];   // cs placed at offset o (the window's misalignment)
  __shared__ float cos39[DL_FIR], hann39[DL_FIR];
  __shared__ float red[4 * 32];
  constexpr int H = (DL_FIR - 1) / 2, K = DL_K, RUN = 8;
  const int ntap = c.dl_taps, Nd = c.dl_nd, nlag = c.dl_P * DL_B;
  dl_tables(cos39, hann39);
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, x = w.y / ntap, m = w.y % ntap;
    const NodeDev nd = c.nodes[v];
    const int4_ e = c.ext[v];
    const float* aux = c.dl_aux + size_t(e.z) * 2 * ntap * (DL_FIR + 1) + (x * ntap + m) * (DL_FIR + 1);
    const float* r = c.dl_r + size_t(e.z) * 2 * nlag + x * nlag + DL_B;  // r[n] at r + n
    const float* rs = r + m * c.dl_slot;                                 // the tap's slot: rs[n] = r[m S + n]
    const float* q = c.params + size_t(nd.prow) * c.pcols + (x * ntap + m) * DL_ROW;
    float* out = c.dparams + size_t(nd.grow) * c.pcols + (x * ntap + m) * DL_ROW;
    const int d = int(aux[DL_FIR]);
    // a run's window rs[n0 - H ..] starts o floats past a 16-byte boundary, the same o for
    // every run (n0 is a multiple of RUN): it is read from that boundary as float4 and the
    // taps are shifted by o instead
    const int o = int((reinterpret_cast<uintptr_t>(rs - H) >> 2) & 3);
    const float* ra = rs - H - o;
    __syncthreads();
    if (threadIdx.x < DL_SH) {
      const int j = int(threadIdx.x) - o;
      csh[threadIdx.x] = j >= 0 && j < DL_FIR ? aux[j] : 0.f;
    }
    if (threadIdx.x == 0) {
      // the tap's surrogate constants, once per item in double (B300's FP64 rate is a
      // small fraction of FP32: every thread forming them was most of this kernel's time)
      const double zr = q[0], zi = q[1];
      const double rho = sqrt(zr * zr + zi * zi), th = atan2(zi, zr);
      const double lr = log(rho);
      const double rN = exp(Nd * lr);
      double sN, cN;
      sincos(0.5 * Nd * th, &sN, &cN);
      const double c1 = -2.0 * sN * sN;                   // cos(N th) - 1
      const double s1 = 2.0 * sN * cN;                    // sin(N th)
      const long long d0r = llrint(double(Nd) * (-th) / (2.0 * M_PI));   // |arg z / pi + 2 d0r / N_d| <= 1/N_d
      long long d0l = d0r % Nd;
      if (d0l < 0) d0l += Nd;
      sc.zN = {float(rN * (1.0 + c1)), float(rN * s1)};
      sc.bz = {float(rN * c1 + (rN - 1.0)), float(rN * s1)};   // z^N - 1
      sc.zinv = {float(zr / (rho * rho) / Nd), float(-zi / (rho * rho) / Nd)};
      sc.dlt = float(th / M_PI + 2.0 * double(d0r) / Nd);
      sc.d0 = int(d0l);
      sc.tx = float(Nd * lr);
      sc.npi = float(Nd * M_PI);
      sc.rf = float(rho);
      sc.one_m_rho = float(1.0 - rho);
      sc.rot_c = float(cos(M_PI / Nd));
      sc.rot_s = float(sin(M_PI / Nd));
    }
    __syncthreads();
    // FIR taps: dL/dc[j] = r[d + j]; chain through the window, cosine sum and exp
    if (threadIdx.x < K) {
      const int k = threadIdx.x;
      float acc = 0.f;
      for (int j = 0; j < DL_FIR; ++j) {
        const int an = j < H ? H - j : j - H;
        acc += hann39[j] * r[d + j - H] * cos39[(k * an) % DL_FIR];
      }
      out[2 + k] = expf(q[2 + k]) * acc * (k == 0 ? 1.f : 2.f) / float(DL_FIR);
    }
    // surrogate z: Q = sum_n g[n] phi[n] with phi[n] = F(q_n) / (N z) and, away from the
    // pole, F = -(t1 / a + (z^N - 1) / a^2), a = 1 - q_n, t1 = 1 + (N - 1) z^N: the thread
    // sums g / a and g / a^2 (and g F where the Taylor branch gives F), the tap's constants
    // multiply the CTA's sums once
    const cplx zN = sc.zN, bz = sc.bz, zinv = sc.zinv;
    const float dlt = sc.dlt, tx = sc.tx, npi = sc.npi, rf = sc.rf, one_m_rho = sc.one_m_rho;
    const int d0 = sc.d0;
    const float two_n = 2.f / float(Nd);
    float s1x = 0.f, s1y = 0.f, s2x = 0.f, s2y = 0.f, ftx = 0.f, fty = 0.f;
    for (int n0 = threadIdx.x * RUN; n0 < Nd; n0 += blockDim.x * RUN) {
      // win[i] = rs[n0 - H - o + i]; the lags' range [-H, N_d + H) plus the read-ahead
      // to the next 16 bytes lies inside the partitions' lags (values past N_d + H meet
      // only lags >= N_d, which are dropped)
      constexpr int WL = (RUN + DL_SH - 1 + 3) & ~3;
      float win[WL];
#pragma unroll
      for (int k = 0; k < WL / 4; ++k) {
        const float4 q4 = ldg4(ra + n0 + 4 * k);
        win[4 * k] = q4.x, win[4 * k + 1] = q4.y, win[4 * k + 2] = q4.z, win[4 * k + 3] = q4.w;
      }
      // g[n0 + u] = sum_jj c[jj] r[n0 + u + jj - H]: RUN independent chains
      float gv[RUN];
#pragma unroll
      for (int u = 0; u < RUN; ++u) gv[u] = 0.f;
#pragma unroll
      for (int jp = 0; jp < DL_SH; ++jp) {
        const float cj = csh[jp];
#pragma unroll
        for (int u = 0; u < RUN; ++u) gv[u] += cj * win[u + jp];
      }
      // Runs of lags away from the pole (|m| >= DL_FAR for every lag of the run) take the
      // half-angle phasor of their first lag from sincospif and rotate it by pi / N_d per lag
      // (the wrap of m at N_d/2 flips the phasor's sign, which a = 1 - q does not see);
      // runs near the pole evaluate every lag exactly, with the Taylor branch next to it.
      int mm0 = n0 - d0;
      if (mm0 < 0) mm0 += Nd;
      if (2 * mm0 > Nd) mm0 -= Nd;
      const bool far = mm0 >= DL_FAR || mm0 <= -(DL_FAR + RUN);
      float sh0 = 0.f, ch0 = 1.f;
      if (far) sincospif(0.5f * (dlt + float(mm0) * two_n), &sh0, &ch0);
#pragma unroll
      for (int u = 0; u < RUN; ++u) {
        const int n = n0 + u;
        if (n < Nd) {
          const float g = gv[u];
          float sh = sh0, chh = ch0;
          bool taylor = false;
          if (!far) {
            int mm = n - d0;
            if (mm < 0) mm += Nd;
            if (2 * mm > Nd) mm -= Nd;
            const float phf = dlt + float(mm) * two_n;   // arg q / pi
            const float ty = npi * phf;                   // t = N ln q = tx + i ty
            taylor = tx * tx + ty * ty < 0.25f;
            if (taylor) {
              // F = N^2 sum_j e_j t^j with e_j = (sum_k k^(j+1)) / (N^(j+2) j!)
              cplx t = {tx, ty}, tp = {1.f, 0.f}, F = {0.f, 0.f};
#pragma unroll
              for (int j = 0; j < 9; ++j) {
                F.x += c.dl_taylor[j] * tp.x;
                F.y += c.dl_taylor[j] * tp.y;
                tp = cm(tp, t);
              }
              const float n2 = float(Nd) * float(Nd);
              ftx += g * (F.x * n2);
              fty += g * (F.y * n2);
            } else {
              sincospif(0.5f * phf, &sh, &chh);
            }
          }
          if (!taylor) {
            // a = 1 - q = (1 - rho) + 2 rho sin^2(ph/2) - i rho sin(ph); b = 1 / a
            const float ax = one_m_rho + 2.f * rf * sh * sh, ay = -rf * 2.f * sh * chh;
            const float ia = __frcp_rn(ax * ax + ay * ay);
            const float bx = ax * ia, by = -ay * ia;
            const float gx = g * bx, gy = g * by;
            s1x += gx;
            s1y += gy;
            s2x += gx * bx - gy * by;   // g Re(b^2)
            s2y += gx * by + gy * bx;   // g Im(b^2)
          }
          if (far) {   // the next lag's half-angle phasor
            const float s2 = sh * sc.rot_c + ch0 * sc.rot_s;
            ch0 = ch0 * sc.rot_c - sh * sc.rot_s;
            sh0 = s2;
          }
        }
      }
    }
    float v1[4] = {s1x, s1y, s2x, s2y};
    block_sum<4>(v1, red);
    float v2[2] = {ftx, fty};
    block_sum<2>(v2, red);
    if (threadIdx.x == 0) {
      // sum g F = T - t1 S1 - (z^N - 1) S2; Q = (sum g F) / (N z)
      const double t1x = 1.0 + double(Nd - 1) * zN.x, t1y = double(Nd - 1) * zN.y;
      const double S1x = v1[0], S1y = v1[1], S2x = v1[2], S2y = v1[3];
      const double Fx = double(v2[0]) - (t1x * S1x - t1y * S1y) - (double(bz.x) * S2x - double(bz.y) * S2y);
      const double Fy = double(v2[1]) - (t1x * S1y + t1y * S1x) - (double(bz.x) * S2y + double(bz.y) * S2x);
      out[0] = float(Fx * zinv.x - Fy * zinv.y);
      out[1] = float(-(Fx * zinv.y + Fy * zinv.x));
    }
  }
}

int launch_delay(int what, const DevCtx& c, int a, int b, cudaStream_t s) {
  static bool init = false;
  const size_t sm_fft = sizeof(float2) * fft::Padded<DL_M>::size;
  // the accumulation stages nb + P u windows and nb ybar blocks of DL_CHUNK bins: sized by
  // the plan's longest delay signal, so that short signals keep several CTAs per SM
  const size_t sm_acc = sizeof(float2) * 2 * DL_CHUNK * size_t(2 * std::max(c.dl_nbmax, 1) + c.dl_P);
  const int acc_per_sm = std::max(1, std::min(4, int((228 * 1024) / (sm_acc + 1024))));
  // resident CTAs per SM of the strided item loops (one wave each)
  static int res_fir0 = 1, res_fir1 = 1, res_spec = 1, res_lags = 1, res_grad = 1;
  if (!init) {
    const size_t sm_acc_max = sizeof(float2) * 2 * DL_CHUNK * size_t(2 * DL_MAX_BLOCKS + DL_PMAX);
    cudaFuncSetAttribute(k_delay_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    cudaFuncSetAttribute(k_delay_lags, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_fft));
    cudaFuncSetAttribute(k_delay_acc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_acc_max));
    cudaFuncSetAttribute(k_delay_acc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_acc_max));
    res_fir0 = resident_per_sm(reinterpret_cast<const void*>(k_delay_fir<false>), DL_FT, 0);
    res_fir1 = resident_per_sm(reinterpret_cast<const void*>(k_delay_fir<true>), DL_FT, 0);
    res_spec = resident_per_sm(reinterpret_cast<const void*>(k_delay_spec), DL_M / 16, sm_fft);
    res_lags = resident_per_sm(reinterpret_cast<const void*>(k_delay_lags), DL_M / 16, sm_fft);
    res_grad = resident_per_sm(reinterpret_cast<const void*>(k_delay_grad), 256, 0);
    init = true;
  }
  if (what < 0) return 0;
  switch (what) {
    case 0:
      if (b <= a) return 0;
      k_delay_design<<<b - a, 128, 0, s>>>(c, a);
      return 1;
    case 1: if (b > 0) k_delay_fir<false><<<grid_size(b, res_fir0), DL_FT, 0, s>>>(c, a, b); return b > 0;
    case 2: if (b > 0) k_delay_fir<true><<<grid_size(b, res_fir1), DL_FT, 0, s>>>(c, a, b); return b > 0;
    case 3: if (b > 0) k_delay_spec<<<grid_size(b, res_spec), DL_M / 16, sm_fft, s>>>(c, a, b); return b > 0;
    case 4:   // one thread per bin and group of lag partitions
      if (b > 0) {
        const int g4 = (c.dl_P + 3) / 4, g2 = (c.dl_P + 1) / 2;
        if (4 * g4 <= 2 * g2)
          k_delay_acc<4><<<grid_size(b, acc_per_sm), DL_CHUNK * g4, sm_acc, s>>>(c, a, b);
        else
          k_delay_acc<2><<<grid_size(b, acc_per_sm), DL_CHUNK * g2, sm_acc, s>>>(c, a, b);
      }
      return b > 0;
    case 5: if (b > 0) k_delay_lags<<<grid_size(b, res_lags), DL_M / 16, sm_fft, s>>>(c, a, b); return b > 0;
    case 6: if (b > 0) k_delay_grad<<<grid_size(b, res_grad), 256, 0, s>>>(c, a, b); return b > 0;
  }
  return 0;
}

}  // namespace grafx
