// Multi-resolution STFT magnitude loss and its gradient, on the shared-memory FFT.
//
// A work item is up to 8 consecutive frames of one output row at one resolution M
// (hop M/4, periodic Hann, no padding).  4096/M frames are transformed at once by
// groups of M/16 threads; left and right are packed as l + i r and separated from
// the packed spectrum by conjugate symmetry.  The forward pass writes per-item
// partial sums (sum (|Y|-|T|)^2, sum |T|^2, sum |ln(|Y|+e) - ln(|T|+e)| per channel);
// a single-CTA reduce turns them into the loss and keeps the norms for the
// backward pass.  The backward pass recomputes the spectra, forms dL/dY per bin,
// builds the Hermitian spectra of both channels, packs them and inverts with one
// FFT, windows the frame and writes it to a frame buffer; an overlap-add kernel
// then sums the (at most 4 per resolution) frames covering each sample, so no
// atomics are used anywhere.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {

constexpr float MAG_EPS = 1e-7f;
__host__ __device__ constexpr int res_m(int q) { return 512 << q; }

struct LossArgs {
  const LossRow* rows;
  const int2_* items;      // items of this resolution
  const float* y;          // out buffer
  const float* tgt;        // target buffer
  float4* part;            // [group] x 2 float4: (s1_l, s2_l, s3_l, 0), (s1_r, s2_r, s3_r, 0)
  float4* stats;           // [row][res] x 2: (nd_l, nt_l, F*(M/2+1), 0), (nd_r, nt_r, ., 0)
  float* frames;           // frame buffer
  const float2_* tw;
  int q;                   // resolution index
  int n_items;
};

// periodic Hann from the twiddle table: 0.5 - 0.5 cos(2 pi n / M)
template <int M>
__device__ __forceinline__ float hann(const float2_* tw, int n) {
  return 0.5f - 0.5f * tw[n * (TWIDDLE_N / M)].x;
}

template <int M>
__device__ __forceinline__ void load_frame(const LossArgs& a, const LossRow& r, const float* base, int f, int gtid,
                                           float2* buf, bool active) {
  constexpr int T = M / 16;
  if (!active) return;
  const float* row = base + r.off;
  const int t0 = f * (M / 4);
  for (int n = gtid; n < M; n += T) {
    float w = hann<M>(a.tw, n);
    buf[fft::pad(n)] = make_float2(w * row[t0 + n], w * row[r.pitch + t0 + n]);
  }
}

// Split packed spectrum Z of l + i r at bin k into the two channel spectra.
__device__ __forceinline__ void split(float2 z, float2 zm, float2* L, float2* R) {
  // L = (Z[k] + conj(Z[M-k]))/2 ; R = (Z[k] - conj(Z[M-k]))/(2i)
  *L = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
  float dx = z.x - zm.x, dy = z.y + zm.y;   // Z - conj(Zm)
  *R = make_float2(0.5f * dy, -0.5f * dx);
}

template <int M>
__global__ void __launch_bounds__(256) k_loss_fwd(LossArgs a) {
  constexpr int T = M / 16, G = 256 / T;
  extern __shared__ float2 smem2[];
  float2* by = smem2;                                // G frames of y
  float2* bt = smem2 + G * fft::Padded<M>::size;     // G frames of target
  __shared__ float red[6 * 32 + 8];
  const int g = threadIdx.x / T, gtid = threadIdx.x % T;
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2_ item = a.items[it];
    const LossRow r = a.rows[item.x];
    const int F = r.n_frames[a.q];
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int f0 = item.y; f0 < min(item.y + LOSS_FRAMES_PER_ITEM, F); f0 += G) {
      const int f = f0 + g;
      const bool act = f < min(item.y + LOSS_FRAMES_PER_ITEM, F);
      float2* fy = by + g * fft::Padded<M>::size;
      float2* ft = bt + g * fft::Padded<M>::size;
      load_frame<M>(a, r, a.y, f, gtid, fy, act);
      load_frame<M>(a, r, a.tgt, f, gtid, ft, act);
      __syncthreads();
      fft::forward<M>(fy, a.tw, gtid, true);
      fft::forward<M>(ft, a.tw, gtid, true);
      if (act) {
        for (int k = gtid; k <= M / 2; k += T) {
          int km = (M - k) & (M - 1);
          float2 yl, yr, tl, tr;
          split(fy[fft::pad(k)], fy[fft::pad(km)], &yl, &yr);
          split(ft[fft::pad(k)], ft[fft::pad(km)], &tl, &tr);
          float al = sqrtf(yl.x * yl.x + yl.y * yl.y), ar = sqrtf(yr.x * yr.x + yr.y * yr.y);
          float bl = sqrtf(tl.x * tl.x + tl.y * tl.y), br = sqrtf(tr.x * tr.x + tr.y * tr.y);
          s[0] += (al - bl) * (al - bl);
          s[1] += bl * bl;
          s[2] += fabsf(logf(al + MAG_EPS) - logf(bl + MAG_EPS));
          s[3] += (ar - br) * (ar - br);
          s[4] += br * br;
          s[5] += fabsf(logf(ar + MAG_EPS) - logf(br + MAG_EPS));
        }
      }
      __syncthreads();
    }
    float lo[3] = {s[0], s[1], s[2]}, hi[3] = {s[3], s[4], s[5]};
    block_sum<3>(lo, red);
    block_sum<3>(hi, red + 3 * 32);
    if (threadIdx.x == 0) {
      int gi = r.group_off[a.q] + item.y / LOSS_FRAMES_PER_ITEM;
      a.part[2 * gi] = make_float4(lo[0], lo[1], lo[2], 0.f);
      a.part[2 * gi + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
    __syncthreads();
  }
}

// One CTA: per row and resolution, sum the groups in order; loss = sum over rows of
// the mean over (resolution, channel) of sc + mag.
__global__ void k_loss_reduce(const LossRow* rows, int n_rows, const float4* part, float4* stats, float* loss) {
  __shared__ float rl[1024];
  float acc = 0.f;
  for (int j = threadIdx.x; j < n_rows; j += blockDim.x) {
    const LossRow r = rows[j];
    float row_loss = 0.f;
    for (int q = 0; q < N_RES; ++q) {
      float sl[3] = {0.f, 0.f, 0.f}, sr[3] = {0.f, 0.f, 0.f};
      for (int gi = 0; gi < r.n_groups[q]; ++gi) {
        float4 a = part[2 * (r.group_off[q] + gi)], b = part[2 * (r.group_off[q] + gi) + 1];
        sl[0] += a.x; sl[1] += a.y; sl[2] += a.z;
        sr[0] += b.x; sr[1] += b.y; sr[2] += b.z;
      }
      const float nb = float(r.n_frames[q]) * float(res_m(q) / 2 + 1);
      float ndl = sqrtf(sl[0]), ntl = sqrtf(sl[1]), ndr = sqrtf(sr[0]), ntr = sqrtf(sr[1]);
      stats[2 * (j * N_RES + q)] = make_float4(ndl, ntl, nb, 0.f);
      stats[2 * (j * N_RES + q) + 1] = make_float4(ndr, ntr, nb, 0.f);
      row_loss += ndl / ntl + sl[2] / nb + ndr / ntr + sr[2] / nb;
    }
    acc += row_loss / float(2 * N_RES);
  }
  rl[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < int(blockDim.x); ++i) t += rl[i];
    *loss = t;
  }
}

template <int M>
__global__ void __launch_bounds__(256) k_loss_bwd(LossArgs a) {
  constexpr int T = M / 16, G = 256 / T;
  constexpr int NB = (M / 2 + 1 + T - 1) / T;
  extern __shared__ float2 smem2[];
  float2* by = smem2;
  float2* bt = smem2 + G * fft::Padded<M>::size;
  const int g = threadIdx.x / T, gtid = threadIdx.x % T;
  const float w_res = 1.f / float(2 * N_RES);
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2_ item = a.items[it];
    const LossRow r = a.rows[item.x];
    const int F = r.n_frames[a.q];
    const float4 stl = a.stats[2 * (item.x * N_RES + a.q)], str = a.stats[2 * (item.x * N_RES + a.q) + 1];
    for (int f0 = item.y; f0 < min(item.y + LOSS_FRAMES_PER_ITEM, F); f0 += G) {
      const int f = f0 + g;
      const bool act = f < min(item.y + LOSS_FRAMES_PER_ITEM, F);
      float2* fy = by + g * fft::Padded<M>::size;
      float2* ft = bt + g * fft::Padded<M>::size;
      load_frame<M>(a, r, a.y, f, gtid, fy, act);
      load_frame<M>(a, r, a.tgt, f, gtid, ft, act);
      __syncthreads();
      fft::forward<M>(fy, a.tw, gtid, true);
      fft::forward<M>(ft, a.tw, gtid, true);
      // dL/dY per bin, as the Hermitian spectra of both channels packed l + i r
      float2 wk[NB], wm[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        int k = gtid + i * T;
        wk[i] = wm[i] = make_float2(0.f, 0.f);
        if (act && k <= M / 2) {
          int km = (M - k) & (M - 1);
          float2 yv[2], tv[2];
          split(fy[fft::pad(k)], fy[fft::pad(km)], &yv[0], &yv[1]);
          split(ft[fft::pad(k)], ft[fft::pad(km)], &tv[0], &tv[1]);
          float2 gh[2];
#pragma unroll
          for (int ch = 0; ch < 2; ++ch) {
            const float4 st = ch ? str : stl;
            float A = sqrtf(yv[ch].x * yv[ch].x + yv[ch].y * yv[ch].y);
            float B = sqrtf(tv[ch].x * tv[ch].x + tv[ch].y * tv[ch].y);
            float dA = 0.f;
            if (st.x > 0.f) dA += (A - B) / (st.x * st.y);
            float dl = logf(A + MAG_EPS) - logf(B + MAG_EPS);
            float sg = dl > 0.f ? 1.f : (dl < 0.f ? -1.f : 0.f);
            dA += sg / ((A + MAG_EPS) * st.z);
            dA *= w_res;
            float2 G2 = A > 0.f ? make_float2(dA * yv[ch].x / A, dA * yv[ch].y / A) : make_float2(0.f, 0.f);
            // Hermitian fill: DC and Nyquist keep their real part, others are halved
            if (k == 0 || k == M / 2) G2 = make_float2(G2.x, 0.f);
            else G2 = make_float2(0.5f * G2.x, 0.5f * G2.y);
            gh[ch] = G2;
          }
          // W[k] = Gl[k] + i Gr[k]; W[M-k] = conj(Gl[k]) + i conj(Gr[k]); stored conjugated
          float2 Wk = make_float2(gh[0].x - gh[1].y, gh[0].y + gh[1].x);
          float2 Wm = make_float2(gh[0].x + gh[1].y, -gh[0].y + gh[1].x);
          wk[i] = make_float2(Wk.x, -Wk.y);
          wm[i] = make_float2(Wm.x, -Wm.y);
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          int k = gtid + i * T;
          if (k <= M / 2) {
            fy[fft::pad(k)] = wk[i];
            if (k > 0 && k < M / 2) fy[fft::pad(M - k)] = wm[i];
          }
        }
      }
      __syncthreads();
      fft::forward<M>(fy, a.tw, gtid, true);
      if (act) {
        float* fr = a.frames + r.frame_off[a.q] + int64_t(f) * 2 * M;
        for (int n = gtid; n < M; n += T) {
          float2 z = fy[fft::pad(n)];
          float w = hann<M>(a.tw, n);
          fr[n] = w * z.x;          // conj of the result: real part is l
          fr[M + n] = -w * z.y;     // minus imaginary part is r
        }
      }
      __syncthreads();
    }
  }
}

// d_out[ch][t] = sum over resolutions and covering frames of the windowed frame adjoint.
__global__ void k_loss_ola(const LossRow* rows, const float* frames, float* d_out) {
  const int j = blockIdx.y;
  const LossRow r = rows[j];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= r.pitch) return;
  float sl = 0.f, sr = 0.f;
  if (t < r.len) {
#pragma unroll
    for (int q = 0; q < N_RES; ++q) {
      const int M = res_m(q), hop = M / 4;
      const int F = r.n_frames[q];
      int fhi = min(F - 1, t / hop);
      int flo = t - M + 1 <= 0 ? 0 : (t - M + 1 + hop - 1) / hop;
      for (int f = flo; f <= fhi; ++f) {
        const float* fr = frames + r.frame_off[q] + int64_t(f) * 2 * M;
        int n = t - f * hop;
        sl += fr[n];
        sr += fr[M + n];
      }
    }
  }
  d_out[r.off + t] = sl;
  d_out[r.off + r.pitch + t] = sr;
}

template <int M>
static void loss_launch(bool bwd, LossArgs a, cudaStream_t s) {
  constexpr int T = M / 16, G = 256 / T;
  const size_t sm = 2 * G * fft::Padded<M>::size * sizeof(float2);
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_loss_fwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    cudaFuncSetAttribute(k_loss_bwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    init = true;
  }
  int g = grid_size(a.n_items, 3);
  if (bwd) k_loss_bwd<M><<<g, 256, sm, s>>>(a);
  else k_loss_fwd<M><<<g, 256, sm, s>>>(a);
}

int launch_loss(int what, const LossLaunch& L, cudaStream_t s) {
  int n = 0;
  if (what == 0 || what == 2) {
    for (int q = 0; q < N_RES; ++q) {
      if (L.n_items[q] <= 0) continue;
      LossArgs a{L.rows, L.items[q], L.y, L.tgt, L.part, L.stats, L.frames, L.tw, q, L.n_items[q]};
      if (q == 0) loss_launch<512>(what == 2, a, s);
      if (q == 1) loss_launch<1024>(what == 2, a, s);
      if (q == 2) loss_launch<2048>(what == 2, a, s);
      ++n;
    }
    if (what == 0) {
      k_loss_reduce<<<1, 256, 0, s>>>(L.rows, L.n_rows, L.part, L.stats, L.loss);
      ++n;
    } else {
      dim3 grid((L.max_pitch + 255) / 256, L.n_rows);
      k_loss_ola<<<grid, 256, 0, s>>>(L.rows, L.frames, L.d_out);
      ++n;
    }
  }
  return n;
}

}  // namespace grafx
