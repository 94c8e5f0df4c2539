// Multi-resolution STFT magnitude loss and its gradient, on the shared-memory FFT.
//
// A work item is up to 8 consecutive frames of one output row at one resolution M
// (hop M/4, periodic Hann, no padding).  4096/M frames are transformed at once by
// groups of M/16 threads; left and right are packed as l + i r and separated from
// the packed spectrum by conjugate symmetry.  The forward pass writes per-item
// partial sums (sum (|Y|-|T|)^2, sum |T|^2, sum |ln(|Y|+e) - ln(|T|+e)| per channel)
// and keeps every bin's Y_l, Y_r and |T_l|, |T_r| in a spectrum cache; a per-row
// reduce turns the partials into the loss and keeps the norms for the backward pass.
// The backward pass reads the cached spectra (no transforms of y or the target),
// forms dL/dY per bin, builds the Hermitian spectra of both channels, packs them and
// inverts with one FFT, windows the frame and writes it to a frame buffer; an
// overlap-add kernel then sums the (at most 4 per resolution) frames covering each
// sample, so no atomics are used anywhere.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace grafx {

constexpr float MAG_EPS = 1e-7f;
__host__ __device__ constexpr int res_m(int q) { return 512 << q; }

struct LossArgs {
  const LossRow* rows;
  const int4_* items;      // (row, resolution, first frame, group) for every resolution
  const float* y;          // out buffer
  const float* tgt;        // target buffer
  float4* part;            // [group] x 2 float4: (s1_l, s2_l, s3_l, 0), (s1_r, s2_r, s3_r, 0)
  float4* stats;           // [row][res] x 2: (nd_l, nt_l, F*(M/2+1), 0), (nd_r, nt_r, ., 0)
  float* frames;           // frame buffer
  float2* spec;            // spectrum cache: per (row, resolution) planes Y_l, Y_r, (|T_l|, |T_r|)
  const float2_* tw;
  const float2_* ptw;
  int n_items;
};

// periodic Hann from the twiddle table: 0.5 - 0.5 cos(2 pi n / M)
template <int M>
__device__ __forceinline__ float hann(const float2_* tw, int n) {
  return 0.5f - 0.5f * tw[n * (TWIDDLE_N / M)].x;
}

// Split packed spectrum Z of l + i r at bin k into the two channel spectra.
__device__ __forceinline__ void split(float2 z, float2 zm, float2* L, float2* R) {
  // L = (Z[k] + conj(Z[M-k]))/2 ; R = (Z[k] - conj(Z[M-k]))/(2i)
  *L = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
  float dx = z.x - zm.x, dy = z.y + zm.y;   // Z - conj(Zm)
  *R = make_float2(0.5f * dy, -0.5f * dx);
}

// One item: the 4096/M frames f0.. of one row at resolution M, y and target together.
template <int M>
__device__ __forceinline__ void loss_item_fwd(const LossArgs& a, const int4_ item, float2* smem) {
  constexpr int T = M / 16, G = 256 / T;
  float2* by = smem;
  float2* bt = smem + G * fft::Padded<M>::size;
  __shared__ float red[6 * 32];
  const int g = threadIdx.x / T, gtid = threadIdx.x % T;
  const LossRow r = a.rows[item.x];
  constexpr int q = M == 512 ? 0 : M == 1024 ? 1 : 2;  // == item.y (dispatch)
  const int F = r.n_frames[q];
  const int f = item.z + g;
  const bool act = f < F;
  float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float2* fy = by + g * fft::Padded<M>::size;
  float2* ft = bt + g * fft::Padded<M>::size;
  // both windowed frames straight into the transforms' registers (thread gtid: samples
  // gtid + T m), all loads issued together
  float2 xy[16], xt[16];
  {
    const float* ry = a.y + r.off;
    const float* rt = a.tgt + r.off;
    const int t0 = f * (M / 4);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = gtid + T * m;
      const float w = hann<M>(a.tw, n);
      xy[m] = act ? make_float2(w * ry[t0 + n], w * ry[r.pitch + t0 + n]) : make_float2(0.f, 0.f);
      xt[m] = act ? make_float2(w * rt[t0 + n], w * rt[r.pitch + t0 + n]) : make_float2(0.f, 0.f);
    }
  }
  fft::forward_regs_1buf<M>(xy, fy, a.ptw, gtid);
  fft::forward_regs_1buf<M>(xt, ft, a.ptw, gtid);
  __syncthreads();   // every thread's last pass has read the buffers
#pragma unroll
  for (int m = 0; m < 16; ++m) {   // the spectra in natural order for the bin pairs (k, M - k)
    fy[fft::pad(gtid + T * m)] = xy[m];
    ft[fft::pad(gtid + T * m)] = xt[m];
  }
  __syncthreads();
  if (act) {
    constexpr int nb = M / 2 + 1;
    float2* sp = a.spec + r.spec_off[q] + int64_t(f) * nb;
    const int64_t plane = int64_t(F) * nb;
    for (int k = gtid; k <= M / 2; k += T) {
      int km = (M - k) & (M - 1);
      float2 yl, yr, tl, tr;
      split(fy[fft::pad(k)], fy[fft::pad(km)], &yl, &yr);
      split(ft[fft::pad(k)], ft[fft::pad(km)], &tl, &tr);
      float al = sqrtf(yl.x * yl.x + yl.y * yl.y), ar = sqrtf(yr.x * yr.x + yr.y * yr.y);
      float bl = sqrtf(tl.x * tl.x + tl.y * tl.y), br = sqrtf(tr.x * tr.x + tr.y * tr.y);
      sp[k] = yl;
      sp[plane + k] = yr;
      sp[2 * plane + k] = make_float2(bl, br);
      s[0] += (al - bl) * (al - bl);
      s[1] += bl * bl;
      s[2] += fabsf(logf(al + MAG_EPS) - logf(bl + MAG_EPS));
      s[3] += (ar - br) * (ar - br);
      s[4] += br * br;
      s[5] += fabsf(logf(ar + MAG_EPS) - logf(br + MAG_EPS));
    }
  }
  float lo[3] = {s[0], s[1], s[2]}, hi[3] = {s[3], s[4], s[5]};
  block_sum<3>(lo, red);
  block_sum<3>(hi, red + 3 * 32);
  if (threadIdx.x == 0) {
    a.part[2 * item.w] = make_float4(lo[0], lo[1], lo[2], 0.f);
    a.part[2 * item.w + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256, 2) k_loss_fwd(LossArgs a) {
  extern __shared__ float2 smem2[];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int4_ item = a.items[it];
    __syncthreads();   // the previous item's readers of the buffers are done
    switch (item.y) {
      case 0: loss_item_fwd<512>(a, item, smem2); break;
      case 1: loss_item_fwd<1024>(a, item, smem2); break;
      default: loss_item_fwd<2048>(a, item, smem2); break;
    }
  }
}

// One CTA per row: sum its groups per resolution, keep the norms for the backward
// pass, and write the row loss (mean over resolution and channel of sc + mag).
__global__ void __launch_bounds__(256) k_loss_rows(const LossRow* rows, const float4* part, float4* stats,
                                                   float* row_loss) {
  __shared__ float red[6 * 32];
  const int j = blockIdx.x;
  const LossRow r = rows[j];
  float total = 0.f;
  for (int q = 0; q < N_RES; ++q) {
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    for (int gi = threadIdx.x; gi < r.n_groups[q]; gi += blockDim.x) {
      float4 a = part[2 * (r.group_off[q] + gi)], b = part[2 * (r.group_off[q] + gi) + 1];
      lo[0] += a.x; lo[1] += a.y; lo[2] += a.z;
      hi[0] += b.x; hi[1] += b.y; hi[2] += b.z;
    }
    block_sum<3>(lo, red);
    block_sum<3>(hi, red + 3 * 32);
    if (threadIdx.x == 0) {
      const float nb = float(r.n_frames[q]) * float(res_m(q) / 2 + 1);
      float ndl = sqrtf(lo[0]), ntl = sqrtf(lo[1]), ndr = sqrtf(hi[0]), ntr = sqrtf(hi[1]);
      stats[2 * (j * N_RES + q)] = make_float4(ndl, ntl, nb, 0.f);
      stats[2 * (j * N_RES + q) + 1] = make_float4(ndr, ntr, nb, 0.f);
      total += ndl / ntl + lo[2] / nb + ndr / ntr + hi[2] / nb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) row_loss[j] = total / float(2 * N_RES);
}

__global__ void k_loss_total(const float* row_loss, int n_rows, float* loss) {
  float t = 0.f;
  for (int j = 0; j < n_rows; ++j) t += row_loss[j];
  *loss = t;
}

template <int M>
__device__ __forceinline__ void loss_item_bwd(const LossArgs& a, const int4_ item, float2* smem) {
  constexpr int T = M / 16;
  constexpr int nb = M / 2 + 1;
  const int g = threadIdx.x / T, gtid = threadIdx.x % T;
  const float w_res = 1.f / float(2 * N_RES);
  const LossRow r = a.rows[item.x];
  constexpr int q = M == 512 ? 0 : M == 1024 ? 1 : 2;  // == item.y (dispatch)
  const int F = r.n_frames[q];
  const float4 stl = a.stats[2 * (item.x * N_RES + q)], str = a.stats[2 * (item.x * N_RES + q) + 1];
  const int f = item.z + g;
  const bool act = f < F;
  float2* fy = smem + g * fft::Padded<M>::size;
  __syncthreads();   // the previous item's readers of the buffers are done
  if (act) {
    // dL/dY per bin from the forward's cached spectra, as the Hermitian spectra of
    // both channels packed l + i r (stored conjugated: the forward FFT then inverts)
    const float2* sp = a.spec + r.spec_off[q] + int64_t(f) * nb;
    const int64_t plane = int64_t(F) * nb;
    for (int k = gtid; k <= M / 2; k += T) {
      const float2 yv[2] = {sp[k], sp[plane + k]};
      const float2 bt = sp[2 * plane + k];
      float2 gh[2];
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const float4 st = ch ? str : stl;
        float A = sqrtf(yv[ch].x * yv[ch].x + yv[ch].y * yv[ch].y);
        float B = ch ? bt.y : bt.x;
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
      const float2 Wk = make_float2(gh[0].x - gh[1].y, gh[0].y + gh[1].x);
      const float2 Wm = make_float2(gh[0].x + gh[1].y, -gh[0].y + gh[1].x);
      fy[fft::pad(k)] = make_float2(Wk.x, -Wk.y);
      if (k > 0 && k < M / 2) fy[fft::pad(M - k)] = make_float2(Wm.x, -Wm.y);
    }
  }
  __syncthreads();
  // the packed spectrum into the transform's registers (thread gtid: bins gtid + T m); the
  // windowed frame comes straight out of them
  float2 x[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) x[m] = fy[fft::pad(gtid + T * m)];
  __syncthreads();   // every thread has read its bins before the first pass writes
  fft::forward_regs_1buf<M>(x, fy, a.ptw, gtid);
  if (act) {
    float* fr = a.frames + r.frame_off[q] + int64_t(f) * 2 * M;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = gtid + T * m;
      const float w = hann<M>(a.tw, n);
      fr[n] = w * x[m].x;          // conj of the result: real part is l
      fr[M + n] = -w * x[m].y;     // minus imaginary part is r
    }
  }
}

__global__ void __launch_bounds__(256, 3) k_loss_bwd(LossArgs a) {
  extern __shared__ float2 smem2[];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int4_ item = a.items[it];
    switch (item.y) {
      case 0: loss_item_bwd<512>(a, item, smem2); break;
      case 1: loss_item_bwd<1024>(a, item, smem2); break;
      default: loss_item_bwd<2048>(a, item, smem2); break;
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

int launch_loss(int what, const LossLaunch& L, cudaStream_t s) {
  static bool init = false;
  // forward: y and target frames, 2 x (4096/M frames of M padded points) for every M;
  // backward: one set of frames
  const size_t smem = 2 * size_t(fft::Padded<4096>::size) * sizeof(float2);
  const size_t smem_b = size_t(fft::Padded<4096>::size) * sizeof(float2);
  static int res_fwd = 1, res_bwd = 1;   // resident CTAs per SM (one wave of the item loops)
  if (!init) {
    cudaFuncSetAttribute(k_loss_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(k_loss_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_b));
    res_fwd = resident_per_sm(reinterpret_cast<const void*>(k_loss_fwd), 256, smem);
    res_bwd = resident_per_sm(reinterpret_cast<const void*>(k_loss_bwd), 256, smem_b);
    init = true;
  }
  if (what < 0 || L.n_items <= 0) return 0;
  LossArgs a{L.rows, L.items, L.y, L.tgt, L.part, L.stats, L.frames, L.spec, L.tw, L.ptw, L.n_items};
  if (what == 0) {
    k_loss_fwd<<<grid_size(L.n_items, res_fwd), 256, smem, s>>>(a);
    k_loss_rows<<<L.n_rows, 256, 0, s>>>(L.rows, L.part, L.stats, L.row_loss);
    k_loss_total<<<1, 1, 0, s>>>(L.row_loss, L.n_rows, L.loss);
    return 3;
  }
  k_loss_bwd<<<grid_size(L.n_items, res_bwd), 256, smem_b, s>>>(a);
  dim3 grid((L.max_pitch + 255) / 256, L.n_rows);
  k_loss_ola<<<grid, 256, 0, s>>>(L.rows, L.frames, L.d_out);
  return 2;
}

}  // namespace grafx
