// Elementwise step kernels: mix/output (identity on the aggregated input), gain/panning
// (Eq. 2) and stereo imager (Eq. 3), forward and backward.  One work item is a tile
// of EW_TILE samples of one node; the gather of the predecessors and the
// aggregation (Algorithm 1 Gather + Aggregate) are fused into the loads, the store
// (Algorithm 1 Store) into the epilogue.  HBM-bound: 8 B x in-degree read and 8 B
// written per node-sample forward.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace grafx {

template <int TYPE>
struct Ew {
  // forward: y = f(u) for one quad of both channels
  __device__ static void fwd(const float* p, float4& l, float4& r) {
    if (TYPE == GRAFX_T_GAIN) {
      // rounded products (never contracted into a following add): a fused pair of steps
      // rounds exactly where the separate kernels' stored rows do
      float gl = expf(p[0]), gr = expf(p[1]);
      l = make_float4(__fmul_rn(gl, l.x), __fmul_rn(gl, l.y), __fmul_rn(gl, l.z), __fmul_rn(gl, l.w));
      r = make_float4(__fmul_rn(gr, r.x), __fmul_rn(gr, r.y), __fmul_rn(gr, r.z), __fmul_rn(gr, r.w));
    } else if (TYPE == GRAFX_T_IMAGER) {
      // mid = l + r, side = e^{p} (l - r); l' = (mid + side)/2, r' = (mid - side)/2
      float a = expf(p[0]);
      float4 m = make_float4(l.x + r.x, l.y + r.y, l.z + r.z, l.w + r.w);
      float4 s = make_float4(a * (l.x - r.x), a * (l.y - r.y), a * (l.z - r.z), a * (l.w - r.w));
      l = make_float4(0.5f * (m.x + s.x), 0.5f * (m.y + s.y), 0.5f * (m.z + s.z), 0.5f * (m.w + s.w));
      r = make_float4(0.5f * (m.x - s.x), 0.5f * (m.y - s.y), 0.5f * (m.z - s.z), 0.5f * (m.w - s.w));
    }
  }
};

constexpr int EW_Q = EW_TILE / 1024;  // quads per thread and channel in one tile

// The thread's EW_Q quads (stride 1024 samples) of both channels, summed over the
// edges [e0, e1): in-edges (ADJ = false: an input u, Eq. 1b) or consumer edges
// (ADJ = true: the adjoint of an output).  All loads of an edge are issued before any
// is used.
template <bool ADJ>
__device__ __forceinline__ void gather_range(const DevCtx& c, int e0, int e1, int t, int len, int pitch,
                                             float4 (&l)[EW_Q], float4 (&r)[EW_Q]) {
#pragma unroll
  for (int q = 0; q < EW_Q; ++q) l[q] = r[q] = f4zero();
  for (int e = e0; e < e1; ++e) {
    const float* row = ADJ ? out_adj_row(c, e) : in_row(c, e);
    float4 a[EW_Q], b[EW_Q];
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      const int tq = t + 1024 * q;
      if (tq < len) {
        a[q] = ld4(row + tq);
        b[q] = ld4(row + pitch + tq);
      } else {
        a[q] = b[q] = f4zero();
      }
    }
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      l[q] = f4add(l[q], a[q]);
      r[q] = f4add(r[q], b[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < EW_Q; ++q) {
    l[q] = mask4(l[q], t + 1024 * q, len);
    r[q] = mask4(r[q], t + 1024 * q, len);
  }
}

// Every in-edge (ADJ = false) or every consumer edge (ADJ = true) of a single-port node.
template <bool ADJ>
__device__ __forceinline__ void gather_q(const DevCtx& c, int v, int t, int len, int pitch, float4 (&l)[EW_Q],
                                         float4 (&r)[EW_Q]) {
  gather_range<ADJ>(c, ADJ ? c.tcsr_ptr[v] : c.csr_ptr[v], ADJ ? c.tcsr_ptr[v + 1] : c.csr_ptr[v + 1], t, len,
                    pitch, l, r);
}

__device__ __forceinline__ void store_q(float* row, int pitch, int t, int len, const float4 (&l)[EW_Q],
                                        const float4 (&r)[EW_Q]) {
#pragma unroll
  for (int q = 0; q < EW_Q; ++q) {
    const int tq = t + 1024 * q;
    if (tq < len) {
      st4(row + tq, l[q]);
      st4(row + pitch + tq, r[q]);
    }
  }
}

// Multi-port elementwise nodes (Eq. 1a with M, N > 1).  split: output 0 = (m, m),
// output 1 = (s, s) with m = (l + r)/2, s = (l - r)/2; merge: (u0_l + u1_l, u0_r - u1_r)
// of its inputs 0 and 1.  Backward: split's input adjoint from its two outputs'
// adjoints, merge's two input adjoints from its output's.
template <bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_ms_fwd(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev nd = c.nodes[v];
    float4 l[EW_Q], r[EW_Q];
    float* y = yrow_w(c, nd);
    if (SPLIT) {
      gather_q<false>(c, v, t, nd.len, nd.pitch, l, r);
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) {
        const float4 m = f4scale(f4add(l[q], r[q]), 0.5f), s = f4scale(f4sub(l[q], r[q]), 0.5f);
        l[q] = m;
        r[q] = s;
      }
      store_q(y, nd.pitch, t, nd.len, l, l);                 // output 0: (m, m)
      store_q(y + nd.rstride, nd.pitch, t, nd.len, r, r);    // output 1: (s, s)
    } else {
      float4 a[EW_Q], b[EW_Q];
      gather_range<false>(c, c.csr_ptr[v], c.in1_begin[v], t, nd.len, nd.pitch, l, r);
      gather_range<false>(c, c.in1_begin[v], c.csr_ptr[v + 1], t, nd.len, nd.pitch, a, b);
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) {
        l[q] = f4add(l[q], a[q]);
        r[q] = f4sub(r[q], b[q]);
      }
      store_q(y, nd.pitch, t, nd.len, l, r);
    }
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_ms_bwd(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev nd = c.nodes[v];
    float4 l[EW_Q], r[EW_Q];
    float* ub = arow_w(c, nd);
    if (SPLIT) {
      float4 a[EW_Q], b[EW_Q];
      gather_range<true>(c, c.tcsr_ptr[v], c.out1_begin[v], t, nd.len, nd.pitch, l, r);   // output 0
      gather_range<true>(c, c.out1_begin[v], c.tcsr_ptr[v + 1], t, nd.len, nd.pitch, a, b);   // output 1
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) {
        const float4 m = f4scale(f4add(l[q], r[q]), 0.5f), s = f4scale(f4add(a[q], b[q]), 0.5f);
        l[q] = f4add(m, s);
        r[q] = f4sub(m, s);
      }
      store_q(ub, nd.pitch, t, nd.len, l, r);
    } else {
      gather_q<true>(c, v, t, nd.len, nd.pitch, l, r);
      store_q(ub, nd.pitch, t, nd.len, l, r);                // input 0: ybar
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) r[q] = f4scale(r[q], -1.f);
      store_q(ub + nd.rstride, nd.pitch, t, nd.len, l, r);   // input 1: (ybar_l, -ybar_r)
    }
  }
}

template <int TYPE>
__global__ void __launch_bounds__(256, 4) k_ew_fwd(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev nd = c.nodes[v];
    float p[2] = {0.f, 0.f};
    if (TYPE == GRAFX_T_GAIN) { p[0] = c.params[nd.prow * 2]; p[1] = c.params[nd.prow * 2 + 1]; }
    if (TYPE == GRAFX_T_IMAGER) p[0] = c.params[nd.prow];
    float* y = yrow_w(c, nd);
    float4 l[EW_Q], r[EW_Q];
    gather_q<false>(c, v, t, nd.len, nd.pitch, l, r);
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      const int tq = t + 1024 * q;
      if (tq < nd.len) {
        Ew<TYPE>::fwd(p, l[q], r[q]);
        st4(y + tq, l[q]);
        st4(y + nd.pitch + tq, r[q]);
      }
    }
  }
}

// One quad of the backward of a gain or imager: the parameter-gradient terms into acc
// and ybar (bl, br) replaced by ubar = (df/du)^T ybar, from the input quad (ul, ur);
// a0, a1 = e^p of the parameters.
template <int TYPE>
__device__ __forceinline__ void ew_bwd_quad(float a0, float a1, float4& bl, float4& br, float4 ul, float4 ur,
                                            float (&acc)[2]) {
  if (TYPE == GRAFX_T_GAIN) {
    acc[0] += bl.x * ul.x + bl.y * ul.y + bl.z * ul.z + bl.w * ul.w;
    acc[1] += br.x * ur.x + br.y * ur.y + br.z * ur.z + br.w * ur.w;
    bl = make_float4(__fmul_rn(a0, bl.x), __fmul_rn(a0, bl.y), __fmul_rn(a0, bl.z), __fmul_rn(a0, bl.w));
    br = make_float4(__fmul_rn(a1, br.x), __fmul_rn(a1, br.y), __fmul_rn(a1, br.z), __fmul_rn(a1, br.w));
  } else if (TYPE == GRAFX_T_IMAGER) {
    const float4 L = bl, R = br, u0 = ul, u1 = ur;
    float4 mb = make_float4(0.5f * (L.x + R.x), 0.5f * (L.y + R.y), 0.5f * (L.z + R.z), 0.5f * (L.w + R.w));
    float4 sb = make_float4(0.5f * (L.x - R.x), 0.5f * (L.y - R.y), 0.5f * (L.z - R.z), 0.5f * (L.w - R.w));
    acc[0] += sb.x * (u0.x - u1.x) + sb.y * (u0.y - u1.y) + sb.z * (u0.z - u1.z) + sb.w * (u0.w - u1.w);
    bl = make_float4(mb.x + a0 * sb.x, mb.y + a0 * sb.y, mb.z + a0 * sb.z, mb.w + a0 * sb.w);
    br = make_float4(mb.x - a0 * sb.x, mb.y - a0 * sb.y, mb.z - a0 * sb.z, mb.w - a0 * sb.w);
  }
}

// Backward: ybar = sum of the consumers' input adjoints; ubar = (df/du)^T ybar;
// parameter-gradient partial of the tile into its own slot (no atomics).
// STORE = false: the input adjoints have no reader (the inputs are sources and no source
// adjoint is requested); only the parameter-gradient partials are formed.
template <int TYPE, bool STORE = true>
__global__ void __launch_bounds__(256, 3) k_ew_bwd(DevCtx c, int item0, int n_items) {
  __shared__ float sh[4 * 32];
  constexpr bool needs_u = TYPE == GRAFX_T_GAIN || TYPE == GRAFX_T_IMAGER;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev nd = c.nodes[v];
    float a0 = 1.f, a1 = 1.f;
    if (TYPE == GRAFX_T_GAIN) { a0 = expf(c.params[nd.prow * 2]); a1 = expf(c.params[nd.prow * 2 + 1]); }
    if (TYPE == GRAFX_T_IMAGER) a0 = expf(c.params[nd.prow]);
    float acc[2] = {0.f, 0.f};
    float* ub = arow_w(c, nd);
    float4 bl[EW_Q], br[EW_Q], ul[EW_Q], ur[EW_Q];
    const int ce = c.tcsr_ptr[v], pe = c.csr_ptr[v];
    if (needs_u && c.tcsr_ptr[v + 1] - ce == 1 && c.csr_ptr[v + 1] - pe == 1) {
      // one consumer and one producer (chains): issue all 4 * EW_Q loads at once
      const float* ar = out_adj_row(c, ce);
      const float* yr = in_row(c, pe);
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) {
        const int tq = t + 1024 * q;
        if (tq < nd.len) {
          bl[q] = ld4(ar + tq);
          br[q] = ld4(ar + nd.pitch + tq);
          ul[q] = ld4(yr + tq);
          ur[q] = ld4(yr + nd.pitch + tq);
        } else {
          bl[q] = br[q] = ul[q] = ur[q] = f4zero();
        }
      }
#pragma unroll
      for (int q = 0; q < EW_Q; ++q) {
        const int tq = t + 1024 * q;
        bl[q] = mask4(bl[q], tq, nd.len);
        br[q] = mask4(br[q], tq, nd.len);
        ul[q] = mask4(ul[q], tq, nd.len);
        ur[q] = mask4(ur[q], tq, nd.len);
      }
    } else {
      gather_q<true>(c, v, t, nd.len, nd.pitch, bl, br);
      if (needs_u) gather_q<false>(c, v, t, nd.len, nd.pitch, ul, ur);
    }
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      const int tq = t + 1024 * q;
      if (tq >= nd.len) continue;
      ew_bwd_quad<TYPE>(a0, a1, bl[q], br[q], ul[q], ur[q], acc);
      if (STORE) {
        st4(ub + tq, bl[q]);
        st4(ub + nd.pitch + tq, br[q]);
      }
    }
    if (needs_u) {
      block_sum<2>(acc, sh);
      if (threadIdx.x == 0) c.partial[w.w] = make_float4(a0 * acc[0], a1 * acc[1], 0.f, 0.f);
      __syncthreads();
    }
  }
}

// Fused pair of elementwise steps (the planner's fuse_next): node w of the second step
// (type TW, parameters c.params) has a single input, node v of the first step (type TV,
// parameters c.params2), whose only consumer is w.  Forward over w's tiles: u_v
// gathered once, y_v = f_v(u_v) stored (the row stays valid for every reader), y_w =
// f_w(y_v) stored.  The same arithmetic as the two separate kernels: bit-identical rows.
__device__ __forceinline__ void ew_params(int type, const float* tab, int prow, float (&p)[2]) {
  p[0] = p[1] = 0.f;
  if (type == GRAFX_T_GAIN) { p[0] = tab[prow * 2]; p[1] = tab[prow * 2 + 1]; }
  if (type == GRAFX_T_IMAGER) p[0] = tab[prow];
}

template <int TV, int TW>
__global__ void __launch_bounds__(256, 4) k_ew2_fwd(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int nw = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev ndw = c.nodes[nw];
    const int nv = c.csr_src[c.csr_ptr[nw]];
    const NodeDev ndv = c.nodes[nv];
    float pv[2], pw[2];
    ew_params(TV, c.params2, ndv.prow, pv);
    ew_params(TW, c.params, ndw.prow, pw);
    float* yv = yrow_w(c, ndv);
    float* yw = yrow_w(c, ndw);
    float4 l[EW_Q], r[EW_Q];
    gather_q<false>(c, nv, t, ndv.len, ndv.pitch, l, r);
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      const int tq = t + 1024 * q;
      if (tq < ndw.len) {
        Ew<TV>::fwd(pv, l[q], r[q]);
        st4(yv + tq, l[q]);
        st4(yv + ndv.pitch + tq, r[q]);
        Ew<TW>::fwd(pw, l[q], r[q]);
        st4(yw + tq, l[q]);
        st4(yw + ndw.pitch + tq, r[q]);
      }
    }
  }
}

// Backward of a fused pair over w's tiles: ybar_w gathered over w's consumers, u_v
// over v's inputs, y_v = f_v(u_v) recomputed (equal to the stored row); w's gradient
// terms and ybar_v = J_w^T ybar_w stay in registers (w's input adjoint row is read by v
// alone), then v's terms and ubar_v = J_v^T ybar_v go to v's adjoint row.  The tile's
// partials go to w's slot and to v's slot for the same tile (v's slots are its tiles in
// order from ext.x).
template <int TV, int TW>
__global__ void __launch_bounds__(256, 3) k_ew2_bwd(DevCtx c, int item0, int n_items) {
  __shared__ float sh[4 * 32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int nw = w.x, t = w.y + 4 * threadIdx.x;
    const NodeDev ndw = c.nodes[nw];
    const int nv = c.csr_src[c.csr_ptr[nw]];
    const NodeDev ndv = c.nodes[nv];
    float pv[2], pw[2];
    ew_params(TV, c.params2, ndv.prow, pv);
    ew_params(TW, c.params, ndw.prow, pw);
    const float av0 = expf(pv[0]), av1 = TV == GRAFX_T_GAIN ? expf(pv[1]) : 1.f;
    const float aw0 = expf(pw[0]), aw1 = TW == GRAFX_T_GAIN ? expf(pw[1]) : 1.f;
    float4 bl[EW_Q], br[EW_Q], ul[EW_Q], ur[EW_Q];
    gather_q<true>(c, nw, t, ndw.len, ndw.pitch, bl, br);
    gather_q<false>(c, nv, t, ndv.len, ndv.pitch, ul, ur);
    float accw[2] = {0.f, 0.f}, accv[2] = {0.f, 0.f};
    float* ub = arow_w(c, ndv);
#pragma unroll
    for (int q = 0; q < EW_Q; ++q) {
      const int tq = t + 1024 * q;
      if (tq >= ndw.len) continue;
      float4 yl = ul[q], yr = ur[q];
      Ew<TV>::fwd(pv, yl, yr);   // u_w = y_v
      ew_bwd_quad<TW>(aw0, aw1, bl[q], br[q], yl, yr, accw);
      ew_bwd_quad<TV>(av0, av1, bl[q], br[q], ul[q], ur[q], accv);
      st4(ub + tq, bl[q]);
      st4(ub + ndv.pitch + tq, br[q]);
    }
    float acc[4] = {accw[0], accw[1], accv[0], accv[1]};
    block_sum<4>(acc, sh);
    if (threadIdx.x == 0) {
      c.partial[w.w] = make_float4(aw0 * acc[0], aw1 * acc[1], 0.f, 0.f);
      c.partial[c.ext[nv].x + w.y / EW_TILE] = make_float4(av0 * acc[2], av1 * acc[3], 0.f, 0.f);
    }
    __syncthreads();
  }
}

// dLoss/dP for gain (2 columns) and imager (1 column): sum each node's tile
// partials in a fixed order.
__global__ void k_ew_finalize(DevCtx c, int node_begin, int node_end, int cols) {
  int v = node_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= node_end) return;
  const int4_ e = c.ext[v];
  float s0 = 0.f, s1 = 0.f;
  for (int k = 0; k < e.y; ++k) {
    float4 q = c.partial[e.x + k];
    s0 += q.x;
    s1 += q.y;
  }
  const int row = c.nodes[v].grow;
  c.dparams[row * cols] = s0;
  if (cols > 1) c.dparams[row * cols + 1] = s1;
}

// Source batch: dst[i] = sum_b part[b n + i] over the B copies in copy order (the
// gradient of a shared parameter row is the sum of its copies' gradients).
__global__ void k_fold_copies(const float* __restrict__ part, float* __restrict__ dst, int64_t n, int B) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += part[int64_t(b) * n + i];
    dst[i] = s;
  }
}

int launch_fold_copies(const float* part, float* dst, int64_t n, int B, cudaStream_t s) {
  if (n <= 0) return 0;
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_fold_copies<<<blocks, 256, 0, s>>>(part, dst, n, B);
  return 1;
}

static int grid_for(int n_items, int per_sm) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return std::max(1, std::min(n_items, sms * per_sm));
}

int resident_per_sm(const void* kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();   // a failed query is not sticky: keep it out of the next launch check
    n = 1;
  }
  return std::max(1, n);
}

int launch_ew2(bool bwd, int tv, int tw, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  const int g = grid_for(n_items, 8);
  constexpr int G = GRAFX_T_GAIN, S = GRAFX_T_IMAGER;
  if (tv == GRAFX_T_MIX) {   // mix -> output: forward only (both identities on the summed input)
    if (!bwd) k_ew2_fwd<GRAFX_T_MIX, GRAFX_T_OUT><<<g, 256, 0, s>>>(c, item0, n_items);
    return bwd ? 0 : 1;
  }
  if (bwd) {
    if (tv == G && tw == G) k_ew2_bwd<G, G><<<g, 256, 0, s>>>(c, item0, n_items);
    else if (tv == G) k_ew2_bwd<G, S><<<g, 256, 0, s>>>(c, item0, n_items);
    else if (tw == G) k_ew2_bwd<S, G><<<g, 256, 0, s>>>(c, item0, n_items);
    else k_ew2_bwd<S, S><<<g, 256, 0, s>>>(c, item0, n_items);
  } else {
    if (tv == G && tw == G) k_ew2_fwd<G, G><<<g, 256, 0, s>>>(c, item0, n_items);
    else if (tv == G) k_ew2_fwd<G, S><<<g, 256, 0, s>>>(c, item0, n_items);
    else if (tw == G) k_ew2_fwd<S, G><<<g, 256, 0, s>>>(c, item0, n_items);
    else k_ew2_fwd<S, S><<<g, 256, 0, s>>>(c, item0, n_items);
  }
  return 1;
}


int launch_ew_fwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  int g = grid_for(n_items, 8);
  switch (type) {
    case GRAFX_T_GAIN: k_ew_fwd<GRAFX_T_GAIN><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_IMAGER: k_ew_fwd<GRAFX_T_IMAGER><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_SPLIT: k_ms_fwd<true><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_MERGE: k_ms_fwd<false><<<g, 256, 0, s>>>(c, item0, n_items); break;
    default: k_ew_fwd<GRAFX_T_MIX><<<g, 256, 0, s>>>(c, item0, n_items); break;
  }
  return 1;
}

int launch_ew_bwd_nostore(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  const int g = grid_for(n_items, 8);
  if (type == GRAFX_T_GAIN) k_ew_bwd<GRAFX_T_GAIN, false><<<g, 256, 0, s>>>(c, item0, n_items);
  else if (type == GRAFX_T_IMAGER) k_ew_bwd<GRAFX_T_IMAGER, false><<<g, 256, 0, s>>>(c, item0, n_items);
  else return 0;   // mix/output: nothing but the adjoints
  return 1;
}

int launch_ew_bwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  int g = grid_for(n_items, 8);
  switch (type) {
    case GRAFX_T_GAIN: k_ew_bwd<GRAFX_T_GAIN><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_IMAGER: k_ew_bwd<GRAFX_T_IMAGER><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_SPLIT: k_ms_bwd<true><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_MERGE: k_ms_bwd<false><<<g, 256, 0, s>>>(c, item0, n_items); break;
    default: k_ew_bwd<GRAFX_T_MIX><<<g, 256, 0, s>>>(c, item0, n_items); break;
  }
  return 1;
}

int launch_ew_finalize(const DevCtx& c, int node_begin, int node_end, int cols, cudaStream_t s) {
  int n = node_end - node_begin;
  if (n <= 0) return 0;
  k_ew_finalize<<<(n + 127) / 128, 128, 0, s>>>(c, node_begin, node_end, cols);
  return 1;
}

int grid_size(int n_items, int per_sm) { return grid_for(n_items, per_sm); }

}  // namespace grafx
