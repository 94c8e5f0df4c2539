// Elementwise step kernels: mix/output (identity on the aggregated input), gain/panning
// (Eq. 2) and stereo imager (Eq. 3), forward and backward.  One work item is a tile
// of EW_TILE samples of one node; the gather of the predecessors and the
// aggregation (Algorithm 1 Gather + Aggregate) are fused into the loads, the store
// (Algorithm 1 Store) into the epilogue.  HBM-bound: 8 B x in-degree read and 8 B
// written per node-sample forward.
#include "common.cuh"
#include "kernels.h"

namespace grafx {

template <int TYPE>
struct Ew {
  // forward: y = f(u) for one quad of both channels
  __device__ static void fwd(const float* p, float4& l, float4& r) {
    if (TYPE == GRAFX_T_GAIN) {
      float gl = expf(p[0]), gr = expf(p[1]);
      l = make_float4(gl * l.x, gl * l.y, gl * l.z, gl * l.w);
      r = make_float4(gr * r.x, gr * r.y, gr * r.z, gr * r.w);
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

template <int TYPE>
__global__ void __launch_bounds__(256) k_ew_fwd(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t0 = w.y;
    const NodeDev nd = c.nodes[v];
    float p[2] = {0.f, 0.f};
    if (TYPE == GRAFX_T_GAIN) { p[0] = c.params[nd.prow * 2]; p[1] = c.params[nd.prow * 2 + 1]; }
    if (TYPE == GRAFX_T_IMAGER) p[0] = c.params[nd.prow];
    float* y = yrow_w(c, nd);
    const int t1 = min(t0 + EW_TILE, nd.len);
    for (int t = t0 + 4 * threadIdx.x; t < t1; t += 4 * blockDim.x) {
      float4 l = gather_in(c, v, 0, t, nd.len, nd.pitch);
      float4 r = gather_in(c, v, 1, t, nd.len, nd.pitch);
      Ew<TYPE>::fwd(p, l, r);
      st4(y + t, l);
      st4(y + nd.pitch + t, r);
    }
  }
}

// Backward: ybar = sum of the consumers' input adjoints; ubar = (df/du)^T ybar;
// parameter-gradient partial of the tile into its own slot (no atomics).
template <int TYPE>
__global__ void __launch_bounds__(256) k_ew_bwd(DevCtx c, int item0, int n_items) {
  __shared__ float sh[4 * 32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x, t0 = w.y;
    const NodeDev nd = c.nodes[v];
    float a0 = 1.f, a1 = 1.f;
    if (TYPE == GRAFX_T_GAIN) { a0 = expf(c.params[nd.prow * 2]); a1 = expf(c.params[nd.prow * 2 + 1]); }
    if (TYPE == GRAFX_T_IMAGER) a0 = expf(c.params[nd.prow]);
    float acc[2] = {0.f, 0.f};
    float* ub = arow_w(c, nd);
    const int t1 = min(t0 + EW_TILE, nd.len);
    for (int t = t0 + 4 * threadIdx.x; t < t1; t += 4 * blockDim.x) {
      float4 bl = gather_out_adj(c, v, 0, t, nd.len, nd.pitch);
      float4 br = gather_out_adj(c, v, 1, t, nd.len, nd.pitch);
      if (TYPE == GRAFX_T_GAIN) {
        float4 ul = gather_in(c, v, 0, t, nd.len, nd.pitch);
        float4 ur = gather_in(c, v, 1, t, nd.len, nd.pitch);
        acc[0] += bl.x * ul.x + bl.y * ul.y + bl.z * ul.z + bl.w * ul.w;
        acc[1] += br.x * ur.x + br.y * ur.y + br.z * ur.z + br.w * ur.w;
        bl = make_float4(a0 * bl.x, a0 * bl.y, a0 * bl.z, a0 * bl.w);
        br = make_float4(a1 * br.x, a1 * br.y, a1 * br.z, a1 * br.w);
      } else if (TYPE == GRAFX_T_IMAGER) {
        float4 ul = gather_in(c, v, 0, t, nd.len, nd.pitch);
        float4 ur = gather_in(c, v, 1, t, nd.len, nd.pitch);
        float4 mb = make_float4(0.5f * (bl.x + br.x), 0.5f * (bl.y + br.y), 0.5f * (bl.z + br.z), 0.5f * (bl.w + br.w));
        float4 sb = make_float4(0.5f * (bl.x - br.x), 0.5f * (bl.y - br.y), 0.5f * (bl.z - br.z), 0.5f * (bl.w - br.w));
        acc[0] += sb.x * (ul.x - ur.x) + sb.y * (ul.y - ur.y) + sb.z * (ul.z - ur.z) + sb.w * (ul.w - ur.w);
        bl = make_float4(mb.x + a0 * sb.x, mb.y + a0 * sb.y, mb.z + a0 * sb.z, mb.w + a0 * sb.w);
        br = make_float4(mb.x - a0 * sb.x, mb.y - a0 * sb.y, mb.z - a0 * sb.z, mb.w - a0 * sb.w);
      }
      st4(ub + t, bl);
      st4(ub + nd.pitch + t, br);
    }
    if (TYPE == GRAFX_T_GAIN || TYPE == GRAFX_T_IMAGER) {
      block_sum<2>(acc, sh);
      if (threadIdx.x == 0) c.partial[w.w] = make_float4(a0 * acc[0], a1 * acc[1], 0.f, 0.f);
      __syncthreads();
    }
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
  const int row = c.nodes[v].prow;
  c.dparams[row * cols] = s0;
  if (cols > 1) c.dparams[row * cols + 1] = s1;
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

int launch_ew_fwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  int g = grid_for(n_items, 8);
  switch (type) {
    case GRAFX_T_GAIN: k_ew_fwd<GRAFX_T_GAIN><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_IMAGER: k_ew_fwd<GRAFX_T_IMAGER><<<g, 256, 0, s>>>(c, item0, n_items); break;
    default: k_ew_fwd<GRAFX_T_MIX><<<g, 256, 0, s>>>(c, item0, n_items); break;
  }
  return 1;
}

int launch_ew_bwd(int type, const DevCtx& c, int item0, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  int g = grid_for(n_items, 8);
  switch (type) {
    case GRAFX_T_GAIN: k_ew_bwd<GRAFX_T_GAIN><<<g, 256, 0, s>>>(c, item0, n_items); break;
    case GRAFX_T_IMAGER: k_ew_bwd<GRAFX_T_IMAGER><<<g, 256, 0, s>>>(c, item0, n_items); break;
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
