// Compressor (Eq. 8-12): exact one-pole envelope g[n] = a g[n-1] + (1-a) x[n],
// x = (u_l + u_r)^2, as a chunked linear-recurrence scan, then the quadratic-knee
// static curve and the gain exp(G_y - G_u).
//
// One work item is a chunk of CH = 256 * SPT samples of one node.  Inside a chunk:
// every thread runs the recursion over its SPT samples with zero initial state, a
// warp-shuffle scan and a cross-warp scan combine the per-thread states with the
// decay a^SPT.  Across chunks, one pass: each chunk publishes its zero-start end state
// (its aggregate) as soon as its in-chunk scan is done, and one warp forms the state
// entering it as a fixed-order, decay-weighted sum of the aggregates of the node's
// earlier chunks (deterministic: no dependence on which chunks had finished).  Chunks
// are handed out by an atomic ticket in chunk-major order (the c-th chunk of every node
// of the step before any node's (c+1)-th), so every chunk waited on is held by a CTA that
// took its ticket earlier and, on steps of many nodes, has long finished; every wait is
// bounded and records ST_TIMEOUT on expiry.  The forward stores each chunk's entering
// state (one float) so that the backward can recompute g[n] exactly.
//
// Backward: ybar gives a_n = dL/dg[n]; lambda[n] = a_n + alpha lambda[n+1] runs the same
// way from each node's end (its own aggregate words); ubar_x = k ybar_x + 2 u_m
// (1 - alpha) lambda and the parameter partials (sum lambda (g[n-1] - x[n]) for alpha,
// sum Gybar dGy/dT|W|R) go to one slot per chunk.
//
// The allocation-free single-row forward at the end of this file takes its chunks in
// order and uses a decoupled look-back instead: each chunk publishes its aggregate, then
// its inclusive end state once its carry is known, and one warp reads the 32 preceding
// states at once, walking back until it meets an inclusive one.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace grafx {

constexpr float COMP_EPS = 1e-7f;
constexpr int SPIN_LIMIT = 1 << 22;

struct Knee {
  float gy, dgu, dt, dw, dr;
};

// Per-node constants of the static curves: the divisions by R and W are taken once
// per chunk instead of per sample.
struct KneeCoef {
  float T, W, R, cR, invR, invRR, inv2W, inv4W, inv4WW;
};
__device__ __forceinline__ KneeCoef knee_coef(float T, float W, float R) {
  KneeCoef q;
  q.T = T;
  q.W = W;
  q.R = R;
  q.invR = 1.f / R;
  q.cR = q.invR - 1.f;
  q.invRR = q.invR * q.invR;
  q.inv2W = 0.5f / W;
  q.inv4W = 0.25f / W;
  q.inv4WW = 0.25f / (W * W);
  return q;
}

// Eq. 13 (noisegate): G_y = G_u above T + W, G_u + (1-R)(G_u-T-W)^2/(4W) in the knee,
// T + R (G_u - T) below T - W; with the partial derivatives of G_y.
__device__ __forceinline__ Knee gate_knee(float gu, const KneeCoef& q) {
  Knee k;
  if (gu >= q.T + q.W) {
    k.gy = gu;
    k.dgu = 1.f;
    k.dt = k.dw = k.dr = 0.f;
  } else if (gu >= q.T - q.W) {
    const float d = gu - q.T - q.W, c = 1.f - q.R;
    k.gy = gu + c * d * d * q.inv4W;
    k.dgu = 1.f + c * d * q.inv2W;
    k.dt = -c * d * q.inv2W;
    k.dw = c * (-d * q.inv2W - d * d * q.inv4WW);
    k.dr = -d * d * q.inv4W;
  } else {
    k.gy = q.T + q.R * (gu - q.T);
    k.dgu = q.R;
    k.dt = 1.f - q.R;
    k.dw = 0.f;
    k.dr = gu - q.T;
  }
  return k;
}

// Eq. 10-11 and the partial derivatives of G_y.
__device__ __forceinline__ Knee knee(float gu, const KneeCoef& q) {
  Knee k;
  if (gu >= q.T + q.W) {
    k.gy = q.T + (gu - q.T) * q.invR;
    k.dgu = q.invR;
    k.dt = -q.cR;
    k.dw = 0.f;
    k.dr = -(gu - q.T) * q.invRR;
  } else if (gu >= q.T - q.W) {
    const float d = gu - q.T + q.W;
    k.gy = gu + q.cR * d * d * q.inv4W;
    k.dgu = 1.f + q.cR * d * q.inv2W;
    k.dt = -q.cR * d * q.inv2W;
    k.dw = q.cR * (d * q.inv2W - d * d * q.inv4WW);
    k.dr = -d * d * q.inv4W * q.invRR;
  } else {
    k.gy = gu;
    k.dgu = 1.f;
    k.dt = k.dw = k.dr = 0.f;
  }
  return k;
}

// ln and exp of the per-sample gain path: the hardware approximations (__logf: absolute
// error <= 2^-21.4 on [0.5, 2], 3 ulp elsewhere; __expf: a few ulp over the gains'
// range), inside the outputs' 1e-5 tolerance.  Built with GRAFX_PRECISE_GAIN, the
// library's correctly rounded logf / expf and an IEEE division instead (the build
// variant "precise" of build.py), to measure what the approximations cost.
#ifdef GRAFX_PRECISE_GAIN
__device__ __forceinline__ float ln_env(float g) { return logf(g + COMP_EPS); }
__device__ __forceinline__ float exp_gain(float x) { return expf(x); }
__device__ __forceinline__ float env_div(float a, float b) { return __fdiv_rn(a, b); }
#else
__device__ __forceinline__ float ln_env(float g) { return __logf(g + COMP_EPS); }
__device__ __forceinline__ float exp_gain(float x) { return __expf(x); }
__device__ __forceinline__ float env_div(float a, float b) { return __fdividef(a, b); }
#endif

__device__ __forceinline__ unsigned long long pack_flag(unsigned st, float v) {
  return (static_cast<unsigned long long>(st) << 32) | __float_as_uint(v);
}

// Wait (bounded by `limit` polls) for the flag word *f; returns its status (1 aggregate,
// 2 inclusive) and value, or on expiry records ST_TIMEOUT in *status and returns 2 with
// a zero value.
__device__ __forceinline__ unsigned wait_word(const unsigned long long* fp, uint32_t* status, int limit, float* val) {
  volatile const unsigned long long* f = fp;
  for (int i = 0; i < limit; ++i) {
    unsigned long long w = *f;
    unsigned st = unsigned(w >> 32);
    if (st) {
      *val = __uint_as_float(unsigned(w & 0xffffffffu));
      return st;
    }
    __nanosleep(64);
  }
  atomicOr(status, ST_TIMEOUT);
  *val = 0.f;
  return 2;
}

// Wait (bounded) for the look-back flag of item j.
__device__ __forceinline__ unsigned wait_flag(const DevCtx& c, int j, float* val) {
  return wait_word(c.flags + j, c.status, SPIN_LIMIT, val);
}

// One warp polls `flag` as a look-back does (failure-detection self-test).
__global__ void k_wait_selftest(const unsigned long long* flag, uint32_t* status, int limit, float* value) {
  float v = 0.f;
  const unsigned st = wait_word(flag, status, limit, &v);
  if (threadIdx.x == 0) *value = st == 2 ? v : -1.f;
}

__device__ __forceinline__ void publish(const DevCtx& c, int j, unsigned st, float v) {
  __threadfence();
  atomicExch(c.flags + j, pack_flag(st, v));
}

// Carry into the current chunk from the chunks before it in ticket order, run by one
// full warp: lane l examines item end - l, so 32 predecessors are read at once.  The
// carry is sum_l exp(la_ch * l) * state(end - l) over the lanes up to the first one
// whose state is inclusive, continuing 32 items further back if none is.  Items before
// `first` (the node's first chunk, which always publishes an inclusive state) are not
// read.  la_ch = ln(decay of one chunk).  Returns the carry in every lane.
__device__ float look_back_warp(const DevCtx& c, int end, int first, float la_ch) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f, dec = 1.f;
  while (true) {
    const int j = end - lane;
    float val = 0.f;
    const unsigned st = j < first ? 2u : wait_flag(c, j, &val);
    const unsigned incl = __ballot_sync(0xffffffffu, st == 2u);
    const int stop = incl ? __ffs(int(incl)) - 1 : 31;
    float w = lane <= stop ? val * expf(la_ch * float(lane)) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    acc += dec * w;
    if (incl) break;
    dec *= expf(la_ch * 32.f);
    end -= 32;
  }
  return acc;
}

// Carry into the current chunk as a fixed-order sum over the aggregates (zero-start end
// states) of the node's earlier chunks, items first .. end with `end` the nearest:
// carry = sum_l D^l agg(end - l), D = exp(la_ch) the decay of one chunk.  Run by one full
// warp: lane i takes l = i, i + 32, ... in increasing order, then a xor-shuffle tree adds
// the lanes (every lane gets the same bits); the value depends on the data only, not on
// which chunks had finished (deterministic, unlike a look-back that stops at the first
// inclusive state).  Terms with D^l < 2^-30 are not read: their sum is at most
// 2^-30 / (1 - D) of the largest aggregate, below 1e-8 for alpha <= 0.9999 (the fit's
// parameter map) and chunks of >= 1024 samples, and the cut depends on alpha only.  Waits
// are bounded (wait_flag).
__device__ float carry_sum_warp(const DevCtx& c, int end, int first, float la_ch) {
  const int lane = threadIdx.x & 31;
  const float lmax = la_ch < 0.f ? -20.794415f / la_ch : 1e30f;   // D^l >= 2^-30
  float acc = 0.f;
  for (int l = lane; end - l >= first && float(l) <= lmax; l += 32) {
    float val = 0.f;
    wait_flag(c, end - l, &val);
    acc += expf(la_ch * float(l)) * val;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Block-wide scan of per-thread states with a common decay D = exp(la_spt): a thread
// maps the state entering it to D * state + b.  Forward: state flows from thread i-1
// to thread i; reverse: from thread i+1 to thread i.  Returns the state entering this
// thread when zero enters the chunk, and sets *total to the state leaving the chunk.
// Requires blockDim.x == 256; `sh` holds >= 17 floats.
template <bool REVERSE>
__device__ __forceinline__ float block_affine_scan(float b, float la_spt, float* sh, float* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float incl = b;  // Hillis-Steele: incl_i += D^d incl_{i-d} (forward) / incl_{i+d} (reverse)
  float Dd = expf(la_spt);  // D^d for d = 1, 2, 4, ... by squaring
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    float o = REVERSE ? __shfl_down_sync(0xffffffffu, incl, d) : __shfl_up_sync(0xffffffffu, incl, d);
    bool ok = REVERSE ? (lane + d < 32) : (lane >= d);
    if (ok) incl += Dd * o;
    Dd *= Dd;
  }
  float excl = REVERSE ? __shfl_down_sync(0xffffffffu, incl, 1) : __shfl_up_sync(0xffffffffu, incl, 1);
  if (REVERSE ? (lane == 31) : (lane == 0)) excl = 0.f;
  if (REVERSE ? (lane == 0) : (lane == 31)) sh[warp] = incl;  // state leaving the warp
  __syncthreads();
  if (threadIdx.x == 0) {
    const float d32 = Dd;  // D^32
    float run = 0.f;
    for (int k = 0; k < 8; ++k) {
      int wi = REVERSE ? 7 - k : k;
      float tw = sh[wi];
      sh[8 + wi] = run;          // state entering warp wi
      run = d32 * run + tw;
    }
    sh[16] = run;
  }
  __syncthreads();
  const int dist = REVERSE ? (31 - lane) : lane;  // threads between the warp edge and this one
  *total = sh[16];
  return excl + expf(la_spt * float(dist)) * sh[8 + warp];
}

// The single row feeding node v (its in-edge source, or with adj the one consumer's
// input-adjoint row), or null when there are several.
__device__ __forceinline__ const float* single_row(const DevCtx& c, int v, bool adj) {
  if (!adj) {
    const int e0 = c.csr_ptr[v];
    return c.csr_ptr[v + 1] - e0 == 1 ? in_row(c, e0) : nullptr;
  }
  const int e0 = c.tcsr_ptr[v];
  return c.tcsr_ptr[v + 1] - e0 == 1 ? out_adj_row(c, e0) : nullptr;
}

template <int SPT>
__device__ __forceinline__ void load_chunk(const DevCtx& c, int v, const NodeDev& nd, int t, float* ul, float* ur,
                                           bool adj) {
  if (const float* row = single_row(c, v, adj)) {  // one row: resolve it once, then plain loads
#pragma unroll
    for (int q = 0; q < SPT / 4; ++q) {
      float4 l = f4zero(), r = f4zero();
      if (t + 4 * q < nd.len) {
        l = mask4(ld4(row + t + 4 * q), t + 4 * q, nd.len);
        r = mask4(ld4(row + nd.pitch + t + 4 * q), t + 4 * q, nd.len);
      }
      ul[4 * q + 0] = l.x; ul[4 * q + 1] = l.y; ul[4 * q + 2] = l.z; ul[4 * q + 3] = l.w;
      ur[4 * q + 0] = r.x; ur[4 * q + 1] = r.y; ur[4 * q + 2] = r.z; ur[4 * q + 3] = r.w;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < SPT / 4; ++q) {
    float4 l, r;
    if (t + 4 * q < nd.len) {
      if (adj) {
        l = gather_out_adj(c, v, 0, t + 4 * q, nd.len, nd.pitch);
        r = gather_out_adj(c, v, 1, t + 4 * q, nd.len, nd.pitch);
      } else {
        l = gather_in(c, v, 0, t + 4 * q, nd.len, nd.pitch);
        r = gather_in(c, v, 1, t + 4 * q, nd.len, nd.pitch);
      }
    } else {
      l = r = f4zero();
    }
    ul[4 * q + 0] = l.x; ul[4 * q + 1] = l.y; ul[4 * q + 2] = l.z; ul[4 * q + 3] = l.w;
    ur[4 * q + 0] = r.x; ur[4 * q + 1] = r.y; ur[4 * q + 2] = r.z; ur[4 * q + 3] = r.w;
  }
}

// This thread's SPT samples of both channels summed over the in-edges [e0, e1) (one
// input port of a multi-input node).
template <int SPT>
__device__ __forceinline__ void load_range(const DevCtx& c, int e0, int e1, const NodeDev& nd, int t, float* l,
                                           float* r) {
#pragma unroll
  for (int q = 0; q < SPT / 4; ++q) {
    float4 a = f4zero(), b = f4zero();
    if (t + 4 * q < nd.len)
      for (int e = e0; e < e1; ++e) {
        const float* row = in_row(c, e);
        a = f4add(a, ld4(row + t + 4 * q));
        b = f4add(b, ld4(row + nd.pitch + t + 4 * q));
      }
    a = mask4(a, t + 4 * q, nd.len);
    b = mask4(b, t + 4 * q, nd.len);
    l[4 * q + 0] = a.x; l[4 * q + 1] = a.y; l[4 * q + 2] = a.z; l[4 * q + 3] = a.w;
    r[4 * q + 0] = b.x; r[4 * q + 1] = b.y; r[4 * q + 2] = b.z; r[4 * q + 3] = b.w;
  }
}

// Kernel variants: the compressor (Eq. 10-11), the noisegate (Eq. 13) and the sidechain
// compressor (the compressor's curve; envelope from input 1, gain on input 0).
constexpr int MODE_COMP = 0, MODE_GATE = 1, MODE_SC = 2;

// Prefetch: this thread's SPT samples of both channels of `row` from t into its own
// slots dst[ch * 256 * SPT + threadIdx.x * SPT ...] (zeros past the node's length).
// Every thread reads back only its own slots, so one buffer serves consecutive chunks.
template <int SPT>
__device__ __forceinline__ void prefetch_rows(float* dst, const float* row, const NodeDev& nd, int t) {
  constexpr int CH = 256 * SPT;
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int q = 0; q < SPT / 4; ++q) {
      const int tq = t + 4 * q;
      const bool in = tq < nd.len;
      cp_async16(dst + ch * CH + threadIdx.x * SPT + 4 * q, in ? row + ch * nd.pitch + tq : row, in ? 16 : 0);
    }
}

template <int SPT>
__device__ __forceinline__ void read_rows(const float* src, const NodeDev& nd, int t, float* l, float* r) {
  constexpr int CH = 256 * SPT;
#pragma unroll
  for (int q = 0; q < SPT / 4; ++q) {
    float4 a = *reinterpret_cast<const float4*>(src + threadIdx.x * SPT + 4 * q);
    float4 b = *reinterpret_cast<const float4*>(src + CH + threadIdx.x * SPT + 4 * q);
    a = mask4(a, t + 4 * q, nd.len);
    b = mask4(b, t + 4 * q, nd.len);
    l[4 * q] = a.x, l[4 * q + 1] = a.y, l[4 * q + 2] = a.z, l[4 * q + 3] = a.w;
    r[4 * q] = b.x, r[4 * q + 1] = b.y, r[4 * q + 2] = b.z, r[4 * q + 3] = b.w;
  }
}

// Start the copies of item `it`'s single-row inputs (u, and with ADJ also ybar) into buf.
template <int SPT, bool ADJ>
__device__ __forceinline__ void prefetch_item(const DevCtx& c, int item, float* buf) {
  constexpr int CH = 256 * SPT;
  const int4_ w = c.items[item];
  const NodeDev nd = c.nodes[w.x];
  const int t = w.y * CH + threadIdx.x * SPT;
  if (const float* row = single_row(c, w.x, false)) prefetch_rows<SPT>(buf, row, nd, t);
  if (ADJ)
    if (const float* row = single_row(c, w.x, true)) prefetch_rows<SPT>(buf + 2 * CH, row, nd, t);
  cp_async_commit();
}

// This thread's u (and ybar) of the current chunk: from the prefetch buffer when the
// node has a single row feeding it, else gathered.
template <int SPT>
__device__ __forceinline__ void fetch_rows(const DevCtx& c, int v, const NodeDev& nd, int t, const float* buf,
                                           float* l, float* r, bool adj) {
  if (single_row(c, v, adj)) read_rows<SPT>(buf, nd, t, l, r);
  else load_chunk<SPT>(c, v, nd, t, l, r, adj);
}

template <int SPT>
__device__ __forceinline__ void store_chunk(float* row, const NodeDev& nd, int t, const float* yl, const float* yr) {
#pragma unroll
  for (int q = 0; q < SPT / 4; ++q) {
    if (t + 4 * q < nd.pitch) {
      st4(row + t + 4 * q, make_float4(yl[4 * q], yl[4 * q + 1], yl[4 * q + 2], yl[4 * q + 3]));
      st4(row + nd.pitch + t + 4 * q, make_float4(yr[4 * q], yr[4 * q + 1], yr[4 * q + 2], yr[4 * q + 3]));
    }
  }
}

// Envelope of the thread's SPT samples from the state entering the thread.
// Identical arithmetic in the forward and backward kernels.
template <int SPT>
__device__ __forceinline__ void envelope(const float* x, float alpha, float cin, float* g) {
  float s = cin;
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    s = alpha * s + (1.f - alpha) * x[i];
    g[i] = s;
  }
}

// The envelope recursion g[n] = alpha g[n-1] + (1 - alpha) x[n] is linear, so a chunk's
// effect on the chunks after it is one number: its state at the chunk's end with zero
// entering it (its aggregate).  Forward and backward each run in one pass: every chunk
// publishes its aggregate and takes the state entering it from the chunks before it
// (after it, for the reverse recursion lambda[n] = a[n] + alpha lambda[n+1] of the
// backward) by a decoupled look-back; the chunks are handed out in chunk-major order, so
// that on steps of many nodes a chunk's neighbour in the recursion has finished long
// before it is needed.

// The envelope input x[n] of this thread's samples: the squared mid of the node's input
// (the compressor and the noisegate) or of its key, input 1 (the sidechain compressor).
template <int SPT, int MODE>
__device__ __forceinline__ void env_input(const DevCtx& c, int v, const NodeDev& nd, int t, float* x) {
  float l[SPT], r[SPT];
  if constexpr (MODE == MODE_SC) load_range<SPT>(c, c.in1_begin[v], c.csr_ptr[v + 1], nd, t, l, r);
  else load_chunk<SPT>(c, v, nd, t, l, r, false);
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    const float m = l[i] + r[i];
    x[i] = m * m;
  }
}

// Forward in one pass: chunks handed out by an atomic ticket in chunk-major order (the
// c-th chunk of every node of the step before any node's (c+1)-th); each publishes its
// aggregate (state at its end with zero entering), forms the state entering it from the
// aggregates of the node's earlier chunks (carry_sum_warp; words indexed by the chunk's
// global id, contiguous per node), stores it for the backward and applies the gain.  The
// inputs are read once.  Bounded waits record ST_TIMEOUT.
template <int SPT, int MODE>
__global__ void __launch_bounds__(256, SPT >= 16 ? 2 : 4) k_comp_fwd_lb(DevCtx c, int item0, int n_items, int ticket) {
  constexpr int CH = 256 * SPT;
  constexpr bool GATE = MODE == MODE_GATE, SC = MODE == MODE_SC;
  extern __shared__ __align__(16) float buf[];   // 2 CH floats: the next ticket's u (prefetched)
  __shared__ float sh[32];
  __shared__ int s_it[2];
  __shared__ float s_cin;
  if (threadIdx.x == 0) s_it[0] = atomicAdd(c.tickets + ticket, 1);
  __syncthreads();
  int it = s_it[0], slot = 0;
  const int chunk0 = c.items[item0].z;   // the step's first chunk (its first node's chunk 0)
  if (!SC && it < n_items) prefetch_item<SPT, false>(c, item0 + it, buf);
  while (it < n_items) {
    if (threadIdx.x == 0) s_it[slot ^ 1] = atomicAdd(c.tickets + ticket, 1);  // read after the scan's barriers
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const float* p = c.params + nd.prow * 4;
    const float alpha = p[0];
    const KneeCoef kq = knee_coef(p[1], p[2], p[3]);
    const float la = logf(alpha);
    const int t = w.y * CH + threadIdx.x * SPT;
    float ul[SPT], ur[SPT], x[SPT], g[SPT];
    cp_async_wait_all();
    if constexpr (SC) {
      load_range<SPT>(c, c.csr_ptr[v], c.in1_begin[v], nd, t, ul, ur);   // main (input 0)
      env_input<SPT, MODE>(c, v, nd, t, x);                               // key (input 1)
    } else {
      fetch_rows<SPT>(c, v, nd, t, buf, ul, ur, false);
#pragma unroll
      for (int i = 0; i < SPT; ++i) { float m = ul[i] + ur[i]; x[i] = m * m; }
    }
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < SPT; ++i) b = alpha * b + (1.f - alpha) * x[i];
    float total;
    const float excl = block_affine_scan<false>(b, la * SPT, sh, &total);
    const int next = s_it[slot ^ 1];
    // every thread has read its own slots of buf (before the scan's barriers)
    if (!SC && next < n_items) prefetch_item<SPT, false>(c, item0 + next, buf);
    if (threadIdx.x < 32) {
      const int fidx = item0 + (w.z - chunk0);
      if (threadIdx.x == 0) publish(c, fidx, 1, total);
      const float cin = w.y == 0 ? 0.f : carry_sum_warp(c, fidx - 1, fidx - w.y, la * CH);
      if (threadIdx.x == 0) {
        s_cin = cin;
        c.comp_carry[w.z] = cin;   // the state entering the chunk, for the backward
      }
    }
    __syncthreads();
    const float cin_t = excl + expf(la * float(SPT * threadIdx.x)) * s_cin;
    envelope<SPT>(x, alpha, cin_t, g);
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      float gu = ln_env(g[i]);
      Knee k = GATE ? gate_knee(gu, kq) : knee(gu, kq);
      float gain = exp_gain(k.gy - gu);
      ul[i] *= gain;
      ur[i] *= gain;
    }
    store_chunk<SPT>(yrow_w(c, nd), nd, t, ul, ur);
    __syncthreads();   // sh and s_cin are reused by the next ticket
    it = next;
    slot ^= 1;
  }
  cp_async_wait_all();
}

// Backward in one pass: the reverse recursion's state entering a chunk is formed from the
// aggregates of the chunks after it (carry_sum_warp; chunks handed out by an atomic
// ticket in chunk-major order from each node's end; the words indexed by the chunk's
// partial slot, contiguous per node from its last chunk; bounded waits record
// ST_TIMEOUT).
template <int SPT, int MODE>
__global__ void __launch_bounds__(256, SPT >= 16 ? 1 : 4) k_comp_bwd_lb(DevCtx c, int item0, int n_items, int ticket) {
  constexpr int CH = 256 * SPT;
  constexpr bool GATE = MODE == MODE_GATE, SC = MODE == MODE_SC;
  extern __shared__ __align__(16) float buf[];  // 4 * CH floats: prefetched u and ybar rows
  __shared__ float sh[32];
  __shared__ float glast[256];
  __shared__ float red[4 * 32];
  __shared__ int s_it[2];
  __shared__ float s_lin;
  if (threadIdx.x == 0) s_it[0] = atomicAdd(c.tickets + ticket, 1);
  __syncthreads();
  int it = s_it[0], slot = 0;
  const int slot0 = c.items[item0].w;   // the step's first partial slot (its first node's last chunk)
  if (!SC && it < n_items) prefetch_item<SPT, true>(c, item0 + it, buf);
  while (it < n_items) {
    if (threadIdx.x == 0) s_it[slot ^ 1] = atomicAdd(c.tickets + ticket, 1);  // read after the scan's barriers
    const int4_ w = c.items[item0 + it];
    const int v = w.x, chunk = w.y;
    const NodeDev nd = c.nodes[v];
    const float* p = c.params + nd.prow * 4;
    const float alpha = p[0];
    const KneeCoef kq = knee_coef(p[1], p[2], p[3]);
    const float la = logf(alpha);
    const int t = chunk * CH + threadIdx.x * SPT;
    const int n_chunks = (nd.len + CH - 1) / CH;
    float ul[SPT], ur[SPT], bl[SPT], br[SPT], x[SPT], g[SPT], a[SPT];
    float km[SC ? SPT : 1];   // sidechain: the key's mid l + r
    cp_async_wait_all();
    if constexpr (SC) {
      float kr[SPT];
      load_range<SPT>(c, c.csr_ptr[v], c.in1_begin[v], nd, t, ul, ur);      // main (input 0)
      load_range<SPT>(c, c.in1_begin[v], c.csr_ptr[v + 1], nd, t, km, kr);  // key (input 1)
      load_chunk<SPT>(c, v, nd, t, bl, br, true);
#pragma unroll
      for (int i = 0; i < SPT; ++i) { km[i] += kr[i]; x[i] = km[i] * km[i]; }
    } else {
      fetch_rows<SPT>(c, v, nd, t, buf, ul, ur, false);
      fetch_rows<SPT>(c, v, nd, t, buf + 2 * CH, bl, br, true);
#pragma unroll
      for (int i = 0; i < SPT; ++i) { float m = ul[i] + ur[i]; x[i] = m * m; }
    }
    // recompute the envelope from the stored chunk carry-in (same arithmetic as forward)
    const float carry_g = c.comp_carry[w.z];
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < SPT; ++i) b = alpha * b + (1.f - alpha) * x[i];
    float total;
    float excl = block_affine_scan<false>(b, la * SPT, sh, &total);
    const int next = s_it[slot ^ 1];
    if (!SC && next < n_items) prefetch_item<SPT, true>(c, item0 + next, buf);
    const float cin = excl + expf(la * float(SPT * threadIdx.x)) * carry_g;
    envelope<SPT>(x, alpha, cin, g);
    // local adjoints
    float gain[SPT], gyb[SPT], dT = 0.f, dW = 0.f, dR = 0.f;
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      float gu = ln_env(g[i]);
      Knee k = GATE ? gate_knee(gu, kq) : knee(gu, kq);
      gain[i] = exp_gain(k.gy - gu);
      float kbar = bl[i] * ul[i] + br[i] * ur[i];
      gyb[i] = kbar * gain[i];
      a[i] = env_div(gyb[i] * (k.dgu - 1.f), g[i] + COMP_EPS);
      dT += gyb[i] * k.dt;
      dW += gyb[i] * k.dw;
      dR += gyb[i] * k.dr;
    }
    // reverse scan lambda[n] = a[n] + alpha lambda[n+1]
    float lb = 0.f;
#pragma unroll
    for (int i = SPT - 1; i >= 0; --i) lb = a[i] + alpha * lb;
    __syncthreads();  // sh reuse
    float rtotal;
    float rexcl = block_affine_scan<true>(lb, la * SPT, sh, &rtotal);
    if (threadIdx.x < 32) {
      // aggregate words by the chunk's partial slot: a node's chunks are contiguous there,
      // from its last chunk, whatever the order of the tickets
      const int fidx = item0 + (w.w - slot0);
      if (threadIdx.x == 0) publish(c, fidx, 1, rtotal);
      const float lin = chunk == n_chunks - 1 ? 0.f
                                              : carry_sum_warp(c, fidx - 1, fidx - (n_chunks - 1 - chunk), la * CH);
      if (threadIdx.x == 0) s_lin = lin;
    }
    glast[threadIdx.x] = g[SPT - 1];
    __syncthreads();
    // state entering this thread from the right: within-chunk part + the chunk carry
    const float lin_t = rexcl + expf(la * float(SPT * (255 - threadIdx.x))) * s_lin;
    float lam[SPT];
    {
      float s = lin_t;
#pragma unroll
      for (int i = SPT - 1; i >= 0; --i) {
        s = a[i] + alpha * s;
        lam[i] = s;
      }
    }
    float gprev = threadIdx.x > 0 ? glast[threadIdx.x - 1] : carry_g;
    float dA = 0.f;
    if constexpr (SC) {
      // input 0 (main): gain ybar; input 1 (key): 2 (k_l + k_r)(1 - alpha) lambda on both channels
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        dA += lam[i] * (gprev - x[i]);
        gprev = g[i];
        bl[i] *= gain[i];
        br[i] *= gain[i];
        km[i] = 2.f * km[i] * (1.f - alpha) * lam[i];
      }
      store_chunk<SPT>(arow_w(c, nd), nd, t, bl, br);
      store_chunk<SPT>(arow_w(c, nd) + nd.rstride, nd, t, km, km);
    } else {
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        dA += lam[i] * (gprev - x[i]);
        gprev = g[i];
        float xb2 = 2.f * (ul[i] + ur[i]) * (1.f - alpha) * lam[i];
        bl[i] = gain[i] * bl[i] + xb2;
        br[i] = gain[i] * br[i] + xb2;
      }
      store_chunk<SPT>(arow_w(c, nd), nd, t, bl, br);
    }
    float acc[4] = {dA, dT, dW, dR};
    block_sum<4>(acc, red);
    if (threadIdx.x == 0) c.partial[w.w] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    __syncthreads();
    it = next;
    slot ^= 1;
  }
  cp_async_wait_all();
}

__global__ void k_comp_finalize(DevCtx c, int node_begin, int node_end) {
  int v = node_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= node_end) return;
  const int4_ e = c.ext[v];
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < e.y; ++k) {
    float4 q = c.partial[e.x + k];
    s.x += q.x; s.y += q.y; s.z += q.z; s.w += q.w;
  }
  float* d = c.dparams + c.nodes[v].grow * 4;
  d[0] = s.x; d[1] = s.y; d[2] = s.z; d[3] = s.w;
}

// what: 0 forward (items [a, a + b), nodes [n0, n1)), 1 backward (the same), 2 finalize
// (nodes [n0, n1)); mode: MODE_COMP, MODE_GATE (the noisegate curve of Eq. 13) or MODE_SC
// (the sidechain compressor).  Returns the number of kernels launched.
template <int SPT, int MODE>
static int comp_launch(int what, const DevCtx& c, int a, int b, int ticket, cudaStream_t s) {
  constexpr int CH = 256 * SPT;
  constexpr int fwd_smem = 2 * CH * sizeof(float), bwd_smem = 4 * CH * sizeof(float);
  static bool init = false;
  if (!init) {   // first call (also the attributes-only call made before a stream capture)
    cudaFuncSetAttribute(k_comp_bwd_lb<SPT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bwd_smem);
    cudaFuncSetAttribute(k_comp_fwd_lb<SPT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd_smem);
    init = true;
  }
  if (what < 0 || b <= 0) return 0;
  // the step's look-back words and its ticket start at zero
  cudaMemsetAsync(c.flags + a, 0, sizeof(unsigned long long) * size_t(b), s);
  cudaMemsetAsync(c.tickets + ticket, 0, sizeof(int32_t), s);
  if (what == 0) k_comp_fwd_lb<SPT, MODE><<<grid_size(b, 4), 256, fwd_smem, s>>>(c, a, b, ticket);
  else k_comp_bwd_lb<SPT, MODE><<<grid_size(b, 4), 256, bwd_smem, s>>>(c, a, b, ticket);
  return 1;
}

template <int SPT>
static int comp_mode(int what, const DevCtx& c, int a, int b, int ticket, int mode, cudaStream_t s) {
  if (mode == MODE_GATE) return comp_launch<SPT, MODE_GATE>(what, c, a, b, ticket, s);
  if (mode == MODE_SC) return comp_launch<SPT, MODE_SC>(what, c, a, b, ticket, s);
  return comp_launch<SPT, MODE_COMP>(what, c, a, b, ticket, s);
}

int launch_comp(int what, const DevCtx& c, int a, int b, int n0, int n1, int ticket, int mode, cudaStream_t s) {
  if (what < 0) {   // kernel attributes of every variant
    for (int m : {MODE_COMP, MODE_GATE, MODE_SC}) {
      comp_mode<4>(-1, c, 0, 0, 0, m, s);
      comp_mode<8>(-1, c, 0, 0, 0, m, s);
      comp_mode<16>(-1, c, 0, 0, 0, m, s);
    }
    return 0;
  }
  if (what == 2) {
    if (n1 <= n0) return 0;
    k_comp_finalize<<<(n1 - n0 + 127) / 128, 128, 0, s>>>(c, n0, n1);
    return 1;
  }
  if (b <= 0) return 0;
  if (c.comp_chunk == 1024) return comp_mode<4>(what, c, a, b, ticket, mode, s);
  if (c.comp_chunk == 4096) return comp_mode<16>(what, c, a, b, ticket, mode, s);
  return comp_mode<8>(what, c, a, b, ticket, mode, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the compressor forward pass, for callers that may not
// allocate device memory (see grafx_compressor_forward_noalloc in grafx.h).  Its only
// scratch, the look-back words of the chunks plus a ticket and a status word, lives in
// this file-scope device array, sized for signals of up to NOALLOC_MAX_LEN samples.
// Every GPU that loads the library keeps the array until the process exits.
constexpr int NOALLOC_CHUNK = 2048;                              // samples per chunk (SPT = 8)
constexpr int NOALLOC_MAX_LEN = 1 << 22;                         // samples per channel
constexpr int NOALLOC_MAX_CHUNKS = NOALLOC_MAX_LEN / NOALLOC_CHUNK;
constexpr int NOALLOC_WORDS = NOALLOC_MAX_CHUNKS + 32;           // + ticket / status words
static __device__ __align__(256) unsigned long long g_comp_noalloc_scratch[NOALLOC_WORDS];

// One stereo row u[2][pitch] -> y[2][pitch]; same chunk arithmetic as k_comp_fwd_lb<8>,
// with the row read directly instead of gathered over in-edges.
__global__ void __launch_bounds__(256) k_comp_fwd_row(DevCtx c, const float* __restrict__ u, const float* p,
                                                     float* y, int len, int pitch, int n_chunks) {
  constexpr int SPT = 8, CH = 256 * SPT;
  __shared__ float sh[32];
  __shared__ int s_it;
  __shared__ float s_carry;
  const float alpha = p[0];
  const KneeCoef kq = knee_coef(p[1], p[2], p[3]);
  const float la = logf(alpha);
  while (true) {
    if (threadIdx.x == 0) s_it = atomicAdd(c.tickets, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= n_chunks) break;
    const int t = it * CH + threadIdx.x * SPT;
    float ul[SPT], ur[SPT], x[SPT], g[SPT];
#pragma unroll
    for (int q = 0; q < SPT / 4; ++q) {
      float4 l = f4zero(), r = f4zero();
      if (t + 4 * q < len) {
        l = mask4(ld4(u + t + 4 * q), t + 4 * q, len);
        r = mask4(ld4(u + pitch + t + 4 * q), t + 4 * q, len);
      }
      ul[4 * q + 0] = l.x; ul[4 * q + 1] = l.y; ul[4 * q + 2] = l.z; ul[4 * q + 3] = l.w;
      ur[4 * q + 0] = r.x; ur[4 * q + 1] = r.y; ur[4 * q + 2] = r.z; ur[4 * q + 3] = r.w;
    }
#pragma unroll
    for (int i = 0; i < SPT; ++i) { float m = ul[i] + ur[i]; x[i] = m * m; }
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < SPT; ++i) b = alpha * b + (1.f - alpha) * x[i];
    float total;
    float excl = block_affine_scan<false>(b, la * SPT, sh, &total);
    if (threadIdx.x < 32) {
      float carry = 0.f;
      if (it == 0) {
        if (threadIdx.x == 0) publish(c, it, 2, total);
      } else {
        if (threadIdx.x == 0) publish(c, it, 1, total);
        carry = look_back_warp(c, it - 1, 0, la * CH);
        if (threadIdx.x == 0) publish(c, it, 2, expf(la * CH) * carry + total);
      }
      if (threadIdx.x == 0) s_carry = carry;
    }
    __syncthreads();
    const float cin = excl + expf(la * float(SPT * threadIdx.x)) * s_carry;
    envelope<SPT>(x, alpha, cin, g);
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      float gu = ln_env(g[i]);
      Knee k = knee(gu, kq);
      float gain = exp_gain(k.gy - gu);
      ul[i] *= gain;
      ur[i] *= gain;
    }
#pragma unroll
    for (int q = 0; q < SPT / 4; ++q) {
      if (t + 4 * q < pitch) {
        st4(y + t + 4 * q, make_float4(ul[4 * q], ul[4 * q + 1], ul[4 * q + 2], ul[4 * q + 3]));
        st4(y + pitch + t + 4 * q, make_float4(ur[4 * q], ur[4 * q + 1], ur[4 * q + 2], ur[4 * q + 3]));
      }
    }
    __syncthreads();
  }
  // padding past the last chunk (pitch may exceed n_chunks * CH): zeros, both channels
  for (int64_t t = int64_t(n_chunks) * CH + 4 * (int64_t(blockIdx.x) * blockDim.x + threadIdx.x); t < pitch;
       t += 4 * int64_t(gridDim.x) * blockDim.x) {
    st4(y + t, f4zero());
    st4(y + pitch + t, f4zero());
  }
}

}  // namespace grafx

extern "C" int grafx_compressor_forward_noalloc(const float* u, int64_t len, int64_t pitch, const float* params,
                                                float* y, uint32_t* status, void* stream) {
  using namespace grafx;
  if (!u || !params || !y) return fail(GRAFX_EINVAL, "null argument");
  if (len < 1 || len > NOALLOC_MAX_LEN)
    return fail(GRAFX_ESHAPE, "grafx_compressor_forward_noalloc: length must be in [1, 4194304] samples, the "
                              "size of its fixed scratch");
  if (pitch < len || pitch % 4 || pitch > (int64_t(1) << 30))
    return fail(GRAFX_ESHAPE, "pitch must be >= length and a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(y)) % 16)
    return fail(GRAFX_EINVAL, "signal rows must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(status) % 4) return fail(GRAFX_EINVAL, "status word must be 4-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return fail(GRAFX_EINVAL, "device ordinal out of range");
  // The context's id (unique for the life of the process) keys the cached address, so a
  // context destroyed and re-created on this device (cudaDeviceReset) gets a fresh lookup.
  using CtxGetId = int (*)(void*, unsigned long long*);
  static CtxGetId ctx_get_id = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<CtxGetId>(fn);
  }();
  if (!ctx_get_id) return fail(GRAFX_ECUDA, "cuCtxGetId is not available from the driver");
  e = cudaSetDevice(dev);  // initialises the device's primary context if nothing has yet
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  unsigned long long ctx = 0;
  if (ctx_get_id(nullptr, &ctx) != 0) return fail(GRAFX_ECUDA, "cuCtxGetId failed");
  // Set-up, once per device (and again only after its context was re-created), with that
  // device current: the device address of the scratch array (in host code its name only
  // stands for it).
  static std::mutex mu;
  static unsigned long long* addr[128] = {nullptr};
  static unsigned long long addr_ctx[128] = {0};
  unsigned long long* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || addr_ctx[dev] != ctx) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_comp_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(GRAFX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      addr[dev] = static_cast<unsigned long long*>(ptr);
      addr_ctx[dev] = ctx;
    }
    scratch = addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_chunks = int((len + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
  // look-back words of this call's chunks, the ticket and the internal status start at zero
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * n_chunks, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + NOALLOC_MAX_CHUNKS, 0, 16, s);
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, std::string("clear scratch: ") + cudaGetErrorString(e));
  DevCtx c;
  std::memset(&c, 0, sizeof(c));
  c.flags = scratch;
  c.tickets = reinterpret_cast<int32_t*>(scratch + NOALLOC_MAX_CHUNKS);
  c.status = status ? status : reinterpret_cast<uint32_t*>(scratch + NOALLOC_MAX_CHUNKS + 1);
  const int g = grid_size(n_chunks, 8);
  k_comp_fwd_row<<<g, 256, 0, s>>>(c, u, params, y, int(len), int(pitch), n_chunks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return GRAFX_OK;
}

// Failure-detection self-test of the bounded look-back wait: one warp polls *flag at most
// `limit` times.  A flag that nothing sets makes the wait expire: ST_TIMEOUT is OR-ed into
// *status and *value = 0; a flag already set to (2 << 32 | bits of v) gives *value = v.
extern "C" int grafx_selftest_bounded_wait(const unsigned long long* flag, uint32_t* status, int32_t limit,
                                           float* value, void* stream) {
  using namespace grafx;
  if (!flag || !status || !value) return fail(GRAFX_EINVAL, "null argument");
  if (limit < 1 || limit > SPIN_LIMIT) return fail(GRAFX_EINVAL, "limit out of range");
  k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(flag, status, limit, value);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRAFX_OK : fail(GRAFX_ECUDA, cudaGetErrorString(e));
}
