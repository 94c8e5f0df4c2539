// Compressor with attack/release ballistics (Sec. 3, Eq. 8 with alpha[n] = alpha_attack
// while the envelope rises, x[n] > g[n-1], and alpha_release while it falls; Eq. 9-12 for
// the rest).  The coefficient depends on the state, so the recursion is not a linear
// scan; it is a composition of max (or min) of two affine maps, which stays a max of
// affine maps over a chunk: the forward composes 64-sample chunks in parallel, walks the
// chunk starts serially (one reduction per chunk) and re-runs every chunk from its start
// in parallel.  Everything else is per sample and runs as tiles over all nodes:
//   forward:  k_bal_mid (u -> the mid m = l + r into scratch), k_bal_maps, k_bal_starts
//             and k_bal_run (g by chunk maps, below), k_bal_gain (gain from g, y = gain u);
//   backward: k_bal_adj (ybar, u, g -> the main adjoint gain ybar, the envelope adjoint
//             a[n] = dL/dg[n], the coefficient alpha[n] of each step and the T, W, R
//             partials per tile), k_bal_rev (lambda[n] = a[n] + alpha[n+1] lambda[n+1] in
//             place, a warp scan of affine maps), k_bal_in (adds
//             2 m (1 - alpha[n]) lambda[n] to both channels' adjoint; the attack and
//             release gradient partials per tile), k_bal_fin (parameter gradients).
// Per node the scratch holds four rows of pitch floats (rounded up to 64): the mid, the
// envelope, the envelope adjoint and the per-step coefficient.  Backward tiles own two
// partial slots (T, W, R and attack, release).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace grafx {

constexpr float BAL_EPS = 1e-7f;
constexpr int BAL_BLOCK = 512;   // samples per block of the reverse scan

__device__ __forceinline__ int bal_rs(const NodeDev& nd) { return (nd.pitch + 63) & ~63; }
__device__ __forceinline__ float* bal_row(const DevCtx& c, int v, const NodeDev& nd, int i) {
  return c.bal + 64 * int64_t(c.ext[v].w) + int64_t(i) * bal_rs(nd);
}

// The compressor's curve (Eq. 10-11) with its partials dGy/dGu, dT, dW, dR.
struct BalKnee {
  float gy, dgu, dt, dw, dr;
};
__device__ __forceinline__ BalKnee bal_knee(float gu, float T, float W, float R) {
  BalKnee k;
  const float invR = 1.f / R, cR = invR - 1.f;
  if (gu >= T + W) {
    k.gy = T + (gu - T) * invR;
    k.dgu = invR;
    k.dt = -cR;
    k.dw = 0.f;
    k.dr = -(gu - T) * invR * invR;
  } else if (gu >= T - W) {
    const float d = gu - T + W;
    k.gy = gu + cR * d * d / (4.f * W);
    k.dgu = 1.f + cR * d / (2.f * W);
    k.dt = -cR * d / (2.f * W);
    k.dw = cR * (d / (2.f * W) - d * d / (4.f * W * W));
    k.dr = -d * d / (4.f * W) * invR * invR;
  } else {
    k.gy = gu;
    k.dgu = 1.f;
    k.dt = k.dw = k.dr = 0.f;
  }
  return k;
}

// forward, per tile: m = l + r of the gathered input
__global__ void __launch_bounds__(256) k_bal_mid(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    float* X = bal_row(c, v, nd, 0);
    for (int t = w.y + 4 * threadIdx.x; t < min(w.y + EW_TILE, nd.pitch); t += 1024) {
      const float4 l = gather_in(c, v, 0, t, nd.len, nd.pitch), r = gather_in(c, v, 1, t, nd.len, nd.pitch);
      st4(X + t, f4add(l, r));
    }
  }
}

// The envelope recursion in parallel.  With the larger candidate taken when the attack
// is the faster coefficient (the smaller one otherwise; the two candidate steps meet at
// x, so this is the branch of Eq. 8), one step is the map
//   F_t(g) = OP(aa g + (1 - aa) x_t, ar g + (1 - ar) x_t),  OP = max (aa <= ar) or min,
// and since both slopes are positive, a chunk of n steps composes to
//   F(g) = OP_k (s_k g + c_k),  s_k = aa^k ar^(n-k),  k = number of attack steps,
// with c_k the OP over the paths with k attacks of their intercepts, found by the
// dynamic programme c'_k = OP(aa c_{k-1} + (1-aa) x, ar c_k + (1-ar) x) (c_0 = 0 and the
// others +-inf at the start).  The forward runs in three kernels: the programme for every
// BAL_N-sample chunk (one warp per chunk), the chunk starts g_in (one warp per node,
// serial over chunks, OP of the lines by a warp reduction), and the recursion inside
// every chunk from its start (one thread per chunk).
constexpr int BAL_N = 64;                  // samples per chunk
constexpr int BAL_L = BAL_N + 1;           // lines per chunk map
__device__ __forceinline__ int bal_chunks(const NodeDev& nd) { return (nd.len + BAL_N - 1) / BAL_N; }
// chunk maps (intercepts, BAL_L per chunk) then the chunk starts, in the node's adjoint
// and coefficient rows (free during the forward): 66 floats per chunk <= 2 rows
__device__ __forceinline__ float* bal_maps(const DevCtx& c, int v, const NodeDev& nd) { return bal_row(c, v, nd, 2); }
__device__ __forceinline__ float* bal_starts(const DevCtx& c, int v, const NodeDev& nd) {
  return bal_row(c, v, nd, 2) + size_t(BAL_L) * bal_chunks(nd);
}

template <bool MAX>
__device__ __forceinline__ float bal_op(float a, float b) { return MAX ? fmaxf(a, b) : fminf(a, b); }

// forward 1: the chunk maps, one chunk per half-warp.  Lane h (0..15) of a half holds
// c_4h .. c_4h+3; the attack step into c_4h comes from lane h-1.  c_64 (64 attacks in
// 64 steps) has a single path, so it is the plain sum over t of aa^(63-t) (1-aa) x_t,
// formed after the programme by the half's lanes and a shuffle reduction.  Samples past
// len are taken as 0 (only the last chunk has them, and its map is not used).
template <bool MAX>
__device__ void bal_chunk_map(const DevCtx& c, int v, const NodeDev& nd, int ck, float aa, float ar, float* xs,
                              bool store) {
  const int h = threadIdx.x & 15;
  const float* X = bal_row(c, v, nd, 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = ck * BAL_N + h + 16 * i;
    const float m = t < nd.len ? X[t] : 0.f;
    xs[h + 16 * i] = m * m;
  }
  __syncwarp();
  const float unreach = MAX ? -INFINITY : INFINITY;
  const float ba = 1.f - aa, br = 1.f - ar;
  float c0 = h == 0 ? 0.f : unreach, c1 = unreach, c2 = unreach, c3 = unreach;
  for (int t = 0; t < BAL_N; ++t) {
    const float x = xs[t];
    const float ax = ba * x, rx = br * x;
    float lo = __shfl_up_sync(0xffffffffu, c3, 1, 16);   // c_{4h-1}
    if (h == 0) lo = unreach;
    const float n0 = bal_op<MAX>(fmaf(aa, lo, ax), fmaf(ar, c0, rx));
    const float n1 = bal_op<MAX>(fmaf(aa, c0, ax), fmaf(ar, c1, rx));
    const float n2 = bal_op<MAX>(fmaf(aa, c1, ax), fmaf(ar, c2, rx));
    const float n3 = bal_op<MAX>(fmaf(aa, c2, ax), fmaf(ar, c3, rx));
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  float all = 0.f;   // c_64: sum_t aa^(63-t) (1-aa) x_t over the lane's 4 samples
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = h + 16 * i;
    all += powf(aa, float(BAL_N - 1 - t)) * (ba * xs[t]);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) all += __shfl_xor_sync(0xffffffffu, all, o, 16);
  if (!store) return;
  float* out = bal_maps(c, v, nd) + size_t(ck) * BAL_L;
  out[4 * h] = c0;
  out[4 * h + 1] = c1;
  out[4 * h + 2] = c2;
  out[4 * h + 3] = c3;
  if (h == 0) out[BAL_N] = all;
}

// grid (ceil(max chunks / 16), ballistic nodes of the step), 8 warps: one chunk per half
__global__ void __launch_bounds__(256) k_bal_maps(DevCtx c, int node_begin) {
  __shared__ float xs[16][BAL_N];
  const int v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int half = threadIdx.x >> 4;
  const int ck = blockIdx.x * 16 + half;
  // both halves of a warp take part in its shuffles: a half past the last chunk runs on
  // a copy of the last chunk and does not store
  const int nck = bal_chunks(nd);
  const float* p = c.params + size_t(nd.prow) * 5;
  const float aa = p[0], ar = p[1];
  if ((blockIdx.x * 16 + (half & ~1)) >= nck) return;   // whole warps leave together
  const int cr = min(ck, nck - 1);
  if (aa <= ar) bal_chunk_map<true>(c, v, nd, cr, aa, ar, xs[half], ck < nck);
  else bal_chunk_map<false>(c, v, nd, cr, aa, ar, xs[half], ck < nck);
}

// forward 2: one warp per node, serial over chunks: g_in of chunk 0 is 0, then
// g_in(c+1) = OP_k (s_k g_in(c) + c_k(c)); every line value is >= 0 (or unreachable), so
// the warp's OP reduces the float bit patterns as unsigned integers.  The slopes are
// formed once in double.  The chunk maps stream through shared memory in batches of
// BAL_BB chunks, a ring of BAL_ST batches in flight (cp.async), so the serial chain waits
// on shared-memory loads only.
constexpr int BAL_BB = 32, BAL_ST = 3;

template <bool MAX>
__device__ void bal_chunk_starts(const DevCtx& c, int v, const NodeDev& nd, float aa, float ar, float (*sm)[BAL_BB * BAL_L]) {
  const int lane = threadIdx.x;
  const int nck = bal_chunks(nd), nbat = (nck + BAL_BB - 1) / BAL_BB;
  const float* maps = bal_maps(c, v, nd);
  float* starts = bal_starts(c, v, nd);
  float sl[3];
  const int ks[3] = {2 * lane, 2 * lane + 1, BAL_N};
#pragma unroll
  for (int i = 0; i < 3; ++i) sl[i] = float(pow(double(aa), ks[i]) * pow(double(ar), BAL_N - ks[i]));
  const float unreach = MAX ? -INFINITY : INFINITY;
  auto issue = [&](int b) {   // batch b's maps (chunks past the last read as nothing)
    if (b < nbat) {
      const int nfl = min(BAL_BB, nck - b * BAL_BB) * BAL_L;   // floats that exist
      const float* src = maps + size_t(b) * BAL_BB * BAL_L;   // 16-byte aligned: 32 x 65 x 4 B
      float* dst = sm[b % BAL_ST];
      for (int i = lane; i < BAL_BB * BAL_L / 4; i += 32) {
        const int n = max(0, min(4, nfl - 4 * i));
        cp_async16(dst + 4 * i, n ? src + 4 * i : src, 4 * n);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int b = 0; b < BAL_ST - 1; ++b) issue(b);
  float g = 0.f;
  for (int b = 0; b < nbat; ++b) {
    issue(b + BAL_ST - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(BAL_ST - 1) : "memory");   // batch b landed
    __syncwarp();
    const float* m = sm[b % BAL_ST];
    const int nj = min(BAL_BB, nck - b * BAL_BB);
#pragma unroll 4
    for (int j = 0; j < nj; ++j) {
      const int ck = b * BAL_BB + j;
      if (lane == 0) starts[ck] = g;
      if (ck + 1 == nck) break;
      const float* mj = m + j * BAL_L;
      const float c0 = mj[2 * lane], c1 = mj[2 * lane + 1], c2 = lane == 31 ? mj[BAL_N] : unreach;
      float best = bal_op<MAX>(fmaf(sl[0], g, c0), fmaf(sl[1], g, c1));
      best = bal_op<MAX>(best, fmaf(sl[2], g, c2));
      const unsigned u = __float_as_uint(MAX ? fmaxf(best, 0.f) : best);
      g = __uint_as_float(MAX ? __reduce_max_sync(0xffffffffu, u) : __reduce_min_sync(0xffffffffu, u));
    }
    __syncwarp();   // every lane is done with this stage before it is staged again
  }
  cp_async_wait_all();
}

__global__ void __launch_bounds__(32) k_bal_starts(DevCtx c, int node_begin) {
  __shared__ __align__(16) float sm[BAL_ST][BAL_BB * BAL_L];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  const float* p = c.params + size_t(nd.prow) * 5;
  const float aa = p[0], ar = p[1];
  if (aa <= ar) bal_chunk_starts<true>(c, v, nd, aa, ar, sm);
  else bal_chunk_starts<false>(c, v, nd, aa, ar, sm);
}

// forward 3: one thread per chunk: the recursion of Eq. 8 over the chunk's samples from
// its start, written to the envelope row.  grid (ceil(max chunks / 128), nodes), 128
// threads.
template <bool MAX>
__device__ void bal_chunk_run(const DevCtx& c, int v, const NodeDev& nd, int ck, float aa, float ar) {
  const float* X = bal_row(c, v, nd, 0);
  float* G = bal_row(c, v, nd, 1);
  const float ba = 1.f - aa, br = 1.f - ar;
  float g = bal_starts(c, v, nd)[ck];
  const int t0 = ck * BAL_N, n = min(BAL_N, nd.len - t0);
  for (int q = 0; q < BAL_N / 4; ++q) {
    if (4 * q >= n) break;
    const float4 m4 = ld4(X + t0 + 4 * q);   // rows are 64-float aligned; X is 0 past len
    const float m[4] = {m4.x, m4.y, m4.z, m4.w};
    float o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float x = m[j] * m[j];
      g = bal_op<MAX>(fmaf(aa, g, ba * x), fmaf(ar, g, br * x));
      o[j] = g;
    }
    st4(G + t0 + 4 * q, make_float4(o[0], o[1], o[2], o[3]));
  }
}

__global__ void __launch_bounds__(128) k_bal_run(DevCtx c, int node_begin) {
  const int v = node_begin + blockIdx.y;
  const NodeDev nd = c.nodes[v];
  const int ck = blockIdx.x * 128 + threadIdx.x;
  if (ck >= bal_chunks(nd)) return;
  const float* p = c.params + size_t(nd.prow) * 5;
  const float aa = p[0], ar = p[1];
  if (aa <= ar) bal_chunk_run<true>(c, v, nd, ck, aa, ar);
  else bal_chunk_run<false>(c, v, nd, ck, aa, ar);
}

// forward, per tile: y = exp(Gy - Gu) u with Gu = ln(g + eps)
__global__ void __launch_bounds__(256) k_bal_gain(DevCtx c, int item0, int n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const float* p = c.params + size_t(nd.prow) * 5;
    const float T = p[2], W = p[3], R = p[4];
    const float* G = bal_row(c, v, nd, 1);
    float* y = yrow_w(c, nd);
    for (int t = w.y + 4 * threadIdx.x; t < min(w.y + EW_TILE, nd.pitch); t += 1024) {
      float4 l = gather_in(c, v, 0, t, nd.len, nd.pitch), r = gather_in(c, v, 1, t, nd.len, nd.pitch);
      float gain[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float g = t + q < nd.len ? G[t + q] : 0.f;
        const float gu = logf(g + BAL_EPS);
        gain[q] = expf(bal_knee(gu, T, W, R).gy - gu);
      }
      l = make_float4(gain[0] * l.x, gain[1] * l.y, gain[2] * l.z, gain[3] * l.w);
      r = make_float4(gain[0] * r.x, gain[1] * r.y, gain[2] * r.z, gain[3] * r.w);
      st4(y + t, l);
      st4(y + nd.pitch + t, r);
    }
  }
}

// backward, per tile: main adjoint gain ybar into the node's adjoint row, the envelope
// adjoint a[n] = (sum_ch ybar u) gain (dGy/dGu - 1) / (g + eps), and the tile's T, W, R partials
__global__ void __launch_bounds__(256) k_bal_adj(DevCtx c, int item0, int n_items) {
  __shared__ float red[4 * 32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const float* p = c.params + size_t(nd.prow) * 5;
    const float T = p[2], W = p[3], R = p[4];
    const float aa = p[0], ar = p[1];
    const float* X = bal_row(c, v, nd, 0);
    const float* G = bal_row(c, v, nd, 1);
    float* A = bal_row(c, v, nd, 2);
    float* AL = bal_row(c, v, nd, 3);
    float* ub = arow_w(c, nd);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int t = w.y + 4 * threadIdx.x; t < min(w.y + EW_TILE, nd.pitch); t += 1024) {
      const float4 ul = gather_in(c, v, 0, t, nd.len, nd.pitch), ur = gather_in(c, v, 1, t, nd.len, nd.pitch);
      float4 bl = gather_out_adj(c, v, 0, t, nd.len, nd.pitch), br = gather_out_adj(c, v, 1, t, nd.len, nd.pitch);
      const float uL[4] = {ul.x, ul.y, ul.z, ul.w}, uR[4] = {ur.x, ur.y, ur.z, ur.w};
      float bL[4] = {bl.x, bl.y, bl.z, bl.w}, bR[4] = {br.x, br.y, br.z, br.w}, a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float g = t + q < nd.len ? G[t + q] : 0.f;
        const float gu = logf(g + BAL_EPS);
        const BalKnee k = bal_knee(gu, T, W, R);
        const float gain = expf(k.gy - gu);
        const float gyb = (bL[q] * uL[q] + bR[q] * uR[q]) * gain;
        a[q] = gyb * (k.dgu - 1.f) / (g + BAL_EPS);
        acc[0] += gyb * k.dt;
        acc[1] += gyb * k.dw;
        acc[2] += gyb * k.dr;
        bL[q] *= gain;
        bR[q] *= gain;
      }
      st4(A + t, make_float4(a[0], a[1], a[2], a[3]));
      float al[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // the coefficient of step t + q (by the branch of Eq. 8)
        const float m = t + q < nd.len ? X[t + q] : 0.f, gp = t + q > 0 && t + q <= nd.len ? G[t + q - 1] : 0.f;
        al[q] = m * m > gp ? aa : ar;
      }
      st4(AL + t, make_float4(al[0], al[1], al[2], al[3]));
      st4(ub + t, make_float4(bL[0], bL[1], bL[2], bL[3]));
      st4(ub + nd.pitch + t, make_float4(bR[0], bR[1], bR[2], bR[3]));
    }
    block_sum<3>(acc, red);
    if (threadIdx.x == 0) c.partial[w.w] = make_float4(acc[0], acc[1], acc[2], 0.f);
    __syncthreads();
  }
}

// backward, per node from the end: lambda[n] = a[n] + alpha[n+1] lambda[n+1], in place of
// a.  With alpha[n] known per sample the recursion is linear, so it runs as a warp scan:
// lane l owns 16 samples of each 512-sample block; with mu[n] = alpha[n] lambda[n] (the
// term handed to step n-1), a lane's segment maps its end value to its start value,
// mu_s = C + Q mu_e; the maps compose across lanes by a shuffle scan from the right, the
// block's carry enters at lane 31, and a second pass over the segment writes lambda.
__global__ void __launch_bounds__(32) k_bal_rev(DevCtx c, int node_begin) {
  constexpr int SEG = BAL_BLOCK / 32, SQ = SEG / 4;
  constexpr int ST = 4;          // blocks in flight: a ring of cp.async stages
  constexpr int LP = SEG + 4;    // floats per lane in a stage (padded: conflict-free float4 reads)
  __shared__ __align__(16) float ring[ST][2][32 * LP];
  const int v = node_begin + blockIdx.x;
  const NodeDev nd = c.nodes[v];
  float* A = bal_row(c, v, nd, 2);
  const float* AL = bal_row(c, v, nd, 3);
  const int nb = (nd.len + BAL_BLOCK - 1) / BAL_BLOCK;
  const int lane = threadIdx.x;
  // each lane copies (and later reads) only its own 16 samples of a and alpha; quads at
  // or past len are zero-filled without a read (a straddling quad's tail is 0 in a)
  auto issue = [&](int b) {
    if (b >= 0) {
      float* da = ring[b % ST][0] + LP * lane;
      float* dl = ring[b % ST][1] + LP * lane;
#pragma unroll
      for (int j = 0; j < SQ; ++j) {
        const int t = b * BAL_BLOCK + SEG * lane + 4 * j;
        const bool in = t < nd.len;
        cp_async16(da + 4 * j, in ? A + t : A, in ? 16 : 0);
        cp_async16(dl + 4 * j, in ? AL + t : AL, in ? 16 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 1; k < ST; ++k) issue(nb - k);
  float mu_in = 0.f;   // mu at the end of the block (0 past the end of the signal)
  for (int b = nb - 1; b >= 0; --b) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(ST - 2) : "memory");   // block b landed
    float a[SEG], al[SEG];
    const float4* ra = reinterpret_cast<const float4*>(ring[b % ST][0] + LP * lane);
    const float4* rl = reinterpret_cast<const float4*>(ring[b % ST][1] + LP * lane);
#pragma unroll
    for (int j = 0; j < SQ; ++j) {
      const float4 x = ra[j], y = rl[j];
      a[4 * j] = x.x, a[4 * j + 1] = x.y, a[4 * j + 2] = x.z, a[4 * j + 3] = x.w;
      al[4 * j] = y.x, al[4 * j + 1] = y.y, al[4 * j + 2] = y.z, al[4 * j + 3] = y.w;
    }
    issue(b - (ST - 1));   // into the stage block b + 1 used
    float C = 0.f, Q = 1.f;
#pragma unroll
    for (int j = SEG - 1; j >= 0; --j) {
      C = al[j] * (a[j] + C);
      Q *= al[j];
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {   // lane l: the map of segments l..31
      const float C2 = __shfl_down_sync(0xffffffffu, C, d), Q2 = __shfl_down_sync(0xffffffffu, Q, d);
      if (lane + d < 32) {
        C = fmaf(Q, C2, C);
        Q *= Q2;
      }
    }
    const float mu_s = fmaf(Q, mu_in, C);   // mu at the start of this lane's segment
    float mu = __shfl_down_sync(0xffffffffu, mu_s, 1);
    if (lane == 31) mu = mu_in;
#pragma unroll
    for (int j = SEG - 1; j >= 0; --j) {
      a[j] += mu;
      mu = al[j] * a[j];
    }
#pragma unroll
    for (int j = 0; j < SQ; ++j) {
      const int t = b * BAL_BLOCK + SEG * lane + 4 * j;
      if (t < nd.len) st4(A + t, make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]));
    }
    mu_in = __shfl_sync(0xffffffffu, mu_s, 0);
  }
  cp_async_wait_all();
}

// backward, per tile: adds 2 m (1 - alpha[n]) lambda[n] to both channels of the adjoint,
// and the tile's sums of lambda[n] (g[n-1] - x[n]) over attack and release steps
__global__ void __launch_bounds__(256) k_bal_in(DevCtx c, int item0, int n_items) {
  __shared__ float red[4 * 32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4_ w = c.items[item0 + it];
    const int v = w.x;
    const NodeDev nd = c.nodes[v];
    const float* p = c.params + size_t(nd.prow) * 5;
    const float aa = p[0], ar = p[1];
    const float* X = bal_row(c, v, nd, 0);
    const float* G = bal_row(c, v, nd, 1);
    const float* L = bal_row(c, v, nd, 2);
    float* ub = arow_w(c, nd);
    float acc[2] = {0.f, 0.f};
    for (int t = w.y + threadIdx.x; t < min(w.y + EW_TILE, nd.len); t += 256) {
      const float m = X[t], x = m * m, gp = t > 0 ? G[t - 1] : 0.f, lam = L[t];
      const bool att = x > gp;   // the branch the forward took (same fp32 operands)
      const float e = 2.f * m * (1.f - (att ? aa : ar)) * lam;
      ub[t] += e;
      ub[nd.pitch + t] += e;
      const float d = lam * (gp - x);
      acc[0] += att ? d : 0.f;
      acc[1] += att ? 0.f : d;
    }
    block_sum<2>(acc, red);
    if (threadIdx.x == 0) c.partial[w.w + 1] = make_float4(acc[0], acc[1], 0.f, 0.f);
    __syncthreads();
  }
}

// parameter gradients [alpha_attack, alpha_release, T, W, R] of a node range
__global__ void k_bal_fin(DevCtx c, int node_begin, int node_end) {
  const int v = node_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= node_end) return;
  const int4_ e = c.ext[v];
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < e.y; ++k) {   // two slots per tile: (T, W, R), (attack, release)
    const float4 q = c.partial[e.x + 2 * k], r = c.partial[e.x + 2 * k + 1];
    s[0] += r.x;
    s[1] += r.y;
    s[2] += q.x;
    s[3] += q.y;
    s[4] += q.z;
  }
  float* d = c.dparams + size_t(c.nodes[v].grow) * 5;
  for (int i = 0; i < 5; ++i) d[i] = s[i];
}

int launch_bal_fwd(const DevCtx& c, int item0, int n_items, int node_begin, int node_end, cudaStream_t s) {
  if (n_items <= 0 || node_end <= node_begin) return 0;
  const int g = grid_size(n_items, 8);
  k_bal_mid<<<g, 256, 0, s>>>(c, item0, n_items);
  const int mck = (c.bal_maxlen + BAL_N - 1) / BAL_N;
  int launches = 2;
  for (int n0 = node_begin; n0 < node_end; n0 += 65535) {   // nodes on grid.y
    const int nb = std::min(65535, node_end - n0);
    k_bal_maps<<<dim3((mck + 15) / 16, nb), 256, 0, s>>>(c, n0);
    k_bal_starts<<<nb, 32, 0, s>>>(c, n0);
    k_bal_run<<<dim3((mck + 127) / 128, nb), 128, 0, s>>>(c, n0);
    launches += 3;
  }
  k_bal_gain<<<g, 256, 0, s>>>(c, item0, n_items);
  return launches;
}

int launch_bal_bwd(const DevCtx& c, int item0, int n_items, int node_begin, int node_end, cudaStream_t s) {
  if (n_items <= 0 || node_end <= node_begin) return 0;
  const int g = grid_size(n_items, 8);
  k_bal_adj<<<g, 256, 0, s>>>(c, item0, n_items);
  k_bal_rev<<<node_end - node_begin, 32, 0, s>>>(c, node_begin);
  k_bal_in<<<g, 256, 0, s>>>(c, item0, n_items);
  return 3;
}

int launch_bal_finalize(const DevCtx& c, int node_begin, int node_end, cudaStream_t s) {
  const int n = node_end - node_begin;
  if (n <= 0) return 0;
  k_bal_fin<<<(n + 127) / 128, 128, 0, s>>>(c, node_begin, node_end);
  return 1;
}

}  // namespace grafx
