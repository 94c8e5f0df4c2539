// Learned warm-start network: predicts every node's unconstrained processor parameters
// theta from audio.  The paper motivates a trained parameter estimator (Sec. 1) without
// fixing one; this network is the library's own.
//
// Features: log-mel of the mono mix of a stereo row (frames 2048, hop 512, no padding,
// periodic Hann, power spectrum, 128 HTK-mel triangles over 0..fs/2, ln(mel + 1e-5)),
// frames average-pooled to WS_T = 32.  A sample is [256][32]: the log-mel of a node's
// input (rendered with neutral parameters) in channels 0..127 and of the target mix in
// 128..255.
// Network: 4 conv1d layers (kernel 5, 'same' zero padding) 256->128->128->128->128 with
// bias and exact GELU, mean over time, then one MLP head per parameterised type
// 128->288->288->N_t.  Weights: one flat FP32 buffer in the order conv0.w [128][256][5],
// conv0.b, conv1.w ... conv3.b, then per head (g, s, e, c, d, r) w1 [288][128], b1,
// w2 [288][288], b2, w3 [N_t][288], b3.
// Every product runs on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulator
// in tensor memory) with BF16 operands (rounded to nearest even by their producers: the
// weight copies, the feature transpose, the products' epilogues, the time mean) copied
// into shared memory by the tensor memory accelerator; pre-activations, gradients and
// weights stay FP32 in HBM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "plan.h"

namespace grafx {

constexpr int WS_T = 32, WS_IN = 256, WS_CH = 128, WS_KW = 5, WS_HID = 288, WS_NHEAD = 6;
constexpr int WS_MEL = 128, WS_NFFT = 2048, WS_HOP = 512, WS_BINS = WS_NFFT / 2 + 1;
constexpr int WS_OUTMAX = 176;
static const int kHeadOut[WS_NHEAD] = {2, 1, 8, 4, 176, 50};

// ------------------------------------------------------------------ BF16 GEMM
// The register-staged product (grafx_gemm_bf16, the public matrix product):
// C[M,N] = alpha * A B + beta * C with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn] (FP32 in memory, BF16 in shared memory), C row-major (ldc).
// Operand tiles are loaded with float4 along whichever dimension has unit stride when
// it is a multiple of 4 (mode VK: along k, VR: along the row dimension m or n), else
// scalar (mode SC).  Split-K (gridDim.z > 1) writes partial tiles to `part` [z][M][N],
// summed in z order by k_gemm_reduce (deterministic).
enum : int { LD_SC = 0, LD_VK = 1, LD_VR = 2 };

// exact GELU and its derivative
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

struct GemmArgs {
  int M, N, K, kchunk;
  const void* A;  // float (the register-staged products; unused by the TMA-fed ones)
  int64_t sam, sak;
  const void* B;
  int64_t sbk, sbn;
  float* C;
  int64_t ldc;
  float alpha, beta;
  float* part;   // split-K partials or null
  int perm_cin;  // > 0: product column n = tap * perm_cin + c is stored at column c * WS_KW + tap
  // epilogue of the TMA-fed products (none with split-K): v = alpha acc + beta C, then
  const float* bias;  // v += bias[n]
  const float* zact;  // v *= gelu'(zact[m ldz + n])
  int64_t ldz;
  __nv_bfloat16* cb;  // BF16 copy cb[m ldcb + n] of gelu(v) (act = 1) or of v
  int64_t ldcb;
  int act;
};

// stored column of product column n
__device__ __forceinline__ int out_col(const GemmArgs& g, int n) {
  if (g.perm_cin <= 0) return n;
  const int tap = n / g.perm_cin;
  return (n - tap * g.perm_cin) * WS_KW + tap;
}

// ------------------------------------------------------------------ tcgen05 GEMM
// The same product on the 5th-generation tensor cores: a 128 x 128 FP32 accumulator
// in tensor memory (128 columns of TMEM), BF16 operand tiles of 128 x 64 in shared
// memory in the canonical K-major 128-byte-swizzled layout, one elected thread issuing
// tcgen05.mma (M = 128, N = 128, K = 16 per instruction, 4 per k-tile) whose completion
// is signalled on an mbarrier by tcgen05.commit.  Two shared-memory stages: the 128
// threads convert and store k-tile kt + 1 (FP32 loads, BF16 rounding) while the tensor
// cores consume k-tile kt.  Epilogue: tcgen05.ld 32x32b (warp w reads TMEM lanes
// 32 (w mod 4).. = rows, half of the columns each), alpha/beta, store (or the split-K
// partial tile).
// Every mbarrier wait is bounded; on expiry the kernel records GEMM_TIMEOUT in
// *status (if given), still waits for its own MMAs with a bound, frees its TMEM and
// returns.
constexpr int TC_M = 128, TC_N = 128, TC_K = 64, TC_THREADS = 256;
constexpr int TC_TMEM_COLS = 128;  // the 128 x 128 FP32 accumulator
constexpr int TC_TILE_BYTES = TC_M * TC_K * 2;              // one operand tile (16 KB)
// 2 stages x (A, B), reused by the epilogue as a padded 128 x 132 FP32 tile, + alignment
// + barriers: at most 3 CTAs per SM, 3 x 128 TMEM columns
constexpr int TC_EPI_LD = TC_N + 4;
constexpr int TC_SMEM = TC_M * TC_EPI_LD * 4 + 1024 + 64;
static_assert(TC_M * TC_EPI_LD * 4 >= 4 * TC_TILE_BYTES, "epilogue tile covers the operand stages");
constexpr uint32_t GEMM_TIMEOUT = 1u << 8;
constexpr int TC_SPIN = 1 << 22;

// byte offset of element (r, k) of a 128 x 64 BF16 tile: rows of 128 B, 8-row atoms of
// 1024 B, 16-byte chunk index XOR (row mod 8)
__device__ __forceinline__ uint32_t sw128(int r, int k) {
  const uint32_t lin = uint32_t(r) * 128u + uint32_t(k) * 2u;
  return lin ^ (((lin >> 7) & 7u) << 4);
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, atoms of 8 rows x 128 B
// (stride between 8-row groups 1024 B), version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N = 128, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TC_N >> 3) << 17) |
                              (uint32_t(TC_M >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < TC_SPIN; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

// This thread's share of a 128 x 64 operand tile X(r, k) = X[r sr + k sk] (rows r0..,
// k0..; zero outside R x kend): TC_V values, loaded into registers (tc_load) and stored
// as BF16 into the swizzled shared-memory tile (tc_store).
constexpr int TC_V = 128 * TC_K / TC_THREADS;  // 32 FP32 words
template <int MODE>
__device__ __forceinline__ void tc_load(uint32_t (&v)[TC_V], const void* Xv, int64_t sr, int64_t sk, int r0, int R,
                                        int k0, int kend) {
  const int tid = threadIdx.x;
  const float* __restrict__ X = static_cast<const float*>(Xv);
  if constexpr (MODE == LD_VK) {  // float4 along k: 128 rows x 16 quads
#pragma unroll
    for (int i = 0; i < TC_V / 4; ++i) {
      const int f = tid + i * TC_THREADS, r = f >> 4, kq = (f & 15) * 4;
      const int m = r0 + r, k = k0 + kq;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < R && k < kend) q = __ldg(reinterpret_cast<const float4*>(X + m * sr + k));
      v[4 * i] = __float_as_uint(q.x), v[4 * i + 1] = __float_as_uint(q.y);
      v[4 * i + 2] = __float_as_uint(q.z), v[4 * i + 3] = __float_as_uint(q.w);
    }
  } else if constexpr (MODE == LD_VR) {  // float4 along the rows: 64 k x 32 row quads
#pragma unroll
    for (int i = 0; i < TC_V / 4; ++i) {
      const int f = tid + i * TC_THREADS, kk = f >> 5, rq = (f & 31) * 4;
      const int m = r0 + rq, k = k0 + kk;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < R && k < kend) q = __ldg(reinterpret_cast<const float4*>(X + m + k * sk));
      v[4 * i] = __float_as_uint(q.x), v[4 * i + 1] = __float_as_uint(q.y);
      v[4 * i + 2] = __float_as_uint(q.z), v[4 * i + 3] = __float_as_uint(q.w);
    }
  } else {  // scalar FP32, k fastest
#pragma unroll
    for (int i = 0; i < TC_V; ++i) {
      const int f = tid + i * TC_THREADS, r = f >> 6, kk = f & 63;
      const int m = r0 + r, k = k0 + kk;
      v[i] = __float_as_uint((m < R && k < kend) ? X[m * sr + k * sk] : 0.f);
    }
  }
}

__device__ __forceinline__ void st_bf16(char* p, float x) {
  *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(x);
}

template <int MODE>
__device__ __forceinline__ void tc_store(char* tile, const uint32_t (&v)[TC_V]) {
  const int tid = threadIdx.x;
  if constexpr (MODE == LD_VK) {
#pragma unroll
    for (int i = 0; i < TC_V / 4; ++i) {
      const int f = tid + i * TC_THREADS, r = f >> 4, kq = (f & 15) * 4;
      __nv_bfloat162 lo = __floats2bfloat162_rn(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]));
      __nv_bfloat162 hi = __floats2bfloat162_rn(__uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3]));
      uint2 w;
      w.x = *reinterpret_cast<uint32_t*>(&lo);
      w.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(tile + sw128(r, kq)) = w;
    }
  } else if constexpr (MODE == LD_VR) {
#pragma unroll
    for (int i = 0; i < TC_V / 4; ++i) {
      const int f = tid + i * TC_THREADS, kk = f >> 5, rq = (f & 31) * 4;
#pragma unroll
      for (int j = 0; j < 4; ++j) st_bf16(tile + sw128(rq + j, kk), __uint_as_float(v[4 * i + j]));
    }
  } else {
#pragma unroll
    for (int i = 0; i < TC_V; ++i) {
      const int f = tid + i * TC_THREADS, r = f >> 6, kk = f & 63;
      st_bf16(tile + sw128(r, kk), __uint_as_float(v[i]));
    }
  }
}

// Epilogue of a 128 x 128 tile: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows),
// columns 64 (w / 4) .. + 63, 16 per tcgen05.ld, into a padded FP32 tile at `base` (the
// idle operand stages); then every warp writes whole rows (coalesced float4) with
// alpha/beta and the optional bias / GELU derivative / BF16 copy, or the split-K partial
// tile `split`.  have = false: the tile is zero (an empty k range).  ok = false: nothing
// is stored.
__device__ __forceinline__ void tc_epilogue(const GemmArgs& g, uint32_t tmem, char* base, int m0, int n0, bool have,
                                            bool ok, int split) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  float* E = reinterpret_cast<float*>(base);
  {
    const int row = quarter * 32 + lane;
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(E + row * TC_EPI_LD + c0 + j) =
            have ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                               __uint_as_float(r[j + 3]))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();
  if (!ok) return;
  float* part = g.part ? g.part + int64_t(split) * g.M * g.N : nullptr;
  float* dst = part ? part : g.C;
  const int64_t ld = part ? g.N : g.ldc;
  const bool perm = !part && g.perm_cin > 0;
  const bool vec = !perm && (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  const float alpha = part ? 1.f : g.alpha, beta = part ? 0.f : g.beta;
  const bool extra = !part && (g.bias || g.zact || g.cb);
  // this thread's columns n .. n + 3 (nv of them valid) are the same in all its rows;
  // rows warp + 8 i + 32 k: four rows per iteration, their global loads issued first
  const int qd = threadIdx.x & 31, n = n0 + 4 * qd, nv = max(0, min(4, g.N - n));
  if (nv == 0) return;
  float bv[4] = {0.f, 0.f, 0.f, 0.f};
  if (extra && g.bias)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < nv) bv[j] = g.bias[n + j];
  const bool zvec = g.zact && (g.ldz % 4) == 0 && (reinterpret_cast<uintptr_t>(g.zact) & 15) == 0;
  const bool cvec = g.cb && (g.ldcb % 4) == 0 && (reinterpret_cast<uintptr_t>(g.cb) & 7) == 0;
#pragma unroll 1
  for (int r0 = threadIdx.x >> 5; r0 < TC_M; r0 += 4 * (TC_THREADS / 32)) {
    float v[4][4], zz[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = r0 + i * (TC_THREADS / 32), m = m0 + rr;
      const float4 a4 = *reinterpret_cast<const float4*>(E + rr * TC_EPI_LD + 4 * qd);
      v[i][0] = alpha * a4.x, v[i][1] = alpha * a4.y, v[i][2] = alpha * a4.z, v[i][3] = alpha * a4.w;
#pragma unroll
      for (int j = 0; j < 4; ++j) zz[i][j] = 0.f;
      if (m >= g.M) continue;
      const float* cp = dst + int64_t(m) * ld;
      if (beta != 0.f) {
        if (vec && nv == 4) {
          const float4 c = *reinterpret_cast<const float4*>(cp + n);
          v[i][0] += beta * c.x, v[i][1] += beta * c.y, v[i][2] += beta * c.z, v[i][3] += beta * c.w;
        } else {
          for (int j = 0; j < nv; ++j) v[i][j] += beta * cp[perm ? out_col(g, n + j) : n + j];
        }
      }
      if (extra && g.zact) {
        const float* zp = g.zact + int64_t(m) * g.ldz + n;
        if (zvec && nv == 4) {
          const float4 z4 = *reinterpret_cast<const float4*>(zp);
          zz[i][0] = z4.x, zz[i][1] = z4.y, zz[i][2] = z4.z, zz[i][3] = z4.w;
        } else {
          for (int j = 0; j < nv; ++j) zz[i][j] = zp[j];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + r0 + i * (TC_THREADS / 32);
      if (m >= g.M) continue;
      if (extra) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          v[i][j] += bv[j];
          if (g.zact) v[i][j] *= gelu_d(zz[i][j]);
        }
        if (g.cb) {
          float h[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) h[j] = g.act ? gelu(v[i][j]) : v[i][j];
          __nv_bfloat16* q = g.cb + int64_t(m) * g.ldcb + n;
          if (cvec && nv == 4) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(h[0], h[1]), hi = __floats2bfloat162_rn(h[2], h[3]);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t*>(&lo);
            w.y = *reinterpret_cast<const uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(q) = w;
          } else {
            for (int j = 0; j < nv; ++j) q[j] = __float2bfloat16_rn(h[j]);
          }
        }
      }
      float* cp = dst + int64_t(m) * ld;
      if (vec && nv == 4) {
        *reinterpret_cast<float4*>(cp + n) = make_float4(v[i][0], v[i][1], v[i][2], v[i][3]);
      } else {
        for (int j = 0; j < nv; ++j) cp[perm ? out_col(g, n + j) : n + j] = v[i][j];
      }
    }
  }
}

template <int AM, int BM>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(GemmArgs g, uint32_t* status) {
  extern __shared__ __align__(1024) char tc_smem_raw[];
  // 1024-byte aligned operand stages, then two mbarriers and the TMEM address
  char* base = tc_smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(tc_smem_raw) & 1023)) & 1023);
  // stage st: A tile at base + st * TILE, B tile at base + (2 + st) * TILE
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TC_M * TC_EPI_LD * 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(bars));  // bar of stage st: bar0 + 8 st
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const int kbeg = blockIdx.z * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  const int ntiles = max(0, (kend - kbeg + TC_K - 1) / TC_K);

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // TMEM columns for the 128 x 128 FP32 accumulator
    const uint32_t slot = static_cast<uint32_t>(__cvta_generic_to_shared(tmem_slot));
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "n"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  int issued = 0;  // k-tiles whose MMAs were issued and committed
  uint32_t va[TC_V], vb[TC_V];  // k-tile kt + 1, loading while k-tile kt is stored and multiplied
  if (ntiles > 0) {
    tc_load<AM>(va, g.A, g.sam, g.sak, m0, g.M, kbeg, kend);
    tc_load<BM>(vb, g.B, g.sbn, g.sbk, n0, g.N, kbeg, kend);
  }
  for (int kt = 0; kt < ntiles; ++kt) {
    const int st = kt & 1;
    char* tA = base + st * TC_TILE_BYTES;
    char* tB = base + (2 + st) * TC_TILE_BYTES;
    // the MMAs of k-tile kt - 2 read this stage: wait for their commit
    if (kt >= 2) ok = __syncthreads_and(mbar_wait(bar0 + 8 * st, uint32_t(((kt - 2) >> 1) & 1))) != 0;
    if (!ok) break;  // an expiry (agreed by the whole CTA): stop issuing
    tc_store<AM>(tA, va);
    tc_store<BM>(tB, vb);
    if (kt + 1 < ntiles) {
      const int k1 = kbeg + (kt + 1) * TC_K;
      tc_load<AM>(va, g.A, g.sam, g.sak, m0, g.M, k1, kend);
      tc_load<BM>(vb, g.B, g.sbn, g.sbk, n0, g.N, k1, kend);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic stores -> async proxy
    __syncthreads();
    issued = kt + 1;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = static_cast<uint32_t>(__cvta_generic_to_shared(tA));
      const uint32_t b0 = static_cast<uint32_t>(__cvta_generic_to_shared(tB));
#pragma unroll
      for (int j = 0; j < TC_K / 16; ++j) {
        const uint64_t ad = umma_desc(a0 + 32u * j), bd = umma_desc(b0 + 32u * j);
        const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       bar0 + 8 * st)
                   : "memory");
    }
  }
  // the last commit covers every MMA issued before it (waited for, bounded, even after
  // an expiry, so that no MMA still writes the TMEM that is freed below)
  if (issued > 0) {
    const int last = issued - 1;
    const bool done = __syncthreads_and(mbar_wait(bar0 + 8 * (last & 1), uint32_t((last >> 1) & 1))) != 0;
    ok = ok && done;
  }
  if (!ok && threadIdx.x == 0 && status) atomicOr(status, GEMM_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  tc_epilogue(g, tmem, base, m0, n0, ntiles > 0, ok, blockIdx.z);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TC_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ TMA-fed conv products
// The conv layers' products as implicit GEMMs whose operand tiles are copied by the
// tensor memory accelerator (cp.async.bulk.tensor, 128-byte swizzle) straight from the
// BF16 activations, gradients and weight copies; no im2col or col2im matrix exists.
// Product index k (or n) = tap * cin + c for a tap 0..4 of the kernel and channel c, and
// a row is (sample b, frame t).  Operand tile modes (128 rows x 64 k):
//   TM_K2  K-major, 2-D map over X[rows][K]: one box {64, 128} at (k0, r0).
//   TM_K3  K-major, 3-D map over activations X[B][T][cin] (box {64, 32, 4}): tile row
//          (b, t) holds X[b][t + sign (tap - 2)][c0 .. c0 + 63] for k0 = tap cin + c0;
//          frames outside 0..T-1 and samples past B arrive as zeros (the conv's 'same'
//          zero padding).
//   TM_N2  MN-major, 2-D map over X[K][MN] (box {64, 64}): two boxes, rows r0 and r0 + 64.
//   TM_N3  MN-major, 3-D map over activations X[B][T][cin] (box {64, 32, 2}) with the tap
//          taken from the tile's rows: r0 = tap cin + c0, k0 = 32 b0 (two boxes, c0 and
//          c0 + 64).
// MN-major tiles hold 64 k-rows of 64 MN elements (128 B) per box, the boxes 8 KB apart:
// the descriptor's leading offset is that 8 KB (MN direction), its stride offset the
// 1 KB between groups of 8 k-rows.
enum : int { TM_K2 = 0, TM_K3 = 1, TM_N2 = 2, TM_N3 = 3 };
// A tile never straddles two taps and every box starts its innermost (channel)
// coordinate on a 64-element (128-byte) boundary: the channel counts are multiples of
// the k-tile, and of the 128-row tile for TM_N3, whose rows index tap * cin + c.
static_assert(WS_IN % TC_M == 0 && WS_CH % TC_M == 0 && TC_M % TC_K == 0 && TC_K == 64,
              "3-D activation maps need channel counts in whole 128-row tiles");
static_assert(WS_T == 32, "TM_K3 / TM_N3 boxes cover 32 frames per sample");
struct TmaGeom {
  int a_cin, a_sign, b_cin, b_sign;
};
constexpr int TM_STAGES = 3;
constexpr int TM_STAGE_BYTES = 2 * TC_TILE_BYTES;
constexpr int TM_BAR_BYTES = 8 * (2 * TM_STAGES + 1) + 16;
constexpr int TM_SMEM = TM_STAGES * TM_STAGE_BYTES + 1024 + TM_BAR_BYTES;
static_assert(TM_STAGES * TM_STAGE_BYTES >= TC_M * TC_EPI_LD * 4, "epilogue tile covers the operand stages");

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* m, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* m, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];\n" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// one 128 x 64 operand tile (rows r0.., k0..) into dst, completing on bar
template <int MODE>
__device__ __forceinline__ void tma_tile(const CUtensorMap* m, uint32_t dst, uint32_t bar, int r0, int k0, int cin,
                                         int sign) {
  if constexpr (MODE == TM_K2) {
    tma_load_2d(dst, m, bar, k0, r0);
  } else if constexpr (MODE == TM_K3) {
    const int tap = k0 / cin;
    tma_load_3d(dst, m, bar, k0 - tap * cin, sign * (tap - 2), r0 / WS_T);
  } else if constexpr (MODE == TM_N2) {
    tma_load_2d(dst, m, bar, r0, k0);
    tma_load_2d(dst + TC_TILE_BYTES / 2, m, bar, r0 + 64, k0);
  } else {
    const int tap = r0 / cin, c0 = r0 - tap * cin;
    tma_load_3d(dst, m, bar, c0, sign * (tap - 2), k0 / WS_T);
    tma_load_3d(dst + TC_TILE_BYTES / 2, m, bar, c0 + 64, sign * (tap - 2), k0 / WS_T);
  }
}

// descriptor of the K = 16 slice j of a tile in mode MODE
template <int MODE>
__device__ __forceinline__ uint64_t tm_desc(uint32_t tile, int j) {
  if constexpr (MODE == TM_K2 || MODE == TM_K3) {
    return umma_desc(tile + 32u * j);
  } else {  // MN-major: LBO 8192 B between the 64-element halves, SBO 1024 B between 8-k groups
    const uint32_t a = tile + 2048u * j;
    return uint64_t((a >> 4) & 0x3FFFu) | (uint64_t(8192 >> 4) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
  }
}

// One 128 x 128 output tile (k-tiles of split `split`).
// Warp 0 lane 0 issues the copies of k-tile kt into stage kt mod TM_STAGES once the MMAs
// of k-tile kt - TM_STAGES have released it (an mbarrier signalled by tcgen05.commit); warp 1 lane 0
// waits for each stage's bytes (expect_tx on the stage's full barrier) and issues its
// four MMAs; all 8 warps run the epilogue.  Every wait is bounded: on expiry the issuing
// stops, the CTA waits (bounded) for the MMAs and copies it started, records
// GEMM_TIMEOUT, frees its TMEM and stores nothing.
template <int AM, int BM>
__device__ __forceinline__ void tma_gemm(const CUtensorMap* ta, const CUtensorMap* tb, const GemmArgs& g,
                                         const TmaGeom& geo, int split, uint32_t* status) {
  extern __shared__ __align__(1024) char tm_smem_raw[];
  char* base = tm_smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(tm_smem_raw) & 1023)) & 1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TM_STAGES * TM_STAGE_BYTES);  // full[], empty[], done
  int* info = reinterpret_cast<int*>(bars + 2 * TM_STAGES + 1);  // tmem address, copies issued, tiles consumed
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(base));
  const uint32_t full0 = static_cast<uint32_t>(__cvta_generic_to_shared(bars));
  const uint32_t empty0 = full0 + 8 * TM_STAGES, done = full0 + 16 * TM_STAGES;
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const int kbeg = split * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  const int ntiles = max(0, (kend - kbeg + TC_K - 1) / TC_K);

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * TM_STAGES + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    info[1] = 0;
    info[2] = 0;
  }
  if (warp == 0) {  // TMEM columns for the 128 x 128 FP32 accumulator
    const uint32_t slot = static_cast<uint32_t>(__cvta_generic_to_shared(info));
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "n"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = static_cast<uint32_t>(info[0]);

  bool ok = true;
  if (threadIdx.x == 0) {  // copies
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(tb)) : "memory");
    int kt = 0;
    for (; kt < ntiles; ++kt) {
      const int st = kt % TM_STAGES;
      if (kt >= TM_STAGES && !mbar_wait(empty0 + 8 * st, uint32_t((kt / TM_STAGES - 1) & 1))) {
        ok = false;
        break;
      }
      const uint32_t fb = full0 + 8 * st, tA = sbase + st * TM_STAGE_BYTES;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "n"(TM_STAGE_BYTES)
                   : "memory");
      const int k0 = kbeg + kt * TC_K;
      tma_tile<AM>(ta, tA, fb, m0, k0, geo.a_cin, geo.a_sign);
      tma_tile<BM>(tb, tA + TC_TILE_BYTES, fb, n0, k0, geo.b_cin, geo.b_sign);
    }
    info[1] = kt;
  } else if (threadIdx.x == 32) {  // MMAs
    constexpr uint32_t idesc = TC_IDESC | (AM >= TM_N2 ? (1u << 15) : 0u) | (BM >= TM_N2 ? (1u << 16) : 0u);
    int kt = 0;
    for (; kt < ntiles; ++kt) {
      const int st = kt % TM_STAGES;
      if (!mbar_wait(full0 + 8 * st, uint32_t((kt / TM_STAGES) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t tA = sbase + st * TM_STAGE_BYTES, tB = tA + TC_TILE_BYTES;
#pragma unroll
      for (int j = 0; j < TC_K / 16; ++j) {
        const uint64_t ad = tm_desc<AM>(tA, j), bd = tm_desc<BM>(tB, j);
        const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       empty0 + 8 * st)
                   : "memory");
    }
    // one more commit: arrives once every MMA issued above has completed
    if (ntiles > 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                   : "memory");
    info[2] = kt;
  }
  __syncwarp();
  ok = __syncthreads_and(ok) != 0;
  const int issued = info[1], consumed = info[2];
  if (ntiles > 0) ok = (__syncthreads_and(mbar_wait(done, 0u)) != 0) && ok;
  if (threadIdx.x == 0)  // copies that were issued but never consumed (after an expiry)
    for (int kt = consumed; kt < issued; ++kt)
      if (!mbar_wait(full0 + 8 * (kt % TM_STAGES), uint32_t((kt / TM_STAGES) & 1))) ok = false;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && threadIdx.x == 0 && status) atomicOr(status, GEMM_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  tc_epilogue(g, tmem, base, m0, n0, ntiles > 0, ok, split);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TC_TMEM_COLS) : "memory");
}

template <int AM, int BM>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tma(const __grid_constant__ CUtensorMap ta,
                                                         const __grid_constant__ CUtensorMap tb, GemmArgs g,
                                                         TmaGeom geo, uint32_t* status) {
  tma_gemm<AM, BM>(&ta, &tb, g, geo, blockIdx.z, status);
}

// Up to WS_NHEAD independent products in one launch (blockIdx.z: the problem; CTAs past
// a problem's tiles return at once).  No split-K.
struct TmaGroup {
  CUtensorMap ta[WS_NHEAD], tb[WS_NHEAD];
  GemmArgs g[WS_NHEAD];
};
template <int AM, int BM>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tma_group(const __grid_constant__ TmaGroup grp,
                                                               uint32_t* status) {
  const GemmArgs& g = grp.g[blockIdx.z];
  if (int(blockIdx.y) * TC_M >= g.M || int(blockIdx.x) * TC_N >= g.N) return;
  tma_gemm<AM, BM>(&grp.ta[blockIdx.z], &grp.tb[blockIdx.z], g, TmaGeom{0, 0, 0, 0}, 0, status);
}

// C = alpha * sum_z part[z] + beta * C, z in order (columns through out_col)
__global__ void k_gemm_reduce(const float* __restrict__ part, int splits, GemmArgs g) {
  const int M = g.M, N = g.N;
  const int64_t ldc = g.ldc;
  const float alpha = g.alpha, beta = g.beta;
  float* __restrict__ C = g.C;
  const int64_t MN = int64_t(M) * N;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < MN; i += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * MN + i];
    float* cp = C + (i / N) * ldc + out_col(g, int(i % N));
    *cp = alpha * s + (beta != 0.f ? beta * *cp : 0.f);
  }
}

// Load mode of an operand X(r, k) = X[r sr + k sk] with R rows and K columns.
static int load_mode(const void* X, int64_t sr, int64_t sk, int R, int K) {
  const bool al = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (al && sk == 1 && sr % 4 == 0 && K % 4 == 0) return LD_VK;
  if (al && sr == 1 && sk % 4 == 0 && R % 4 == 0) return LD_VR;
  return LD_SC;
}

template <int AM, int BM>
static void launch_tc_one(dim3 grid, const GemmArgs& a, uint32_t* status, cudaStream_t s) {
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_gemm_tc<AM, BM>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    init = true;
  }
  k_gemm_tc<AM, BM><<<grid, TC_THREADS, TC_SMEM, s>>>(a, status);
}

template <int AM>
static void launch_tc_b(int bm, dim3 grid, const GemmArgs& a, uint32_t* status, cudaStream_t s) {
  switch (bm) {
    case LD_VK: launch_tc_one<AM, LD_VK>(grid, a, status, s); break;
    case LD_VR: launch_tc_one<AM, LD_VR>(grid, a, status, s); break;
    default: launch_tc_one<AM, LD_SC>(grid, a, status, s);
  }
}

// C = alpha op(A) op(B) + beta C on the tensor cores (tcgen05).  scratch: optional float
// buffer for split-K partials (scratch_floats capacity); status: optional device word
// that records a bounded wait's expiry.
static int gemm(int M, int N, int K, const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbk,
                 int64_t sbn, float* C, int64_t ldc, float alpha, float beta, cudaStream_t s,
                 float* scratch = nullptr, int64_t scratch_floats = 0, uint32_t* status = nullptr) {
  if (M <= 0 || N <= 0) return GRAFX_OK;
  GemmArgs a{M, N, K, 0, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta, nullptr, 0};
  const int tm = (M + TC_M - 1) / TC_M, tn = (N + TC_N - 1) / TC_N;
  const int ktiles = std::max(1, (K + TC_K - 1) / TC_K);
  int splits = 1;
  if (scratch && tm * tn < 2 * 148 && ktiles >= 4) {
    splits = std::min((2 * 148 + tm * tn - 1) / (tm * tn), ktiles / 2);
    splits = int(std::min<int64_t>(splits, scratch_floats / (int64_t(M) * N)));
    splits = std::max(splits, 1);
  }
  const int kt_per = (ktiles + splits - 1) / splits;
  a.kchunk = kt_per * TC_K;
  splits = (ktiles + kt_per - 1) / kt_per;
  if (splits > 1) a.part = scratch;
  dim3 grid(tn, tm, splits);
  const int am = load_mode(A, sam, sak, M, K), bm = load_mode(B, sbn, sbk, N, K);
  switch (am) {
    case LD_VK: launch_tc_b<LD_VK>(bm, grid, a, status, s); break;
    case LD_VR: launch_tc_b<LD_VR>(bm, grid, a, status, s); break;
    default: launch_tc_b<LD_SC>(bm, grid, a, status, s);
  }
  if (splits > 1) {
    const int64_t MN = int64_t(M) * N;
    k_gemm_reduce<<<int(std::min<int64_t>((MN + 255) / 256, 148 * 8)), 256, 0, s>>>(scratch, splits, a);
  }
  return GRAFX_OK;
}

// ------------------------------------------------------------------ TMA product launch
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a BF16 tensor (dims innermost first, rank 2 or 3; rows ld elements apart,
// else dense) read in boxes `box` with 128-byte swizzle; elements outside the tensor
// arrive as zeros.  The base must be 16-byte aligned and every row a multiple of 16 bytes
// (the encoder checks both).
static int bf16_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint32_t* box,
                    uint64_t ld = 0) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return fail(GRAFX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t gd[3], gs[2];
  cuuint32_t bx[3], es[3] = {1, 1, 1};
  uint64_t stride = 2;
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
    if (i > 0) gs[i - 1] = stride;
    stride *= (i == 0 && ld) ? ld : dims[i];
  }
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, cuuint32_t(rank), const_cast<void*>(base), gd, gs, bx, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GRAFX_OK : fail(GRAFX_ECUDA, "cuTensorMapEncodeTiled rejected a tensor map");
}

// X[rows][K] (rows ld >= K elements apart, 0: K), K-major boxes {64, 128}
static int map_k2(CUtensorMap* m, const __nv_bfloat16* X, int64_t rows, int64_t K, int64_t ld = 0) {
  const uint64_t d[2] = {uint64_t(K), uint64_t(rows)};
  const uint32_t bx[2] = {TC_K, TC_M};
  return bf16_map(m, X, 2, d, bx, uint64_t(ld));
}
// X[K][MN] (rows ld >= MN elements apart, 0: MN), MN-major boxes {64, 64}
static int map_n2(CUtensorMap* m, const __nv_bfloat16* X, int64_t K, int64_t MN, int64_t ld = 0) {
  const uint64_t d[2] = {uint64_t(MN), uint64_t(K)};
  const uint32_t bx[2] = {64, 64};
  return bf16_map(m, X, 2, d, bx, uint64_t(ld));
}
// activations X[B][T][C], boxes {64, T, samples}: 4 samples (TM_K3) or 2 (TM_N3)
static int map_act(CUtensorMap* m, const __nv_bfloat16* X, int B, int C, int samples) {
  const uint64_t d[3] = {uint64_t(C), uint64_t(WS_T), uint64_t(B)};
  const uint32_t bx[3] = {64, WS_T, uint32_t(samples)};
  return bf16_map(m, X, 3, d, bx);
}

// Arguments of C[M][N] = A B (ldc) for the TMA-fed products: alpha 1, beta 0, no
// epilogue extras (set by the caller).
static GemmArgs prod_args(int M, int N, int K, float* C, int64_t ldc) {
  GemmArgs a{};
  a.M = M, a.N = N, a.K = K, a.C = C, a.ldc = ldc, a.alpha = 1.f;
  return a;
}

// a.C = A B (stored through a.perm_cin, with a's epilogue extras) with TMA-fed operand
// tiles.  Products without extras and with fewer than 100 output tiles split K (partial
// tiles in scratch, at least 4 k-tiles a split) so that about one CTA runs per SM; the
// partials are summed in order.
template <int AM, int BM>
static int gemm_tma(GemmArgs a, const CUtensorMap& ta, const CUtensorMap& tb, TmaGeom geo, float* scratch,
                    int64_t scratch_floats, uint32_t* status, cudaStream_t s) {
  const int M = a.M, N = a.N, K = a.K;
  if (M <= 0 || N <= 0) return GRAFX_OK;
  const int tm = (M + TC_M - 1) / TC_M, tn = (N + TC_N - 1) / TC_N;
  const int ktiles = std::max(1, (K + TC_K - 1) / TC_K);
  const bool extras = a.bias || a.zact || a.cb;
  int splits = 1;
  if (scratch && !extras && tm * tn < 100 && ktiles >= 8) {
    splits = std::min((148 + tm * tn - 1) / (tm * tn), ktiles / 4);
    splits = int(std::min<int64_t>(splits, scratch_floats / (int64_t(M) * N)));
    splits = std::max(splits, 1);
  }
  const int kt_per = (ktiles + splits - 1) / splits;
  a.kchunk = kt_per * TC_K;
  splits = (ktiles + kt_per - 1) / kt_per;
  if (splits > 1) a.part = scratch;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_gemm_tma<AM, BM>, cudaFuncAttributeMaxDynamicSharedMemorySize, TM_SMEM);
    init = true;
  }
  k_gemm_tma<AM, BM><<<dim3(tn, tm, splits), TC_THREADS, TM_SMEM, s>>>(ta, tb, a, geo, status);
  if (splits > 1) {
    const int64_t MN = int64_t(M) * N;
    k_gemm_reduce<<<int(std::min<int64_t>((MN + 255) / 256, 148 * 8)), 256, 0, s>>>(scratch, splits, a);
  }
  return GRAFX_OK;
}

// The problems of grp (g[i].M = 0: none) in one launch.
template <int AM, int BM>
static int gemm_tma_group(TmaGroup& grp, uint32_t* status, cudaStream_t s) {
  int tm = 0, tn = 0;
  for (int i = 0; i < WS_NHEAD; ++i) {
    GemmArgs& g = grp.g[i];
    if (g.M <= 0 || g.N <= 0) {
      g.M = g.N = 0;
      continue;
    }
    g.kchunk = std::max(1, (g.K + TC_K - 1) / TC_K) * TC_K;
    g.alpha = 1.f;
    tm = std::max(tm, (g.M + TC_M - 1) / TC_M);
    tn = std::max(tn, (g.N + TC_N - 1) / TC_N);
  }
  if (tm == 0) return GRAFX_OK;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_gemm_tma_group<AM, BM>, cudaFuncAttributeMaxDynamicSharedMemorySize, TM_SMEM);
    init = true;
  }
  k_gemm_tma_group<AM, BM><<<dim3(tn, tm, WS_NHEAD), TC_THREADS, TM_SMEM, s>>>(grp, status);
  return GRAFX_OK;
}

// ------------------------------------------------------------------ elementwise pieces

// Features [B][256][32] (float32) to the first conv's operand [B][32][256] (BF16): one
// CTA per sample, transposed through shared memory.
__global__ void __launch_bounds__(256) k_feat_bf16(const float* __restrict__ f, __nv_bfloat16* __restrict__ fb) {
  __shared__ float tile[WS_IN][WS_T + 1];
  const float* src = f + int64_t(blockIdx.x) * WS_IN * WS_T;
  for (int i = threadIdx.x; i < WS_IN * WS_T; i += 256) tile[i / WS_T][i % WS_T] = src[i];
  __syncthreads();
  __nv_bfloat16* dst = fb + int64_t(blockIdx.x) * WS_IN * WS_T;
  for (int i = threadIdx.x; i < WS_IN * WS_T; i += 256) dst[i] = __float2bfloat16_rn(tile[i % WS_IN][i / WS_IN]);
}

// d *= gelu'(z); with db also a BF16 copy of the result (the products' operand)
__global__ void k_gelu_bwd(float* __restrict__ d, const float* __restrict__ z, int64_t n,
                           __nv_bfloat16* __restrict__ db = nullptr) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float v = d[i] * gelu_d(z[i]);
    d[i] = v;
    if (db) db[i] = __float2bfloat16_rn(v);
  }
}

// Column sums out[c] = sum_r x[r ld + c], c < cols (bias gradients), in two
// deterministic stages: CTA (cx, ry) sums rows ry, ry + 32 * gridDim.y, ... of its 32
// columns with 32 row slices and a fixed-order tree into part[ry][c]; then
// k_colsum_final adds the gridDim.y partials in order.
constexpr int CS_SPLIT = 64;
__global__ void __launch_bounds__(1024) k_colsum(const float* __restrict__ x, int64_t rows, int cols, int64_t ld,
                                                 float* __restrict__ part) {
  __shared__ float red[32][33];
  const int cx = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  const int64_t stride = 32 * int64_t(gridDim.y);
  float s = 0.f;
  if (c < cols)
    for (int64_t r = int64_t(blockIdx.y) * 32 + sl; r < rows; r += stride) s += x[r * ld + c];
  red[sl][cx] = s;
  __syncthreads();
  for (int w = 16; w > 0; w >>= 1) {
    if (sl < w) red[sl][cx] += red[sl + w][cx];
    __syncthreads();
  }
  if (sl == 0 && c < cols) part[int64_t(blockIdx.y) * cols + c] = red[0][cx];
}

__global__ void k_colsum_final(const float* __restrict__ part, int splits, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[z * cols + c];
  out[c] = s;
}

static void colsum(const float* x, int64_t rows, int cols, int64_t ld, float* out, float* part, cudaStream_t s) {
  const int splits = int(std::min<int64_t>(CS_SPLIT, std::max<int64_t>(1, rows / 256)));
  k_colsum<<<dim3((cols + 31) / 32, splits), 1024, 0, s>>>(x, rows, cols, ld, part);
  k_colsum_final<<<(cols + 127) / 128, 128, 0, s>>>(part, splits, cols, out);
}

// The column sums of up to WS_NHEAD matrices in two launches (blockIdx.z / blockIdx.y:
// the matrix), the same two stages and orders as colsum; partials of matrix i at
// part + i CS_SPLIT WS_HID.
struct ColsumGroup {
  const float* x[WS_NHEAD];
  float* out[WS_NHEAD];
  int64_t rows[WS_NHEAD], ld[WS_NHEAD];
  int cols[WS_NHEAD], splits[WS_NHEAD];
};
__global__ void __launch_bounds__(1024) k_colsum_group(ColsumGroup G, float* __restrict__ part) {
  const int i = blockIdx.z;
  if (int(blockIdx.y) >= G.splits[i] || int(blockIdx.x) * 32 >= G.cols[i]) return;
  __shared__ float red[32][33];
  const int cx = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx, cols = G.cols[i];
  const int64_t stride = 32 * int64_t(G.splits[i]), ld = G.ld[i];
  const float* x = G.x[i];
  float s = 0.f;
  if (c < cols)
    for (int64_t r = int64_t(blockIdx.y) * 32 + sl; r < G.rows[i]; r += stride) s += x[r * ld + c];
  red[sl][cx] = s;
  __syncthreads();
  for (int w = 16; w > 0; w >>= 1) {
    if (sl < w) red[sl][cx] += red[sl + w][cx];
    __syncthreads();
  }
  if (sl == 0 && c < cols) part[int64_t(i) * CS_SPLIT * WS_HID + int64_t(blockIdx.y) * cols + c] = red[0][cx];
}
__global__ void k_colsum_final_group(ColsumGroup G, const float* __restrict__ part) {
  const int i = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cols[i]) return;
  const float* p = part + int64_t(i) * CS_SPLIT * WS_HID;
  float s = 0.f;
  for (int z = 0; z < G.splits[i]; ++z) s += p[z * G.cols[i] + c];
  G.out[i][c] = s;
}
// G.rows[i] = 0: no matrix i
static void colsum_group(ColsumGroup& G, float* part, cudaStream_t s) {
  int cmax = 0, smax = 0;
  for (int i = 0; i < WS_NHEAD; ++i) {
    G.splits[i] = G.rows[i] > 0 ? int(std::min<int64_t>(CS_SPLIT, std::max<int64_t>(1, G.rows[i] / 256))) : 0;
    if (G.rows[i] <= 0) G.cols[i] = 0;
    cmax = std::max(cmax, G.cols[i]);
    smax = std::max(smax, G.splits[i]);
  }
  if (cmax == 0) return;
  k_colsum_group<<<dim3((cmax + 31) / 32, smax, WS_NHEAD), 1024, 0, s>>>(G, part);
  k_colsum_final_group<<<dim3((cmax + 127) / 128, WS_NHEAD), 128, 0, s>>>(G, part);
}

// x[r][c] (rows x cols, row stride ld) as BF16 y[r][c] (row stride ldy)
__global__ void k_to_bf16(const float* __restrict__ x, int64_t rows, int cols, int64_t ld,
                          __nv_bfloat16* __restrict__ y, int64_t ldy) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / cols;
    const int c = int(i % cols);
    y[r * ldy + c] = __float2bfloat16_rn(x[r * ld + c]);
  }
}

// e[b][c] = mean over the frames of gelu(z[b][t][c]) (the last conv layer's activation),
// stored as BF16: the heads' first operand
__global__ void k_time_mean(const float* __restrict__ z, int B, __nv_bfloat16* __restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * WS_CH) return;
  const int b = i / WS_CH, c = i % WS_CH;
  float s = 0.f;
  for (int t = 0; t < WS_T; ++t) s += gelu(z[(int64_t(b) * WS_T + t) * WS_CH + c]);
  e[i] = __float2bfloat16_rn(s / float(WS_T));
}

__global__ void k_time_mean_bwd(const float* __restrict__ de, int B, float* __restrict__ dh) {
  const int64_t n = int64_t(B) * WS_T * WS_CH;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(i % WS_CH);
    const int b = int(i / (int64_t(WS_T) * WS_CH));
    dh[i] = de[b * WS_CH + c] / float(WS_T);
  }
}

// Masked mean-squared error, every row weighted alike: loss = (1/B) sum_b (1/n_b)
// sum_{j < n_b} (out - tgt)^2 with n_b = n_out[b]; d = 2 (out - tgt) / (B n_b), 0 in
// unused columns.
__global__ void __launch_bounds__(1024) k_ws_mse(const float* __restrict__ out, const float* __restrict__ tgt,
                                                 const int32_t* __restrict__ nout, int B,
                                                 float* __restrict__ loss, float* __restrict__ d) {
  // warp w takes rows w, w + 32, ... two at a time (their loads issued first), lane l
  // columns l + 32 k; the per-thread sums meet in a fixed-order block sum
  constexpr int KC = (WS_OUTMAX + 31) / 32;
  __shared__ float red[4 * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float s = 0.f;
  for (int b0 = warp; b0 < B; b0 += 2 * 32) {
    float o[2][KC], t[2][KC];
    int nb[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int b = b0 + 32 * r;
      nb[r] = b < B ? nout[b] : 0;
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int j = lane + 32 * k;
        const bool in = b < B && j < WS_OUTMAX;
        o[r][k] = in ? out[int64_t(b) * WS_OUTMAX + j] : 0.f;
        t[r][k] = in ? tgt[int64_t(b) * WS_OUTMAX + j] : 0.f;
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int b = b0 + 32 * r;
      if (b >= B) continue;
      const float w = nb[r] > 0 ? 1.f / (float(B) * float(nb[r])) : 0.f;
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int j = lane + 32 * k;
        if (j >= WS_OUTMAX) continue;
        float g = 0.f;
        if (j < nb[r]) {
          const float e = o[r][k] - t[r][k];
          s += e * e * w;
          g = 2.f * e * w;
        }
        d[int64_t(b) * WS_OUTMAX + j] = g;
      }
    }
  }
  float v[1] = {s};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) *loss = v[0];
}

// BF16 weight copies: conv layer l tap-major (0..3), per head w1, w2, w3 (4..21), conv
// layer l = 1..3 transposed tap-major (22..24)
constexpr int WB_MATS = 4 + 3 * WS_NHEAD + 3;
constexpr int WB_CONVT = 4 + 3 * WS_NHEAD;
enum : int { WC_PLAIN = 0, WC_TAPS = 1, WC_TAPS_T = 2 };
struct WeightCopies {
  int64_t src[WB_MATS], dst[WB_MATS], n[WB_MATS];
  int32_t mode[WB_MATS], cin[WB_MATS];
};

// Copy j of the weights as BF16.  WC_TAPS: conv w [128][cin][5] as [128][5][cin] (the
// product index tap * cin + c of the TMA-fed products); WC_TAPS_T: as [cin][5][128].
__global__ void k_weights_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, WeightCopies cp) {
  const int j = blockIdx.y, mode = cp.mode[j], cin = cp.cin[j];
  const float* src = w + cp.src[j];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cp.n[j]; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t q = i;
    if (mode == WC_TAPS) {
      const int K = cin * WS_KW;
      const int o = int(i / K), k = int(i % K), tap = k / cin, c = k % cin;
      q = int64_t(o) * K + c * WS_KW + tap;
    } else if (mode == WC_TAPS_T) {
      const int c = int(i / (WS_KW * WS_CH)), k = int(i % (WS_KW * WS_CH)), tap = k / WS_CH, o = k % WS_CH;
      q = int64_t(o) * cin * WS_KW + c * WS_KW + tap;
    }
    wb[cp.dst[j] + i] = __float2bfloat16_rn(src[q]);
  }
}

// ------------------------------------------------------------------ log-mel features
// Frames 2q and 2q+1 of a row packed as the real and imaginary parts of one complex
// 2048-point FFT; writes ln(mel + 1e-5) of both into fr[row][frame][128].
__global__ void __launch_bounds__(WS_NFFT / 16) k_logmel_frames(const float* __restrict__ rows, int64_t rstride,
                                                                int64_t pitch, int nframes,
                                                                const float* __restrict__ melw,
                                                                const int2_* __restrict__ mel_rng,
                                                                const float2_* __restrict__ tw,
                                                                const float2_* __restrict__ ptw,
                                                                float* __restrict__ fr) {
  __shared__ float2 buf[fft::Padded<WS_NFFT>::size];
  __shared__ float pw[2][WS_BINS];
  const int r = blockIdx.y, f = 2 * blockIdx.x;
  const float* x = rows + int64_t(r) * rstride;
  for (int j = threadIdx.x; j < WS_NFFT; j += blockDim.x) {
    const float w = 0.5f - 0.5f * tw[j * (TWIDDLE_N / WS_NFFT)].x;
    const int64_t t0 = int64_t(f) * WS_HOP + j, t1 = t0 + WS_HOP;
    const float a = (f < nframes) ? 0.5f * (x[t0] + x[pitch + t0]) : 0.f;
    const float b = (f + 1 < nframes) ? 0.5f * (x[t1] + x[pitch + t1]) : 0.f;
    buf[fft::pad(j)] = make_float2(w * a, w * b);
  }
  __syncthreads();
  fft::forward<WS_NFFT>(buf, ptw, threadIdx.x, true);
  for (int k = threadIdx.x; k < WS_BINS; k += blockDim.x) {
    const float2 z = buf[fft::pad(k)], zm = buf[fft::pad((WS_NFFT - k) & (WS_NFFT - 1))];
    const float ax = 0.5f * (z.x + zm.x), ay = 0.5f * (z.y - zm.y);
    const float bx = 0.5f * (z.y + zm.y), by = 0.5f * (zm.x - z.x);
    pw[0][k] = ax * ax + ay * ay;
    pw[1][k] = bx * bx + by * by;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * WS_MEL; i += blockDim.x) {
    const int q = i / WS_MEL, m = i % WS_MEL;
    if (f + q >= nframes) continue;
    const int2_ rg = mel_rng[m];
    float s = 0.f;
    for (int k = rg.x; k < rg.y; ++k) s += melw[m * WS_BINS + k] * pw[q][k];
    fr[(int64_t(r) * nframes + f + q) * WS_MEL + m] = logf(s + 1e-5f);
  }
}

// Average-pool the frames to WS_T: feats[i][coff + m][t] for sample i, which takes
// row row_of[i] (or row i when row_of is null).
__global__ void k_logmel_pool(const float* __restrict__ fr, int nframes, int n_rows, int n_samples,
                              const int32_t* __restrict__ row_of, int coff, float* __restrict__ feats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_samples * WS_MEL * WS_T) return;
  const int t = i % WS_T, m = (i / WS_T) % WS_MEL, smp = i / (WS_T * WS_MEL);
  const int r = row_of ? row_of[smp] : smp;
  float* o = feats + (int64_t(smp) * WS_IN + coff + m) * WS_T + t;
  if (r < 0 || r >= n_rows) {  // invalid row index: zero features
    *o = 0.f;
    return;
  }
  const int a = (t * nframes) / WS_T, b = max(((t + 1) * nframes) / WS_T, a + 1);
  float s = 0.f;
  for (int f = a; f < b; ++f) s += fr[(int64_t(r) * nframes + f) * WS_MEL + m];
  *o = s / float(b - a);
}

// ------------------------------------------------------------------ cross-spectral band gain
// Frame f of sample i: two groups of 128 threads, group h transforming the mid (h = 0) or
// the side (h = 1) of the node input u and of the target t packed as w (u_h + i t_h) in one
// 2048-point FFT; per bin the cross term Re(T conj(U)) and |U|^2; per band pair (mel
// triangles 2b, 2b + 1) their weighted sums C and P into fr[i][f][h][C 0..63, P 64..127].
constexpr int XG_BANDS = WS_MEL / 2;
__global__ void __launch_bounds__(2 * (WS_NFFT / 16)) k_xgain_frames(
    const float* __restrict__ u, int64_t ustride, const float* __restrict__ trows, int64_t tstride,
    const int32_t* __restrict__ row_of, int n_trows, int64_t pitch, int nframes, const float* __restrict__ melw,
    const int2_* __restrict__ mel_rng, const float2_* __restrict__ tw, const float2_* __restrict__ ptw,
    float* __restrict__ fr) {
  constexpr int T = WS_NFFT / 16, PS = fft::Padded<WS_NFFT>::size;
  extern __shared__ float2 xg_smem[];   // [2][PS] transforms, then [2][WS_BINS] cross and power
  float* cr = reinterpret_cast<float*>(xg_smem + 2 * PS);   // cr[h * WS_BINS + k]
  float* pu = cr + 2 * WS_BINS;                              // pu[h * WS_BINS + k]
  const int smp = blockIdx.y, f = blockIdx.x;
  const int h = threadIdx.x / T, gt = threadIdx.x % T;
  float2* buf = xg_smem + h * PS;
  const int r = row_of[smp];
  const bool has_t = r >= 0 && r < n_trows;
  const float* x = u + int64_t(smp) * ustride;
  const float* y = has_t ? trows + int64_t(r) * tstride : nullptr;
  const float sg = h ? -1.f : 1.f;
  for (int j = gt; j < WS_NFFT; j += T) {
    const float w = 0.5f - 0.5f * tw[j * (TWIDDLE_N / WS_NFFT)].x;
    const int64_t t0 = int64_t(f) * WS_HOP + j;
    const float a = 0.5f * (x[t0] + sg * x[pitch + t0]);
    const float b = has_t ? 0.5f * (y[t0] + sg * y[pitch + t0]) : 0.f;
    buf[fft::pad(j)] = make_float2(w * a, w * b);
  }
  __syncthreads();
  fft::forward<WS_NFFT>(buf, ptw, gt, true);
  for (int k = gt; k < WS_BINS; k += T) {
    const float2 z = buf[fft::pad(k)], zm = buf[fft::pad((WS_NFFT - k) & (WS_NFFT - 1))];
    const float ux = 0.5f * (z.x + zm.x), uy = 0.5f * (z.y - zm.y);   // U = (Z + conj Zm) / 2
    const float yx = 0.5f * (z.y + zm.y), yy = 0.5f * (zm.x - z.x);   // Y = (Z - conj Zm) / 2i
    cr[h * WS_BINS + k] = yx * ux + yy * uy;
    pu[h * WS_BINS + k] = ux * ux + uy * uy;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * 2 * XG_BANDS; i += blockDim.x) {
    const int hh = i / (2 * XG_BANDS), q = i % (2 * XG_BANDS), b = q % XG_BANDS;
    const float* src = (q < XG_BANDS ? cr : pu) + hh * WS_BINS;
    float acc = 0.f;
    for (int m = 2 * b; m < 2 * b + 2; ++m) {
      const int2_ rg = mel_rng[m];
      for (int k = rg.x; k < rg.y; ++k) acc += melw[m * WS_BINS + k] * src[k];
    }
    fr[((int64_t(smp) * nframes + f) * 2 + hh) * (2 * XG_BANDS) + q] = acc;
  }
}

// Pool slot t of sample i: C and P summed over the slot's frames (the log-mel's ranges),
// feats[i][coff + h 64 + b][t] = ln(max(C / P, 0) + 1e-2).
__global__ void k_xgain_pool(const float* __restrict__ fr, int nframes, int n_samples, int coff,
                             float* __restrict__ feats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_samples * WS_MEL * WS_T) return;
  const int t = i % WS_T, c = (i / WS_T) % WS_MEL, smp = i / (WS_T * WS_MEL);
  const int hh = c / XG_BANDS, b = c % XG_BANDS;
  const int a = (t * nframes) / WS_T, e = max(((t + 1) * nframes) / WS_T, a + 1);
  float C = 0.f, P = 0.f;
  for (int f = a; f < e; ++f) {
    const float* q = fr + ((int64_t(smp) * nframes + f) * 2 + hh) * (2 * XG_BANDS);
    C += q[b];
    P += q[XG_BANDS + b];
  }
  feats[(int64_t(smp) * WS_IN + coff + c) * WS_T + t] = logf(fmaxf(C / fmaxf(P, 1e-20f), 0.f) + 1e-2f);
}

// ------------------------------------------------------------------ node inputs
// u_v (Eq. 1b, gathered exactly like the step kernels) of the nodes ids.v[0..n) into
// rows dst[ids.first + i][2][dst_pitch]; samples in [len, dst_pitch) are zero.
__global__ void k_node_inputs(DevCtx c, NodeIds ids, float* __restrict__ dst, int64_t dst_pitch) {
  const int i = blockIdx.y;
  const int v = ids.v[i];
  const NodeDev& n = c.nodes[v];
  float* o = dst + int64_t(ids.first + i) * 2 * dst_pitch;
  const int64_t quads = dst_pitch / 4;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < 2 * quads;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int ch = int(q / quads);
    const int t = int(q % quads) * 4;
    float4 val = f4zero();
    if (t < n.len) val = gather_in(c, v, ch, t, n.len, n.pitch);
    st4(o + ch * dst_pitch + t, val);
  }
}

int launch_node_inputs(const DevCtx& c, const NodeIds& ids, int n, float* dst, int64_t dst_pitch, cudaStream_t s) {
  if (n <= 0) return 0;
  const int gx = int(std::min<int64_t>((2 * (dst_pitch / 4) + 255) / 256, 64));
  k_node_inputs<<<dim3(gx, n), 256, 0, s>>>(c, ids, dst, dst_pitch);
  return 1;
}

}  // namespace grafx

// ====================================================================== host side
using namespace grafx;

struct grafx_wsnet {
  int64_t off[4][2];          // conv weight / bias offsets in the flat buffer
  int64_t hoff[WS_NHEAD][6];  // per head: w1 b1 w2 b2 w3 b3
  int64_t n_params = 0;
  WeightCopies wcp;           // BF16 shadows of the weights (k_weights_bf16)
  int64_t wb_elems = 0;
  int32_t max_batch = 0;
  char* ws = nullptr;         // bound workspace
  size_t ws_bytes = 0;
  std::vector<float> melw;    // [128][1025] mel triangles
  std::vector<int2_> mel_rng; // nonzero bin range of each triangle
  std::vector<float2_> tw, ptw;
};

namespace {

// split-K partials of the weight-gradient products: up to 32 partial [128][1280] tiles
constexpr int64_t WS_DBIG_FLOATS = int64_t(32) * WS_CH * WS_IN * WS_KW;

struct WsNetLayout {
  size_t melw, melrng, tw, ptw, status;
  size_t fb, hb[3], z[4], eb, a1, g1b, a2, g2b, dbig, dsmall, dab, dob, dh, dzb[2], cspart, wbf, frames, total;
};

// frame_floats: log-mel frame scratch (rows x frames x 128) in floats
WsNetLayout ws_layout(const grafx_wsnet* n, int64_t frame_floats) {
  WsNetLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = (o + bytes + 255) / 256 * 256;
    return r;
  };
  const size_t B = size_t(n->max_batch), rows = B * WS_T;
  L.melw = take(4 * n->melw.size());
  L.melrng = take(sizeof(int2_) * n->mel_rng.size());
  L.tw = take(sizeof(float2_) * n->tw.size());
  L.ptw = take(sizeof(float2_) * n->ptw.size());
  L.status = take(sizeof(uint32_t));
  L.fb = take(2 * rows * WS_IN);
  for (int l = 0; l < 3; ++l) L.hb[l] = take(2 * rows * WS_CH);
  for (int l = 0; l < 4; ++l) L.z[l] = take(4 * rows * WS_CH);
  L.eb = take(2 * B * WS_CH);
  L.a1 = take(4 * B * WS_HID);
  L.g1b = take(2 * B * WS_HID);
  L.a2 = take(4 * B * WS_HID);
  L.g2b = take(2 * B * WS_HID);
  L.dbig = take(4 * size_t(WS_DBIG_FLOATS));
  L.dsmall = take(4 * B * WS_HID * 2);
  L.dab = take(2 * B * WS_HID * 2);
  L.dob = take(2 * B * WS_OUTMAX);
  L.dh = take(4 * (B * WS_CH + rows * WS_CH));
  for (int i = 0; i < 2; ++i) L.dzb[i] = take(2 * rows * WS_CH);
  L.cspart = take(4 * size_t(WS_NHEAD) * CS_SPLIT * WS_HID);
  L.wbf = take(2 * size_t(n->wb_elems));
  L.frames = take(4 * size_t(std::max<int64_t>(frame_floats, 1)));
  L.total = o;
  return L;
}

int grid1(int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 148 * 16)); }

int cuda_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRAFX_OK : fail(GRAFX_ECUDA, cudaGetErrorString(e));
}

int n_frames_of(int64_t len) { return int(1 + (len - WS_NFFT) / WS_HOP); }

int check_heads(const int32_t* head_count, int32_t B) {
  int64_t sum = 0;
  for (int h = 0; h < WS_NHEAD; ++h) {
    if (head_count[h] < 0) return fail(GRAFX_ESHAPE, "negative head count");
    sum += head_count[h];
  }
  if (sum != B) return fail(GRAFX_ESHAPE, "head counts must sum to the batch");
  return GRAFX_OK;
}

}  // namespace

extern "C" {

int grafx_ws_create(int32_t max_batch, int32_t sample_rate, grafx_wsnet** out) {
  if (!out) return fail(GRAFX_EINVAL, "null argument");
  *out = nullptr;
  if (max_batch < 1 || max_batch > 65536 || sample_rate < 8000) return fail(GRAFX_EINVAL, "bad batch or rate");
  grafx_wsnet* n = new (std::nothrow) grafx_wsnet();
  if (!n) return fail(GRAFX_ENOMEM, "host allocation failed");
  n->max_batch = max_batch;
  int64_t o = 0;
  const int cin[4] = {WS_IN, WS_CH, WS_CH, WS_CH};
  for (int l = 0; l < 4; ++l) {
    n->off[l][0] = o;
    o += int64_t(WS_CH) * cin[l] * WS_KW;
    n->off[l][1] = o;
    o += WS_CH;
  }
  for (int h = 0; h < WS_NHEAD; ++h) {
    const int64_t sz[6] = {int64_t(WS_HID) * WS_CH, WS_HID, int64_t(WS_HID) * WS_HID, WS_HID,
                           int64_t(kHeadOut[h]) * WS_HID, kHeadOut[h]};
    for (int i = 0; i < 6; ++i) {
      n->hoff[h][i] = o;
      o += sz[i];
    }
  }
  n->n_params = o;
  {
    int64_t d = 0;
    auto add = [&](int j, int64_t src, int64_t cnt, int mode, int ci) {
      n->wcp.src[j] = src;
      n->wcp.dst[j] = d;
      n->wcp.n[j] = cnt;
      n->wcp.mode[j] = mode;
      n->wcp.cin[j] = ci;
      d += (cnt + 63) / 64 * 64;  // 128-byte aligned copies (tensor-map bases)
    };
    for (int l = 0; l < 4; ++l) add(l, n->off[l][0], int64_t(WS_CH) * cin[l] * WS_KW, WC_TAPS, cin[l]);
    for (int h = 0; h < WS_NHEAD; ++h) {
      add(4 + 3 * h, n->hoff[h][0], int64_t(WS_HID) * WS_CH, WC_PLAIN, 0);
      add(5 + 3 * h, n->hoff[h][2], int64_t(WS_HID) * WS_HID, WC_PLAIN, 0);
      add(6 + 3 * h, n->hoff[h][4], int64_t(kHeadOut[h]) * WS_HID, WC_PLAIN, 0);
    }
    for (int l = 1; l < 4; ++l)
      add(WB_CONVT + l - 1, n->off[l][0], int64_t(WS_CH) * cin[l] * WS_KW, WC_TAPS_T, cin[l]);
    n->wb_elems = d;
  }
  // HTK-mel triangles over the one-sided bins of a 2048-point frame, edges equally
  // spaced in mel between 0 and fs/2
  auto hz2mel = [](double f) { return 2595.0 * std::log10(1.0 + f / 700.0); };
  auto mel2hz = [](double m) { return 700.0 * (std::pow(10.0, m / 2595.0) - 1.0); };
  const double mtop = hz2mel(sample_rate / 2.0);
  n->melw.assign(size_t(WS_MEL) * WS_BINS, 0.f);
  n->mel_rng.assign(WS_MEL, int2_{0, 0});
  for (int m = 0; m < WS_MEL; ++m) {
    const double lo = mel2hz(mtop * m / (WS_MEL + 1)), c = mel2hz(mtop * (m + 1) / (WS_MEL + 1)),
                 hi = mel2hz(mtop * (m + 2) / (WS_MEL + 1));
    int first = WS_BINS, last = 0;
    for (int k = 0; k < WS_BINS; ++k) {
      const double f = double(k) * sample_rate / WS_NFFT;
      const double w = std::max(0.0, std::min((f - lo) / (c - lo), (hi - f) / (hi - c)));
      n->melw[size_t(m) * WS_BINS + k] = float(w);
      if (w > 0) {
        first = std::min(first, k);
        last = std::max(last, k + 1);
      }
    }
    n->mel_rng[m] = int2_{first < WS_BINS ? first : 0, last};
  }
  fill_fft_tables(n->tw, n->ptw);
  *out = n;
  return GRAFX_OK;
}

int grafx_ws_destroy(grafx_wsnet* n) {
  delete n;
  return GRAFX_OK;
}

int grafx_ws_param_count(const grafx_wsnet* n, int64_t* count) {
  if (!n || !count) return fail(GRAFX_EINVAL, "null argument");
  *count = n->n_params;
  return GRAFX_OK;
}

int grafx_ws_workspace_bytes(const grafx_wsnet* n, int32_t max_rows, int64_t max_len, size_t* bytes) {
  if (!n || !bytes) return fail(GRAFX_EINVAL, "null argument");
  if (max_rows < 0 || max_rows > 65535 || max_len < WS_NFFT)
    return fail(GRAFX_ESHAPE, "log-mel rows: at most 65535, each at least 2048 samples");
  *bytes = ws_layout(n, int64_t(max_rows) * n_frames_of(max_len) * WS_MEL).total;
  return GRAFX_OK;
}

int grafx_ws_bind(grafx_wsnet* n, void* ws, size_t bytes, void* stream) {
  if (!n || !ws) return fail(GRAFX_EINVAL, "null argument");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return fail(GRAFX_EINVAL, "workspace must be 256-byte aligned");
  WsNetLayout L = ws_layout(n, 0);
  if (bytes < L.total) return fail(GRAFX_ESHAPE, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  cudaMemcpyAsync(w + L.melw, n->melw.data(), 4 * n->melw.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + L.melrng, n->mel_rng.data(), sizeof(int2_) * n->mel_rng.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + L.tw, n->tw.data(), sizeof(float2_) * n->tw.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + L.ptw, n->ptw.data(), sizeof(float2_) * n->ptw.size(), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(w + L.status, 0, sizeof(uint32_t), s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, cudaGetErrorString(e));
  n->ws = w;
  n->ws_bytes = bytes;
  return GRAFX_OK;
}

int grafx_ws_logmel(grafx_wsnet* n, const float* rows, int32_t n_rows, int64_t row_stride, int64_t pitch, int64_t len,
                    const int32_t* row_of_sample, int32_t n_samples, int32_t coff, float* feats, void* stream) {
  if (!n || !rows || !feats) return fail(GRAFX_EINVAL, "null argument");
  if (!n->ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_ws_bind)");
  if (n_rows < 1 || n_rows > 65535 || n_samples < 1 || len < WS_NFFT || pitch < len || row_stride < 2 * pitch ||
      (coff != 0 && coff != WS_MEL) || (!row_of_sample && n_samples != n_rows) ||
      int64_t(n_samples) * WS_MEL * WS_T > INT32_MAX)
    return fail(GRAFX_ESHAPE, "bad log-mel shape");
  const int nframes = n_frames_of(len);
  WsNetLayout L = ws_layout(n, int64_t(n_rows) * nframes * WS_MEL);
  if (L.total > n->ws_bytes) return fail(GRAFX_ESHAPE, "workspace too small for these log-mel rows");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* fr = reinterpret_cast<float*>(n->ws + L.frames);
  k_logmel_frames<<<dim3((nframes + 1) / 2, n_rows), WS_NFFT / 16, 0, s>>>(
      rows, row_stride, pitch, nframes, reinterpret_cast<const float*>(n->ws + L.melw),
      reinterpret_cast<const int2_*>(n->ws + L.melrng), reinterpret_cast<const float2_*>(n->ws + L.tw),
      reinterpret_cast<const float2_*>(n->ws + L.ptw), fr);
  k_logmel_pool<<<(n_samples * WS_MEL * WS_T + 255) / 256, 256, 0, s>>>(fr, nframes, n_rows, n_samples,
                                                                          row_of_sample, coff, feats);
  return cuda_status();
}

int grafx_ws_xgain(grafx_wsnet* n, const float* u_rows, int32_t n_samples, int64_t u_stride, const float* t_rows,
                   int32_t n_trows, int64_t t_stride, const int32_t* row_of_sample, int64_t pitch, int64_t len,
                   int32_t coff, float* feats, void* stream) {
  if (!n || !u_rows || !t_rows || !row_of_sample || !feats) return fail(GRAFX_EINVAL, "null argument");
  if (!n->ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_ws_bind)");
  if (n_samples < 1 || n_samples > 65535 || n_trows < 1 || len < WS_NFFT || pitch < len || u_stride < 2 * pitch ||
      t_stride < 2 * pitch || (coff != 0 && coff != WS_MEL) || int64_t(n_samples) * WS_MEL * WS_T > INT32_MAX)
    return fail(GRAFX_ESHAPE, "bad cross-gain shape");
  const int nframes = n_frames_of(len);
  WsNetLayout L = ws_layout(n, int64_t(n_samples) * nframes * 2 * WS_MEL);
  if (L.total > n->ws_bytes) return fail(GRAFX_ESHAPE, "workspace too small for these cross-gain samples");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* fr = reinterpret_cast<float*>(n->ws + L.frames);
  constexpr int smem = int(sizeof(float2)) * 2 * fft::Padded<WS_NFFT>::size + 4 * 4 * WS_BINS;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_xgain_frames, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    init = true;
  }
  k_xgain_frames<<<dim3(nframes, n_samples), 2 * (WS_NFFT / 16), smem, s>>>(
      u_rows, u_stride, t_rows, t_stride, row_of_sample, n_trows, pitch, nframes,
      reinterpret_cast<const float*>(n->ws + L.melw), reinterpret_cast<const int2_*>(n->ws + L.melrng),
      reinterpret_cast<const float2_*>(n->ws + L.tw), reinterpret_cast<const float2_*>(n->ws + L.ptw), fr);
  k_xgain_pool<<<(n_samples * WS_MEL * WS_T + 255) / 256, 256, 0, s>>>(fr, nframes, n_samples, coff, feats);
  return cuda_status();
}

int grafx_ws_forward(grafx_wsnet* n, const float* weights, const float* feats, const int32_t* head_count, int32_t B,
                     float* out, void* stream) {
  if (!n || !weights || !feats || !head_count || !out) return fail(GRAFX_EINVAL, "null argument");
  if (!n->ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_ws_bind)");
  if (B < 1 || B > n->max_batch) return fail(GRAFX_ESHAPE, "batch out of range");
  if (int rc = check_heads(head_count, B)) return rc;
  WsNetLayout L = ws_layout(n, 0);
  auto F = [&](size_t off) { return reinterpret_cast<float*>(n->ws + off); };
  uint32_t* st = reinterpret_cast<uint32_t*>(n->ws + L.status);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rows = B * WS_T;
  const int cin[4] = {WS_IN, WS_CH, WS_CH, WS_CH};
  auto BF = [&](size_t off) { return reinterpret_cast<__nv_bfloat16*>(n->ws + off); };
  __nv_bfloat16* wbf = reinterpret_cast<__nv_bfloat16*>(n->ws + L.wbf);
  auto WB = [&](int j) { return wbf + n->wcp.dst[j]; };  // BF16 weight matrix j
  k_weights_bf16<<<dim3(64, WB_MATS), 256, 0, s>>>(weights, wbf, n->wcp);
  k_feat_bf16<<<B, 256, 0, s>>>(feats, BF(L.fb));
  for (int l = 0; l < 4; ++l) {
    // z = conv(h_{l-1}) + b with h_l = gelu(z) as BF16 in the epilogue (the last layer's
    // GELU is taken by the time mean): A = the activations through a 3-D map (tap shifts
    // along the frames), B = the tap-major weight copy
    const int K = cin[l] * WS_KW;
    CUtensorMap ta, tb;
    if (int rc = map_act(&ta, l == 0 ? BF(L.fb) : BF(L.hb[l - 1]), B, cin[l], 4)) return rc;
    if (int rc = map_k2(&tb, WB(l), WS_CH, K)) return rc;
    GemmArgs a = prod_args(rows, WS_CH, K, F(L.z[l]), WS_CH);
    a.bias = weights + n->off[l][1];
    if (l < 3) a.cb = BF(L.hb[l]), a.ldcb = WS_CH, a.act = 1;
    if (int rc = gemm_tma<TM_K3, TM_K2>(a, ta, tb, TmaGeom{cin[l], 1, 0, 0}, nullptr, 0, st, s)) return rc;
  }
  k_time_mean<<<(B * WS_CH + 255) / 256, 256, 0, s>>>(F(L.z[3]), B, BF(L.eb));
  cudaMemsetAsync(out, 0, sizeof(float) * size_t(B) * WS_OUTMAX, s);
  // the heads, each product of all heads in one launch: a1 = e W1^T + b1 (g1 = gelu(a1)
  // as BF16), a2 = g1 W2^T + b2 (g2), out = g2 W3^T + b3
  TmaGroup f1{}, f2{}, f3{};
  int r0 = 0;
  for (int h = 0; h < WS_NHEAD; ++h) {
    const int nb = head_count[h];
    if (nb == 0) continue;
    const int64_t* o = n->hoff[h];
    __nv_bfloat16 *g1 = BF(L.g1b) + r0 * WS_HID, *g2 = BF(L.g2b) + r0 * WS_HID;
    if (int rc = map_k2(&f1.ta[h], BF(L.eb) + r0 * WS_CH, nb, WS_CH)) return rc;
    if (int rc = map_k2(&f1.tb[h], WB(4 + 3 * h), WS_HID, WS_CH)) return rc;
    f1.g[h] = prod_args(nb, WS_HID, WS_CH, F(L.a1) + r0 * WS_HID, WS_HID);
    f1.g[h].bias = weights + o[1], f1.g[h].cb = g1, f1.g[h].ldcb = WS_HID, f1.g[h].act = 1;
    if (int rc = map_k2(&f2.ta[h], g1, nb, WS_HID)) return rc;
    if (int rc = map_k2(&f2.tb[h], WB(5 + 3 * h), WS_HID, WS_HID)) return rc;
    f2.g[h] = prod_args(nb, WS_HID, WS_HID, F(L.a2) + r0 * WS_HID, WS_HID);
    f2.g[h].bias = weights + o[3], f2.g[h].cb = g2, f2.g[h].ldcb = WS_HID, f2.g[h].act = 1;
    if (int rc = map_k2(&f3.ta[h], g2, nb, WS_HID)) return rc;
    if (int rc = map_k2(&f3.tb[h], WB(6 + 3 * h), kHeadOut[h], WS_HID)) return rc;
    f3.g[h] = prod_args(nb, kHeadOut[h], WS_HID, out + int64_t(r0) * WS_OUTMAX, WS_OUTMAX);
    f3.g[h].bias = weights + o[5];
    r0 += nb;
  }
  if (int rc = gemm_tma_group<TM_K2, TM_K2>(f1, st, s)) return rc;
  if (int rc = gemm_tma_group<TM_K2, TM_K2>(f2, st, s)) return rc;
  if (int rc = gemm_tma_group<TM_K2, TM_K2>(f3, st, s)) return rc;
  return cuda_status();
}

int grafx_ws_backward(grafx_wsnet* n, const float* weights, const float* feats, const int32_t* head_count, int32_t B,
                      const float* d_out, float* d_weights, void* stream) {
  if (!n || !weights || !feats || !head_count || !d_out || !d_weights) return fail(GRAFX_EINVAL, "null argument");
  if (!n->ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_ws_bind)");
  if (B < 1 || B > n->max_batch) return fail(GRAFX_ESHAPE, "batch out of range");
  if (int rc = check_heads(head_count, B)) return rc;
  WsNetLayout L = ws_layout(n, 0);
  auto F = [&](size_t off) { return reinterpret_cast<float*>(n->ws + off); };
  uint32_t* st = reinterpret_cast<uint32_t*>(n->ws + L.status);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(d_weights, 0, sizeof(float) * size_t(n->n_params), s);
  // the BF16 weight copies and activations are the forward's (same weights and batch)
  __nv_bfloat16* wbf = reinterpret_cast<__nv_bfloat16*>(n->ws + L.wbf);
  auto WB = [&](int j) { return wbf + n->wcp.dst[j]; };  // BF16 weight matrix j
  auto BF = [&](size_t off) { return reinterpret_cast<__nv_bfloat16*>(n->ws + off); };
  float* de = F(L.dh);                                 // [B][128]
  float* dh = F(L.dh) + size_t(n->max_batch) * WS_CH;  // [rows][128]
  __nv_bfloat16* dob = BF(L.dob);
  k_to_bf16<<<grid1(int64_t(B) * WS_OUTMAX), 256, 0, s>>>(d_out, B, WS_OUTMAX, WS_OUTMAX, dob, WS_OUTMAX);
  // the heads, each step for all heads in one launch:
  //   dW3 = dO^T g2, db3 = column sums of dO, da2 = (dO W3) gelu'(a2),
  //   dW2 = da2^T g1, db2, da1 = (da2 W2) gelu'(a1), dW1 = da1^T e, db1, de = da1 W1
  TmaGroup w3{}, x2{}, w2{}, x1{}, w1{}, x0{};
  ColsumGroup c3{}, c2{}, c1{};
  int r0 = 0;
  for (int h = 0; h < WS_NHEAD; ++h) {
    const int nb = head_count[h];
    if (nb == 0) continue;
    const int64_t* o = n->hoff[h];
    const int no = kHeadOut[h];
    const __nv_bfloat16* dO = dob + int64_t(r0) * WS_OUTMAX;
    float* da2 = F(L.dsmall) + r0 * WS_HID;
    float* da1 = F(L.dsmall) + size_t(n->max_batch) * WS_HID + r0 * WS_HID;
    __nv_bfloat16* da2b = BF(L.dab) + r0 * WS_HID;
    __nv_bfloat16* da1b = BF(L.dab) + size_t(n->max_batch) * WS_HID + r0 * WS_HID;
    const __nv_bfloat16 *g1 = BF(L.g1b) + r0 * WS_HID, *g2 = BF(L.g2b) + r0 * WS_HID, *e = BF(L.eb) + r0 * WS_CH;
    if (int rc = map_n2(&w3.ta[h], dO, nb, no, WS_OUTMAX)) return rc;
    if (int rc = map_n2(&w3.tb[h], g2, nb, WS_HID)) return rc;
    w3.g[h] = prod_args(no, WS_HID, nb, d_weights + o[4], WS_HID);
    c3.x[h] = d_out + int64_t(r0) * WS_OUTMAX, c3.rows[h] = nb, c3.cols[h] = no, c3.ld[h] = WS_OUTMAX;
    c3.out[h] = d_weights + o[5];
    if (int rc = map_k2(&x2.ta[h], dO, nb, no, WS_OUTMAX)) return rc;
    if (int rc = map_n2(&x2.tb[h], WB(6 + 3 * h), no, WS_HID)) return rc;
    x2.g[h] = prod_args(nb, WS_HID, no, da2, WS_HID);
    x2.g[h].zact = F(L.a2) + r0 * WS_HID, x2.g[h].ldz = WS_HID, x2.g[h].cb = da2b, x2.g[h].ldcb = WS_HID;
    c2.x[h] = da2, c2.rows[h] = nb, c2.cols[h] = WS_HID, c2.ld[h] = WS_HID, c2.out[h] = d_weights + o[3];
    if (int rc = map_n2(&w2.ta[h], da2b, nb, WS_HID)) return rc;
    if (int rc = map_n2(&w2.tb[h], g1, nb, WS_HID)) return rc;
    w2.g[h] = prod_args(WS_HID, WS_HID, nb, d_weights + o[2], WS_HID);
    if (int rc = map_k2(&x1.ta[h], da2b, nb, WS_HID)) return rc;
    if (int rc = map_n2(&x1.tb[h], WB(5 + 3 * h), WS_HID, WS_HID)) return rc;
    x1.g[h] = prod_args(nb, WS_HID, WS_HID, da1, WS_HID);
    x1.g[h].zact = F(L.a1) + r0 * WS_HID, x1.g[h].ldz = WS_HID, x1.g[h].cb = da1b, x1.g[h].ldcb = WS_HID;
    c1.x[h] = da1, c1.rows[h] = nb, c1.cols[h] = WS_HID, c1.ld[h] = WS_HID, c1.out[h] = d_weights + o[1];
    if (int rc = map_n2(&w1.ta[h], da1b, nb, WS_HID)) return rc;
    if (int rc = map_n2(&w1.tb[h], e, nb, WS_CH)) return rc;
    w1.g[h] = prod_args(WS_HID, WS_CH, nb, d_weights + o[0], WS_CH);
    if (int rc = map_k2(&x0.ta[h], da1b, nb, WS_HID)) return rc;
    if (int rc = map_n2(&x0.tb[h], WB(4 + 3 * h), WS_HID, WS_CH)) return rc;
    x0.g[h] = prod_args(nb, WS_CH, WS_HID, de + r0 * WS_CH, WS_CH);
    r0 += nb;
  }
  float* csp = F(L.cspart);
  if (int rc = gemm_tma_group<TM_N2, TM_N2>(w3, st, s)) return rc;
  colsum_group(c3, csp, s);
  if (int rc = gemm_tma_group<TM_K2, TM_N2>(x2, st, s)) return rc;
  colsum_group(c2, csp, s);
  if (int rc = gemm_tma_group<TM_N2, TM_N2>(w2, st, s)) return rc;
  if (int rc = gemm_tma_group<TM_K2, TM_N2>(x1, st, s)) return rc;
  colsum_group(c1, csp, s);
  if (int rc = gemm_tma_group<TM_N2, TM_N2>(w1, st, s)) return rc;
  if (int rc = gemm_tma_group<TM_K2, TM_N2>(x0, st, s)) return rc;

  // the conv layers: dz_l in BF16 alternates between two buffers (a product reads dz_l
  // while its epilogue writes dz_{l-1})
  const int rows = B * WS_T;
  k_time_mean_bwd<<<grid1(int64_t(rows) * WS_CH), 256, 0, s>>>(de, B, dh);
  k_gelu_bwd<<<grid1(int64_t(rows) * WS_CH), 256, 0, s>>>(dh, F(L.z[3]), int64_t(rows) * WS_CH, BF(L.dzb[1]));
  const int cin[4] = {WS_IN, WS_CH, WS_CH, WS_CH};
  for (int l = 3; l >= 0; --l) {
    const int K = cin[l] * WS_KW;
    __nv_bfloat16* dzb = BF(L.dzb[l & 1]);  // dz_l; dh holds it in FP32
    // dW[o][c][tap] = sum_(b,t) dz[b][t][o] h_{l-1}[b][t + tap - 2][c]: M = 128, N = 5 cin
    // (tap-major, stored through the permutation), K = rows; both operands MN-major
    CUtensorMap tz, th;
    if (int rc = map_n2(&tz, dzb, rows, WS_CH)) return rc;
    if (int rc = map_act(&th, l == 0 ? BF(L.fb) : BF(L.hb[l - 1]), B, cin[l], 2)) return rc;
    GemmArgs a = prod_args(WS_CH, K, rows, d_weights + n->off[l][0], K);
    a.perm_cin = cin[l];
    if (int rc = gemm_tma<TM_N2, TM_N3>(a, tz, th, TmaGeom{0, 0, cin[l], 1}, F(L.dbig), WS_DBIG_FLOATS, st, s))
      return rc;
    colsum(dh, rows, WS_CH, WS_CH, d_weights + n->off[l][1], csp, s);
    if (l > 0) {
      // dz_{l-1}[b][t][c] = gelu'(z_{l-1}) sum_(tap, o) dz[b][t - tap + 2][o] W[o][c][tap]:
      // A = dz_l through the 3-D map (shift 2 - tap), B = the transposed tap-major weight
      // copy; FP32 into dh (its last reader, the bias column sums, precedes it on the
      // stream), BF16 into the other buffer
      CUtensorMap tk, tw;
      if (int rc = map_act(&tk, dzb, B, WS_CH, 4)) return rc;
      if (int rc = map_k2(&tw, WB(WB_CONVT + l - 1), cin[l], WS_KW * WS_CH)) return rc;
      GemmArgs d = prod_args(rows, cin[l], WS_KW * WS_CH, dh, cin[l]);
      d.zact = F(L.z[l - 1]), d.ldz = WS_CH, d.cb = BF(L.dzb[(l - 1) & 1]), d.ldcb = WS_CH;
      if (int rc = gemm_tma<TM_K3, TM_K2>(d, tk, tw, TmaGeom{WS_CH, -1, 0, 0}, nullptr, 0, st, s)) return rc;
    }
  }
  return cuda_status();
}

// Row i of x [B][cols] through its head's column statistics (mu, sd: [n_heads][cols]):
// forward (x - mu) / sd, or back mu + sd x; columns at or past n_out[i] are written 0.
__global__ void k_ws_standardise(const float* __restrict__ x, const int32_t* __restrict__ head,
                                 const int32_t* __restrict__ n_out, const float* __restrict__ mu,
                                 const float* __restrict__ sd, int B, int cols, int back, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < int64_t(B) * cols;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(i / cols), col = int(i % cols);
    const int h = head[r];
    const float m = mu[h * cols + col], s = sd[h * cols + col];
    y[i] = col < n_out[r] ? (back ? m + s * x[i] : (x[i] - m) / s) : 0.f;
  }
}

int grafx_ws_standardise(const float* x, const int32_t* head, const int32_t* n_out, const float* mu, const float* sd,
                         int32_t B, int32_t cols, int32_t back, float* y, void* stream) {
  if (!x || !head || !n_out || !mu || !sd || !y) return fail(GRAFX_EINVAL, "null argument");
  if (B < 0 || cols < 1) return fail(GRAFX_ESHAPE, "bad standardisation shape");
  if (B == 0) return GRAFX_OK;
  const int64_t n = int64_t(B) * cols;
  const int g = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_ws_standardise<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, head, n_out, mu, sd, B, cols, back ? 1 : 0, y);
  return cuda_status();
}

int grafx_ws_mse(const float* out, const float* target, const int32_t* n_out, int32_t B, float* loss, float* d_out,
                 void* stream) {
  if (!out || !target || !n_out || !loss || !d_out) return fail(GRAFX_EINVAL, "null argument");
  if (B < 1 || int64_t(B) * WS_OUTMAX > INT32_MAX) return fail(GRAFX_ESHAPE, "bad batch");
  k_ws_mse<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(out, target, n_out, B, loss, d_out);
  return cuda_status();
}

int grafx_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak, const float* B,
                    int64_t sbk, int64_t sbn, float* C, int64_t ldc, float alpha, float beta, float* scratch,
                    int64_t scratch_floats, void* stream) {
  if (!A || !B || !C) return fail(GRAFX_EINVAL, "null argument");
  if (M < 0 || N < 0 || K < 0 || ldc < N || M > 65535 * TC_M || scratch_floats < 0)
    return fail(GRAFX_ESHAPE, "bad GEMM shape");
  if (int rc = gemm(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta, static_cast<cudaStream_t>(stream),
                    scratch, scratch ? scratch_floats : 0))
    return rc;
  return cuda_status();
}

int grafx_ws_sync_status(grafx_wsnet* n, void* stream) {
  if (!n || !n->ws) return fail(GRAFX_ESTATE, "workspace not bound (grafx_ws_bind)");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, cudaGetErrorString(e));
  const WsNetLayout L = ws_layout(n, 0);
  uint32_t st = 0;
  e = cudaMemcpy(&st, n->ws + L.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(GRAFX_ECUDA, cudaGetErrorString(e));
  if (st) {
    cudaMemset(n->ws + L.status, 0, sizeof(st));
    return fail(GRAFX_ETIMEOUT, "a bounded tensor-core wait expired");
  }
  return GRAFX_OK;
}

}  // extern "C"
