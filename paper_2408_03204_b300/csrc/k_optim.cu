// Gradient-descent fitting of processor parameters (the paper's GD application,
// Abstract and Sec. 4): Adam on unconstrained theta, element-wise maps theta -> p to
// the processors' physical parameters, and their chain rule, fused in one kernel.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace grafx {

enum : int8_t {
  MAP_IDENT = 0, MAP_ALPHA = 1, MAP_SOFTPLUS = 2, MAP_RATIO = 3, MAP_NEGSP = 4, MAP_ATTACK = 5,
  MAP_ZRE = 6, MAP_ZIM = 7   // a multitap delay tap's (Re z, Im z): identity maps, updated as a pair
};
// Weight of the delay taps' unit-circle penalty lam (|z| - 1)^2 (Sec. 3 "Multitap delay":
// the paper pulls z towards the unit circle without giving a weight; 1e-2 is a reading).
constexpr float Z_PENALTY = 1e-2f;

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }
__device__ __forceinline__ float softplusf_(float x) { return x > 20.f ? x : log1pf(expf(x)); }

__device__ __forceinline__ float map_param(float th, int code) {
  switch (code) {
    case MAP_ALPHA: return 0.9f + 0.0999f * sigmoidf_(th);
    case MAP_ATTACK: return 0.5f + 0.4999f * sigmoidf_(th);
    case MAP_SOFTPLUS: return softplusf_(th);
    case MAP_RATIO: return 1.f + softplusf_(th);
    case MAP_NEGSP: return -softplusf_(th);
    default: return th;
  }
}

__device__ __forceinline__ float map_slope(float th, int code) {
  const float s = sigmoidf_(th);
  switch (code) {
    case MAP_ALPHA: return 0.0999f * s * (1.f - s);
    case MAP_ATTACK: return 0.4999f * s * (1.f - s);
    case MAP_SOFTPLUS:
    case MAP_RATIO: return s;
    case MAP_NEGSP: return -s;
    default: return 1.f;
  }
}

// theta <- inverse map of p (start of a fit from physical parameters).
__device__ __forceinline__ float unmap_param(float p, int code) {
  switch (code) {
    case MAP_ALPHA: {
      float a = (p - 0.9f) / 0.0999f;
      return logf(a) - log1pf(-a);
    }
    case MAP_ATTACK: {
      float b = (p - 0.5f) / 0.4999f;
      return logf(b) - log1pf(-b);
    }
    case MAP_SOFTPLUS: return p + logf(-expm1f(-p));
    case MAP_RATIO: return (p - 1.f) + logf(-expm1f(-(p - 1.f)));
    case MAP_NEGSP: return -p + logf(-expm1f(p));
    default: return p;
  }
}

// One Adam update of element i with gradient g (dLoss/dtheta).
__device__ __forceinline__ void adam_elem(float* theta, float* m, float* v, float* p, int64_t i, float g, int code,
                                          float b1, float b2, float lr, float eps, float bc1, float bc2) {
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  const float nt = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  m[i] = mi;
  v[i] = vi;
  theta[i] = nt;
  p[i] = map_param(nt, code);
}

// The update direction of one delay tap's z = (zr, zi) from its gradient (gr, gi): the
// 2-vector scaled to unit length (zero stays zero), plus the gradient of the penalty
// Z_PENALTY (|z| - 1)^2, 2 Z_PENALTY (|z| - 1) z / |z| (zero at z = 0).
__device__ __forceinline__ void delay_z_grad(float zr, float zi, float gr, float gi, float* outr, float* outi) {
  const float n = hypotf(gr, gi);
  if (n > 0.f) {
    gr /= n;
    gi /= n;
  } else {
    gr = gi = 0.f;
  }
  const float r = hypotf(zr, zi);
  const float k = r > 0.f ? 2.f * Z_PENALTY * (r - 1.f) / r : 0.f;
  *outr = gr + k * zr;
  *outi = gi + k * zi;
}

__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ gp, float* __restrict__ p, const int8_t* __restrict__ codes,
                       int cols, int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int code = codes[i % cols];
    if (code == MAP_ZIM) continue;   // updated with its Re z partner
    if (code == MAP_ZRE) {
      float gr, gi;
      delay_z_grad(theta[i], theta[i + 1], gp[i], gp[i + 1], &gr, &gi);
      adam_elem(theta, m, v, p, i, gr, MAP_IDENT, b1, b2, lr, eps, bc1, bc2);
      adam_elem(theta, m, v, p, i + 1, gi, MAP_IDENT, b1, b2, lr, eps, bc1, bc2);
      continue;
    }
    adam_elem(theta, m, v, p, i, gp[i] * map_slope(theta[i], code), code, b1, b2, lr, eps, bc1, bc2);
  }
}

// Same update with the step number read from device memory (for a captured fit step
// whose step counter advances on the device); bias corrections in double once per block.
__global__ void k_adam_dev(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ gp, float* __restrict__ p, const int8_t* __restrict__ codes,
                           int cols, int64_t n, float lr, float b1, float b2, float eps,
                           const int32_t* __restrict__ step) {
  __shared__ float bc[2];
  if (threadIdx.x == 0) {
    const int st = max(*step, 1);
    bc[0] = float(1.0 - pow(double(b1), double(st)));
    bc[1] = float(1.0 - pow(double(b2), double(st)));
  }
  __syncthreads();
  const float bc1 = bc[0], bc2 = bc[1];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int code = codes[i % cols];
    if (code == MAP_ZIM) continue;   // updated with its Re z partner
    if (code == MAP_ZRE) {
      float gr, gi;
      delay_z_grad(theta[i], theta[i + 1], gp[i], gp[i + 1], &gr, &gi);
      adam_elem(theta, m, v, p, i, gr, MAP_IDENT, b1, b2, lr, eps, bc1, bc2);
      adam_elem(theta, m, v, p, i + 1, gi, MAP_IDENT, b1, b2, lr, eps, bc1, bc2);
      continue;
    }
    adam_elem(theta, m, v, p, i, gp[i] * map_slope(theta[i], code), code, b1, b2, lr, eps, bc1, bc2);
  }
}

__global__ void k_to_theta(const float* __restrict__ p, const int8_t* __restrict__ codes, int cols, int64_t n,
                           float* __restrict__ theta) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    theta[i] = unmap_param(p[i], codes[i % cols]);
}

}  // namespace grafx

using namespace grafx;

extern "C" int grafx_adam_step(float* theta, float* m, float* v, const float* grad_param, float* param,
                               const int8_t* codes, int32_t cols, int64_t n, int32_t step, float lr, float beta1,
                               float beta2, float eps, void* stream) {
  if (!theta || !m || !v || !grad_param || !param || !codes) return fail(GRAFX_EINVAL, "null argument");
  if (n < 0 || cols < 1 || step < 1) return fail(GRAFX_EINVAL, "need n >= 0, cols >= 1, step >= 1");
  if (n == 0) return GRAFX_OK;
  const float bc1 = float(1.0 - std::pow(double(beta1), step));
  const float bc2 = float(1.0 - std::pow(double(beta2), step));
  const int g = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_adam<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(theta, m, v, grad_param, param, codes, cols, n, lr,
                                                            beta1, beta2, eps, bc1, bc2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRAFX_OK : fail(GRAFX_ECUDA, cudaGetErrorString(e));
}

extern "C" int grafx_adam_step_dev(float* theta, float* m, float* v, const float* grad_param, float* param,
                                   const int8_t* codes, int32_t cols, int64_t n, const int32_t* step, float lr,
                                   float beta1, float beta2, float eps, void* stream) {
  if (!theta || !m || !v || !grad_param || !param || !codes || !step) return fail(GRAFX_EINVAL, "null argument");
  if (n < 0 || cols < 1) return fail(GRAFX_EINVAL, "need n >= 0, cols >= 1");
  if (n == 0) return GRAFX_OK;
  const int g = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_adam_dev<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(theta, m, v, grad_param, param, codes, cols, n, lr,
                                                                beta1, beta2, eps, step);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRAFX_OK : fail(GRAFX_ECUDA, cudaGetErrorString(e));
}

extern "C" int grafx_params_to_theta(const float* param, const int8_t* codes, int32_t cols, int64_t n, float* theta,
                                     void* stream) {
  if (!param || !codes || !theta) return fail(GRAFX_EINVAL, "null argument");
  if (n < 0 || cols < 1) return fail(GRAFX_EINVAL, "need n >= 0, cols >= 1");
  if (n == 0) return GRAFX_OK;
  const int g = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_to_theta<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(param, codes, cols, n, theta);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRAFX_OK : fail(GRAFX_ECUDA, cudaGetErrorString(e));
}
