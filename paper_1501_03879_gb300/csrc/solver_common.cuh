// Definitions shared by the solver kernels (one problem per CTA and pixel pairs): the solve
// parameters of Algorithm 1 and a few small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace nlemk {

constexpr unsigned kFull = 0xffffffffu;

struct SolveParams {
  float lo, hi;        // box C = [lo, hi]^d
  float mu, inv_mu;    // penalty (rho) and its inverse
  int iters;           // iteration cap
  float tol;           // <= 0: fixed count
  int check_every;     // residual check period
  int d;               // runtime dimension (used when D == 0)
  int solver;          // 0 = EM-ADMM (Algorithm 1), 1 = IRLS on the surrogate of Eq. 2, 2 = accelerated EM-ADMM
  float eps;           // IRLS smoothing epsilon of Eq. 2
  int restart_every;   // accelerated EM-ADMM: 0 = restart by the combined-residual test, k > 0 = every k steps
};

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float f4get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

}  // namespace nlemk
