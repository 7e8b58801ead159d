// FP32 FMA throughput probe: the roofline denominator for the ALU-bound solver kernels.
// Every thread runs 8 independent FMA chains held in registers; nothing touches memory
// inside the timed loop.  FLOPs = 2 per FMA.
#include <cuda_runtime.h>

#include "kernels.h"

namespace nlemk {

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) fma_chain_kernel(float seed, float* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + (float)(threadIdx.x + i);
  const float b = 0.999999f, c = 1e-7f;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

int measure_fp32_peak(int sm_count, double* tflops) {
  float* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 256 * sizeof(float));
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sm_count * 8;   // 8 x 256 threads = 64 warps per SM
  fma_chain_kernel<<<blocks, 256>>>(1.0f, sink);   // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    fma_chain_kernel<<<blocks, 256>>>(1.0f, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return (int)e;
  const double flops = 2.0 * kChains * 8.0 * kIters * 256.0 * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return 0;
}

}  // namespace nlemk
