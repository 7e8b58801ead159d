// Device-side generator for the standalone Euclidean-median point batches.
//
// Part of the seeded input generator, not of the method: it fills a [B][n][d] float buffer
// with the same bits as synth.em_points() on the host.  SplitMix64 (Steele, Lea & Flood 2014)
// in counter mode: draw i of the stream with state `key` is mix64(key + (i+1)*GOLDEN).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kOutlierThreshold24 = 1677721u;   // floor(0.1 * 2^24)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t idx) {
  return mix64(key + (idx + 1ull) * kGolden);
}

__global__ void em_points_kernel(uint64_t kv, uint64_t ko, uint64_t kb, long long total,
                                 int d, float* __restrict__ out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x; L < total; L += stride) {
    uint64_t point = (uint64_t)(L / d);
    float v;
    if ((uint32_t)(draw(ko, point) >> 40) < kOutlierThreshold24) {
      v = (draw(kb, (uint64_t)L) >> 63) ? 255.0f : 0.0f;
    } else {
      float k24 = (float)(uint32_t)(draw(kv, (uint64_t)L) >> 40);   // exact (< 2^24)
      v = __fmul_rn(__fmul_rn(k24, 255.0f), 5.9604644775390625e-08f);  // * 2^-24, exact
    }
    out[L] = v;
  }
}

}  // namespace

extern "C" int synth_em_points(uint64_t key_value, uint64_t key_outlier, uint64_t key_bernoulli,
                               long long B, int n, int d, void* out, void* stream) {
  long long total = B * (long long)n * d;
  if (total <= 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (total + 255) / 256;
  long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  em_points_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key_value, key_outlier, key_bernoulli,
                                                                        total, d, (float*)out);
  return (int)cudaGetLastError();
}
