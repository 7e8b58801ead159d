// Internal descriptors of the batched persistent NLEM launch.
#pragma once
#include <cuda_runtime.h>

#include "admm_core.cuh"

namespace nlemk {

// One image of a batch as the device sees it (lives in the context workspace).
struct BatchImage {
  const float* img;
  float* out;
  int* iters;
  float* resid;
  int H, W, pitch, patch, S;
  float inv_h2;
  double ih2;
  long long pix_begin;   // index of the image's first pixel in the batch's item order
};

// Launch shape chosen by the autotuner.
struct BatchConfig {
  int variant;       // kernel shape pair (see batch_variant_name)
  int fetch;         // work items taken per queue access
  int ctas_per_sm;   // persistent CTAs per SM
};

struct BatchLaunch {
  const BatchImage* imgs;
  int count;
  long long total;       // items in the batch
  long long stride;      // run items 0, stride, 2*stride, ... (1 = every item; >1 = tuning sample)
  unsigned long long* queue;
  BatchConfig cfg;
  SolveParams prm;
  int init_mode;
  int sm_count;
  cudaStream_t stream;
};

constexpr int kBatchVariants = 2;

int launch_batch(const BatchLaunch& L);          // cudaError_t, or -1 for an unknown variant
int batch_max_points(int patch, int variant);    // 0 when the patch size is not compiled
int batch_tile_fits(int patch, int window);
const char* batch_variant_name(int v, int solver);   // solver: SolveParams::solver (2 = accelerated)

}  // namespace nlemk
