// Internal launch descriptors shared by the C-ABI layer and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "solver_common.cuh"

namespace nlemk {

struct EmLaunch {
  const float* pts;
  const float* w;
  long long B;
  int n, d;
  SolveParams prm;
  const float* x0;
  float* x_out;
  int* iters_used;
  float* resid;
  double* obj64;
  double* kkt64;
  int sm_count;
  cudaStream_t stream;
  int penalty = 0;       // NLEM_PENALTY_* (1: per-point penalties mu_k = rho w_k)
};

// Optional per-pixel inputs and outputs of the NLEM kernel (all NULL = plain NLEM).
struct PixelExtra {
  const float* x0;      // [pixel][d] start points (projected onto C), or NULL
  const float* rho;     // [pixel] penalties, or NULL for the launch's rho
  float* z_out;         // [pixel][d] full solution patch, or NULL
};

struct NlemLaunch {
  const float* img;
  int H, W, pitch, patch, S;
  float inv_h2;
  double inv_h2_exact;   // 1/h^2 in double, for the FP64 check
  SolveParams prm;
  int init_mode;
  float* out;
  int* iters_used;
  float* resid;
  double* obj64;
  double* kkt64;
  const float* wtab;     // precomputed weights [pixel][window index] or NULL
  const int* pix_list;   // process only these pixels (count in *n_list), or NULL for all
  const long long* n_list;
  long long max_items;   // upper bound of *n_list (sizes the grid)
  PixelExtra ex;
  int layout;            // NLEM_LAYOUT_* of the options (0 = auto)
  int sm_count;
  cudaStream_t stream;
  int penalty = 0;       // NLEM_PENALTY_* (1: per-point penalties mu_k = rho w_k)
};

// Multichannel NLEM: planar image, channel c at img + c*cstride, out [channels][H][W].
struct NlemColorLaunch {
  const float* img;
  int H, W, pitch;
  long long cstride;     // elements between channel planes
  int channels, patch, S;
  float inv_h2;
  double inv_h2_exact;
  SolveParams prm;
  int init_mode;
  float* out;
  int* iters_used;
  float* resid;
  double* obj64;
  double* kkt64;
  int sm_count;
  cudaStream_t stream;
};

// BF16 tensor-core cross terms -> weight table wtab [H*W][S*S]; err set to 1 if an MMA wait
// ran out.  Returns cudaError_t, or -1 for an uncompiled patch size.
// wait_tries: bound on the mbarrier polls per tensor-core chunk (0 = the default); issue_mma = 0
// withholds the tensor-core step so that the bounded wait runs out (timeout self-test only).
int launch_bf16_weights(const float* img, int H, int W, int pitch, int patch, int S, float inv_h2, float* wtab,
                        int* err, cudaStream_t stream, uint32_t wait_tries = 0, int issue_mma = 1);

// Return cudaError_t codes (0 = launched), or -1 when no compiled shape holds the problem.
int launch_em_batch(const EmLaunch& L);
int launch_nlem_fp32(const NlemLaunch& L);
// NLEM-IRLS (L.prm.solver == 1) on the one-pixel kernel, patch 5, 7 or 9.
int launch_nlem_irls(const NlemLaunch& L);
// The pixel-pair kernel (7x7 patches, window <= 21, plain FP32 NLEM over the whole image).
bool nlem_pair_eligible(const NlemLaunch& L);
int launch_nlem_pair_k7(const NlemLaunch& L);
int em_capacity(int d);
int nlem_capacity(int patch);
// Per-point penalties mu_k = rho w_k (compiled for d = 49 standalone problems and 7x7 NLEM
// patches on the one-pixel layout); -1 for any other shape.
int launch_em_wpen_d49(const EmLaunch& L);
int launch_nlem_wpen_k7(const NlemLaunch& L);
// Accelerated EM-ADMM (L.prm.solver == 2, fast ADMM with restart; L.prm.restart_every): standalone
// problems of d = 49 and NLEM with 7x7 patches on the one-pixel layout, up to fast_capacity()
// points; -1 for any other shape.
int launch_em_fast_d49(const EmLaunch& L);
int launch_nlem_fast_k7(const NlemLaunch& L);
int fast_capacity();
// Standalone batch over per-coordinate boxes (kind 1: a = lo, b = hi, device [d]) or the ball
// ||x - a|| <= r (kind 2: a = centre, device [d]); its point capacity for dimension d.
int launch_em_set(const EmLaunch& L, int kind, const float* a, const float* b, float r);
int em_set_capacity(int d);
// Multichannel NLEM (3 channels; patch 5 or 7): the largest window point count, or 0; and the
// largest one CTA holds (larger windows split each pixel over a two-CTA cluster).
int nlem_color_capacity(int channels, int patch);
int nlem_color_single_cta_capacity(int channels, int patch);
int launch_nlem_color(const NlemColorLaunch& L);

// Warm-start features [item][2 patch^2 + 2] of the listed pixels (or all pixels, row-major);
// returns cudaError_t, or -1 for an uncompiled patch or a tile larger than 32 x 32.
int launch_features(const float* img, int H, int W, int pitch, int patch, int S, float inv_h2, const int* pix_list,
                    const long long* n_list, long long max_items, float* feats, int sm_count, cudaStream_t stream);

// Sets the calling thread's message returned by nlem_last_error().
void set_last_error(const char* msg);

// FP32 FMA-chain throughput probe; returns cudaError_t.
int measure_fp32_peak(int sm_count, double* tflops);

}  // namespace nlemk
