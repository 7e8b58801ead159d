// Internal interface of the learned warm start (model state and its device kernels).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace nlemk {

constexpr int kWsHidden = 128;
constexpr float kDeltaScale = 16.f;    // x0 = P_C(m + kDeltaScale * y[0:d])
constexpr float kLogRhoMin = -12.f;    // rho = exp(clamp(y[d], kLogRhoMin, kLogRhoMax))
constexpr float kLogRhoMax = 4.f;

struct WsModel {
  int d = 0;
  float nref = 441.f;       // entropy normaliser: H / log(nref)
  long long step = 0;       // Adam steps taken
  float* p32 = nullptr;     // FP32 master parameters
  __half* w16 = nullptr;    // FP16 copy read by the forward pass
  float* adam_m = nullptr;
  float* adam_v = nullptr;
};

// Activations and gradients of one training batch (grown on demand).
struct WsScratch {
  long long cap = 0;
  float *y = nullptr, *xs = nullptr, *a1 = nullptr, *a2 = nullptr, *dy = nullptr, *da1 = nullptr, *da2 = nullptr;
  float* grad = nullptr;
};

long long ws_num_params(int d);
int ws_forward(const WsModel& m, const float* feats, long long B, float* y, float* xs, float* a1s, float* a2s,
               int sm_count, cudaStream_t s);
int ws_loss_grad(const WsModel& m, WsScratch& sc, const float* feats, const float* tgt, long long B, float* loss,
                 float* grad, int sm_count, cudaStream_t s);
int ws_adam(WsModel& m, const float* grad, float lr, int sm_count, cudaStream_t s);
int ws_sync_half(WsModel& m, int sm_count, cudaStream_t s);
int ws_apply(const float* feats, const float* y, long long B, int d, float lo, float hi, float* x0, float* rho,
             int sm_count, cudaStream_t s);
// dst[r][c] = src[rows[r]][c] for r < nrows, c < cols (minibatch gather).
int ws_gather_rows(const float* src, int cols, const int* rows, long long nrows, float* dst, int sm_count,
                   cudaStream_t s);
// The entries of in[0, n) that lie in [0, total), compacted into out (any order), their count in
// *count (device).
int ws_compact_list(const int* in, long long n, long long total, int* out, long long* count, int sm_count,
                    cudaStream_t s);
int ws_fallback_list(const int* iters_used, long long npix, int cap, int* list, long long* count, int sm_count,
                     cudaStream_t s);
// Training labels: best_it = INT_MAX, best_rho = 1; the selection after the grid solve with
// penalty rho (iters_img is the solve's [H*W] iteration image); the scatter of the label penalties
// into rho_map (with a count per grid value); the targets [(z* - m) / kDeltaScale, ln rho*].
int ws_label_init(long long n, int* best_it, float* best_rho, int sm_count, cudaStream_t s);
// List entries outside [0, total) are skipped (their targets are NaN).
int ws_label_select(const int* iters_img, long long total, const int* pix, long long n, float rho, int* best_it,
                    float* best_rho, int sm_count, cudaStream_t s);
int ws_label_scatter(const int* pix, long long n, long long total, const float* best_rho, float* rho_map,
                     const float* grid, int n_rho, unsigned long long* counts, int sm_count, cudaStream_t s);
int ws_label_targets(const float* z_full, long long total, const int* pix, long long n, int d, const float* feats,
                     const float* best_rho, float* targets, int sm_count, cudaStream_t s);
int ws_fill(float* p, long long n, float v, int sm_count, cudaStream_t s);

}  // namespace nlemk
