// Context object behind the nlem_ctx handle of the C ABI (shared by the host-side units).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "batch.h"

// A captured batch: the descriptors and parameters it was built for, the launch shape and the
// instantiated graph (queue reset + persistent launch), which reads the workspace below.
struct BatchPlan {
  std::vector<nlemk::BatchImage> imgs;
  nlemk::SolveParams prm{};
  int init_mode = 0;
  nlemk::BatchConfig cfg{};
  long long total = 0;
  cudaGraphExec_t exec = nullptr;
};

struct nlem_ctx {
  int device = 0;
  int sm_count = 0;
  // double-buffered chunks of the pipelined host-buffer batch solve (grown on demand), the copy
  // stream that fills them, and the events that order buffer reuse
  char* ws_em = nullptr;
  size_t ws_em_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;
  // workspace for the host-buffer entry point (grown on demand, freed by destroy)
  float* ws_img = nullptr;
  float* ws_out = nullptr;
  int* ws_iters = nullptr;
  size_t ws_pixels = 0;
  // workspace of the mixed-precision path: weight table [pixel][window index] and the flag the
  // tensor-core kernel raises if one of its bounded waits runs out
  float* ws_wtab = nullptr;
  size_t ws_wtab_floats = 0;
  int* ws_err = nullptr;
  // workspace of the batched launch: image descriptors and the work-queue counter
  nlemk::BatchImage* ws_batch = nullptr;
  int ws_batch_cap = 0;
  unsigned long long* ws_queue = nullptr;
  cudaStream_t cap_stream = nullptr;                // private stream used for graph capture
  std::map<std::string, nlemk::BatchConfig> tune;   // autotuner results by workload class
  nlemk::BatchConfig forced{-1, 0, 0};              // a launch shape set by nlem_batch_force_config
  BatchPlan plan;
  bool have_plan = false;
  std::string last_cfg;
  // workspace of the warm-started and pixel-list entry points
  float* ws_feats = nullptr;
  float* ws_y = nullptr;
  float* ws_x0 = nullptr;
  float* ws_rho = nullptr;
  int* ws_list = nullptr;
  int* ws_ulist = nullptr;         // a caller's pixel list with the entries outside the image removed
  size_t ws_ulist_cap = 0;
  long long* ws_count = nullptr;   // device element counts: [0] fallback list, [1] caller list
  size_t ws_warm_pixels = 0;
  int ws_warm_d = 0;
  // workspace of the training labels (grown on demand): the grid solves' output and iteration
  // images, the label penalty map, the tight solves' patches [pixel][d], the per-entry best
  // iteration count and penalty, the penalty grid and its counts
  float* lab_out = nullptr;
  size_t lab_out_cap = 0;
  int* lab_iters = nullptr;
  size_t lab_iters_cap = 0;
  float* lab_rho_map = nullptr;
  size_t lab_rho_map_cap = 0;
  float* lab_z = nullptr;
  size_t lab_z_cap = 0;
  int* lab_best_it = nullptr;
  size_t lab_best_it_cap = 0;
  float* lab_best_rho = nullptr;
  size_t lab_best_rho_cap = 0;
  float* lab_grid = nullptr;
  size_t lab_grid_cap = 0;
  unsigned long long* lab_counts = nullptr;
  size_t lab_counts_cap = 0;
};

