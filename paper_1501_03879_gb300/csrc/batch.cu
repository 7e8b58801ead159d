// Batched NLEM over images of uneven sizes in ONE persistent launch (Sec. 3 applied to many
// images at once): every (image, pixel) pair is a work item; CTAs take items from a device
// work queue (one atomic counter in the context workspace) until the queue is empty.  Images
// with 5x5 and 7x7 patches share the launch: the CTA solves each item with a kernel shape
// compiled for that patch size (one per patch size, or one per window-size class), with Algorithm 1 or the
// accelerated solver.  The host side captures queue reset + launch in a CUDA graph and picks the launch
// shape with a small autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "batch.h"
#include "debug.h"
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {

namespace {

// One work item: pixel `pix` of image `im`, solved on shape C (its carve at `base`).
template <class C, int K, bool FAST>
__device__ __forceinline__ void batch_item(float* base, const BatchImage& im, const SolveParams& prm, int init_mode,
                                           long long pix) {
  Smem<C> sm(base);
  nlem_pixel<C, K, false, false, FAST, FAST>(sm, im.img, im.H, im.W, im.pitch, im.S, im.inv_h2, im.ih2, prm,
                                             init_mode, pix, im.out, im.iters, im.resid, nullptr, nullptr, nullptr,
                                             PixelExtra{});
}

// The solver shape of an item: CA (patch KA) or CB (patch KB) for the largest windows, and with
// SIZED the shapes of fewer point slots for smaller windows (CA1 / CA2 up to their capacities for
// patch KA, CB1 for patch KB), so that a small window does not iterate over empty slots.  All
// shapes use the same CTA size; their shared-memory carves alias one buffer (one item at a time).
// FAST: the accelerated solver (admm_fast_iterate) on its shapes, one CTA per SM.
template <class CA, int KA, class CB, int KB, bool SIZED = false, class CA1 = CA, class CA2 = CA, class CB1 = CB,
          bool FAST = false>
__global__ void __launch_bounds__(CA::NT, FAST ? 1 : 2)
nlem_batch_kernel(const BatchImage* __restrict__ imgs, int count, long long total, long long stride,
                  unsigned long long* __restrict__ queue, int fetch, SolveParams prm, int init_mode) {
  static_assert(CA::NT == CB::NT && CA1::NT == CA::NT && CA2::NT == CA::NT && CB1::NT == CB::NT,
                "every shape must use the same CTA size");
  extern __shared__ float4 smem_raw[];
  __shared__ long long s_base;
  for (;;) {
    if (threadIdx.x == 0) s_base = (long long)atomicAdd(queue, (unsigned long long)fetch);
    __syncthreads();
    const long long base = s_base;
    __syncthreads();
    if (base >= total) break;
    const long long end = base + fetch < total ? base + fetch : total;
    for (long long it = base; it < end; ++it) {
      const long long item = it * stride;
      int lo = 0, hi = count - 1;   // last image whose first item is <= item
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].pix_begin <= item) lo = mid; else hi = mid - 1;
      }
      const BatchImage& im = imgs[lo];
      const long long pix = item - im.pix_begin;
      if (!NLEM_DBG_OK(pix, (long long)im.H * im.W, kDbgBatchItem)) continue;
      const int nmax = im.S * im.S;
      float* carve = reinterpret_cast<float*>(smem_raw);
      if (im.patch == KA) {
        if (SIZED && nmax <= CA1::CAP)
          batch_item<CA1, KA, FAST>(carve, im, prm, init_mode, pix);
        else if (SIZED && nmax <= CA2::CAP)
          batch_item<CA2, KA, FAST>(carve, im, prm, init_mode, pix);
        else
          batch_item<CA, KA, FAST>(carve, im, prm, init_mode, pix);
      } else {
        if (SIZED && nmax <= CB1::CAP)
          batch_item<CB1, KB, FAST>(carve, im, prm, init_mode, pix);
        else
          batch_item<CB, KB, FAST>(carve, im, prm, init_mode, pix);
      }
    }
  }
}

template <class C, bool FAST>
constexpr size_t batch_smem() {
  return C::SMEM_BYTES + (FAST ? FastVec<C>::BYTES : 0);
}

template <class CA, int KA, class CB, int KB, bool SIZED = false, class CA1 = CA, class CA2 = CA, class CB1 = CB,
          bool FAST = false>
int launch_variant(const BatchLaunch& L) {
  auto kern = nlem_batch_kernel<CA, KA, CB, KB, SIZED, CA1, CA2, CB1, FAST>;
  const size_t smem = std::max(std::max(batch_smem<CA, FAST>(), batch_smem<CB, FAST>()),
                               std::max(std::max(batch_smem<CA1, FAST>(), batch_smem<CA2, FAST>()),
                                        batch_smem<CB1, FAST>()));
  if (smem > 232448) return -1;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const long long items = (L.total + L.stride - 1) / L.stride;
  long long grid = (long long)L.sm_count * (FAST ? 1 : L.cfg.ctas_per_sm);   // the accelerated shapes fill an SM
  const long long need = (items + L.cfg.fetch - 1) / L.cfg.fetch;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, CA::NT, smem, L.stream>>>(L.imgs, L.count, items, L.stride, L.queue, L.cfg.fetch, L.prm,
                                                   L.init_mode);
  return (int)cudaGetLastError();
}

}  // namespace

int batch_max_points(int patch, int variant) {
  (void)variant;   // both variants hold the largest windows in the same shapes
  if (patch == 7) return E49_7::CAP;
  if (patch == 5) return E25_4::CAP;
  return 0;
}

int batch_tile_fits(int patch, int window) {
  const int k = patch, S = window;
  if (k == 7) return (S + k - 1) * (S + k - 1) <= E49_7::SZ_WRED;
  if (k == 5) return (S + k - 1) * (S + k - 1) <= std::min(E25_4::SZ_WRED, E25_7::SZ_WRED);
  return 0;
}

int launch_batch(const BatchLaunch& L) {
  if (L.prm.solver == 2) {   // accelerated EM-ADMM
    switch (L.cfg.variant) {
      case 0: return launch_variant<F49_7, 7, F25_4, 5, false, F49_7, F49_7, F25_4, true>(L);
      case 1: return launch_variant<F49_7, 7, F25_4, 5, true, F49_2, F49_4, F25_2, true>(L);
      default: return -1;
    }
  }
  switch (L.cfg.variant) {
    case 0: return launch_variant<E49_7, 7, E25_4, 5>(L);
    case 1: return launch_variant<E49_7, 7, E25_4, 5, true, E49_2, E49_4x3, E25_2>(L);
    default: return -1;
  }
}

const char* batch_variant_name(int v, int solver) {
  if (solver == 2) {
    switch (v) {
      case 0: return "accelerated: d49:G4xQ13xP7 + d25:G2xQ13xP4, 256thr, 1 CTA/SM";
      case 1:
        return "accelerated, by window: d49 P2 (n<=128) / P4 (n<=256) / P7 + d25 P2 (n<=256) / P4, 256thr, "
               "1 CTA/SM";
      default: return "?";
    }
  }
  switch (v) {
    case 0: return "d49:G2xQ25xP7/128thr + d25:G1xQ25xP4/128thr";
    case 1: return "by window: d49 P2 (n<=128) / P4 (n<=256) / P7 + d25 P2 (n<=256) / P4, 128thr";
    default: return "?";
  }
}

}  // namespace nlemk
