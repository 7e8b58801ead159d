// Batched NLEM over images of uneven sizes in ONE persistent launch (Sec. 3 applied to many
// images at once): every (image, pixel) pair is a work item; CTAs take items from a device
// work queue (one atomic counter in the context workspace) until the queue is empty.  Images
// with 5x5 and 7x7 patches share the launch: the CTA solves each item with the kernel shape
// compiled for that patch size.  The host side captures queue reset + launch in a CUDA graph
// and picks the launch shape with a small autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "batch.h"
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {

namespace {

template <class CA, int KA, class CB, int KB>
__global__ void __launch_bounds__(CA::NT, 2)
nlem_batch_kernel(const BatchImage* __restrict__ imgs, int count, long long total, long long stride,
                  unsigned long long* __restrict__ queue, int fetch, SolveParams prm, int init_mode) {
  static_assert(CA::NT == CB::NT, "both shapes must use the same CTA size");
  extern __shared__ float4 smem_raw[];
  Smem<CA> smA(reinterpret_cast<float*>(smem_raw));   // the two carves share the buffer:
  Smem<CB> smB(reinterpret_cast<float*>(smem_raw));   // one item is solved at a time
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
      if (im.patch == KA) {
        nlem_pixel<CA, KA>(smA, im.img, im.H, im.W, im.pitch, im.S, im.inv_h2, im.ih2, prm, init_mode, pix, im.out,
                           im.iters, im.resid, nullptr, nullptr, nullptr, PixelExtra{});
      } else {
        nlem_pixel<CB, KB>(smB, im.img, im.H, im.W, im.pitch, im.S, im.inv_h2, im.ih2, prm, init_mode, pix, im.out,
                           im.iters, im.resid, nullptr, nullptr, nullptr, PixelExtra{});
      }
    }
  }
}

template <class CA, int KA, class CB, int KB>
int launch_variant(const BatchLaunch& L) {
  auto kern = nlem_batch_kernel<CA, KA, CB, KB>;
  const size_t smem = std::max(CA::SMEM_BYTES, CB::SMEM_BYTES);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const long long items = (L.total + L.stride - 1) / L.stride;
  long long grid = (long long)L.sm_count * L.cfg.ctas_per_sm;
  const long long need = (items + L.cfg.fetch - 1) / L.cfg.fetch;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, CA::NT, smem, L.stream>>>(L.imgs, L.count, items, L.stride, L.queue, L.cfg.fetch, L.prm,
                                                   L.init_mode);
  return (int)cudaGetLastError();
}

}  // namespace

int batch_max_points(int patch, int variant) {
  if (patch == 7) return E49_7::CAP;
  if (patch == 5) return variant == 0 ? E25_4::CAP : E25_7::CAP;
  return 0;
}

int batch_tile_fits(int patch, int window) {
  const int k = patch, S = window;
  if (k == 7) return (S + k - 1) * (S + k - 1) <= E49_7::SZ_WRED;
  if (k == 5) return (S + k - 1) * (S + k - 1) <= std::min(E25_4::SZ_WRED, E25_7::SZ_WRED);
  return 0;
}

int launch_batch(const BatchLaunch& L) {
  switch (L.cfg.variant) {
    case 0: return launch_variant<E49_7, 7, E25_4, 5>(L);
    case 1: return launch_variant<E49_7, 7, E25_7, 5>(L);
    default: return -1;
  }
}

const char* batch_variant_name(int v) {
  switch (v) {
    case 0: return "d49:G2xQ25xP7/128thr + d25:G1xQ25xP4/128thr";
    case 1: return "d49:G2xQ25xP7/128thr + d25:G1xQ25xP7/128thr";
    default: return "?";
  }
}

}  // namespace nlemk
