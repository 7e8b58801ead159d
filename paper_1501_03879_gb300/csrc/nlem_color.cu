// NLEM on multichannel images (Sec. 3 with colour patches): the patch of pixel j is the CH
// channels' k x k patches stacked, coordinate q = c*k*k + r*k + s, so d = CH*k*k and
// ||P_i - P_j||^2 sums over every channel.  Each pixel's problem is solved by the same
// register-resident EM-ADMM core as grayscale NLEM (one pixel per CTA); the output is the
// centre coordinate of every channel.
#include <cuda_runtime.h>

#include "admm_core.cuh"
#include "kernels.h"

namespace nlemk {
namespace {

__device__ __forceinline__ int reflect_c(int x, int N) { return x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x); }

// One colour pixel solved by the whole CTA; ends with a barrier.  img is planar:
// channel c, row r, column s at img[c*cstride + r*pitch + s].
template <class C, int K, int CH>
__device__ void color_pixel(Smem<C>& sm, const float* __restrict__ img, int H, int W, int pitch, long long cstride,
                            int S, float inv_h2, double ih2, const SolveParams& prm, int init_mode, long long pix,
                            float* __restrict__ out, int* __restrict__ iters_used, float* __restrict__ resid,
                            double* __restrict__ obj64, double* __restrict__ kkt64) {
  static_assert(CH * K * K == C::D, "channels x patch^2 must match the compiled dimension");
  constexpr int KK = K * K;
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>();
  const bool last = (g == C::G - 1);
  constexpr int HK = (K - 1) / 2;
  const int R = (S - 1) / 2;
  const int ir = (int)(pix / W), ic = (int)(pix - (long long)ir * W);
  const int r0 = max(ir - R, 0), r1 = min(ir + R, H - 1);
  const int c0 = max(ic - R, 0), c1 = min(ic + R, W - 1);
  const int nwr = r1 - r0 + 1, nwc = c1 - c0 + 1, n = nwr * nwc;
  const int TR = nwr + 2 * HK, TC = nwc + 2 * HK, TS = TR * TC;
  // CH tiles of the reflect-padded image around the clipped window (a warp per row)
  {
    const int lane = t & 31, warp = t >> 5;
    for (int tr = warp; tr < CH * TR; tr += C::NW) {
      const int ch = tr / TR, rr = tr - ch * TR;
      const float* grow = img + ch * cstride + (size_t)reflect_c(r0 - HK + rr, H) * pitch;
      for (int tc = lane; tc < TC; tc += 32) sm.tile[ch * TS + rr * TC + tc] = __ldg(grow + reflect_c(c0 - HK + tc, W));
    }
  }
  for (int i = n * C::DP + t; i < C::CAP * C::DP; i += C::NT) sm.pts[i] = 0.f;
  __syncthreads();
  // patch rows: point j = window position (jr, jc), coordinate q = (channel, qr, qc)
  for (int j = t; j < n; j += C::NT) {
    const int jr = j / nwc, jc = j - jr * nwc;
    const float* tp = sm.tile + jr * TC + jc;
    float4* row = reinterpret_cast<float4*>(sm.pts + j * C::DP);
#pragma unroll
    for (int sg = 0; sg < C::G; ++sg) {
#pragma unroll
      for (int i4 = 0; i4 < C::NQA; ++i4) {
        if (sg * C::QA + 4 * i4 >= C::DP) continue;
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int slot = 4 * i4 + c, q = sg * C::Q + slot;
          const int ch = q / KK, qq = q - ch * KK;
          v[c] = (slot < C::Q && q < C::D) ? tp[ch * TS + (qq / K) * TC + (qq % K)] : 0.f;
        }
        row[(sg * C::QA) / 4 + i4] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  }
  // centre patch in slice layout
  for (int i = t; i < C::VEC; i += C::NT) {
    const int sg = i / C::QA, slot = i - sg * C::QA;
    float v = 0.f;
    if (slot < slice_real<C>(sg, C::D)) {
      const int q = sg * C::Q + slot;
      const int ch = q / KK, qq = q - ch * KK;
      v = sm.tile[ch * TS + (ir - r0 + qq / K) * TC + (ic - c0 + qq % K)];
    }
    sm.pcv[i] = v;
  }
  __syncthreads();
  // weights exp(-||P_i - P_j||^2 / h^2) over all channels
  float wreg[C::P];
  {
    float pc[C::Q];
    load_slice<C>(sm.pcv + g * C::QA, last, pc);
#pragma unroll
    for (int p = 0; p < C::P; ++p) {
      const int j = pg + p * C::NG;
      const float* arow = sm.pts + j * C::DP + g * C::QA;
      float D0 = 0.f, D1 = 0.f;
#pragma unroll
      for (int i = 0; i < C::NQA; ++i) {
        const float4 a4 = load_quad<C>(arow, i, last);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int q = 4 * i + c;
          if (q < C::Q) {
            const float e = pc[q] - f4get(a4, c);
            if (c & 1) D1 = fmaf(e, e, D1); else D0 = fmaf(e, e, D0);
          }
        }
      }
      const float Dp = point_sum<C>(D0 + D1);
      const float w = j < n ? expf(-Dp * inv_h2) : 0.f;
      wreg[p] = w;
      if (g == 0) sm.lam[j] = w * prm.inv_mu;
    }
  }
  if (init_mode == 1) {
    for (int i = t; i < C::VEC; i += C::NT) {
      const int sg = i / C::QA, slot = i - sg * C::QA;
      const float zz = slot < slice_real<C>(sg, C::D) ? clampf(sm.pcv[i], prm.lo, prm.hi) : 0.f;
      sm.zv[i] = zz;
      sm.cv[i] = zz;
      sm.sgv[i] = 0.f;
    }
    __syncthreads();
  } else {
    __syncthreads();   // lam visible, tiles no longer needed (wred aliases them)
    weighted_mean_start<C>(sm, wreg, n, C::D, prm);
  }
  admm_iterate<C>(sm, n, C::D, prm);
  if (t < CH) {
    const int q = t * KK + (KK - 1) / 2;
    out[(long long)t * H * W + pix] = sm.zv[(q / C::Q) * C::QA + (q % C::Q)];
  }
  if (t == 0) {
    if (iters_used) iters_used[pix] = (int)sm.scal[2];
    if (resid) resid[pix] = sm.scal[3];
  }
  if (obj64 || kkt64) {
    double F, Rk;
    auto wfun = [&](int j) {
      double D = 0.0;
      for (int q = 0; q < C::D; ++q) {
        const int sg = q / C::Q, i = q - sg * C::Q;
        const double e = (double)sm.pcv[sg * C::QA + i] - (double)sm.pts[j * C::DP + sg * C::QA + i];
        D += e * e;
      }
      return exp(-D * ih2);
    };
    fp64_check<C>(sm, n, C::D, prm, wfun, F, Rk);
    if (t == 0) {
      if (obj64) obj64[pix] = F;
      if (kkt64) kkt64[pix] = Rk;
    }
  }
  __syncthreads();
}

template <class C, int K, int CH>
__global__ void __launch_bounds__(C::NT, C::MIN_BLOCKS)
nlem_color_kernel(const float* __restrict__ img, int H, int W, int pitch, long long cstride, int S, float inv_h2,
                  double ih2, SolveParams prm, int init_mode, float* __restrict__ out, int* __restrict__ iters_used,
                  float* __restrict__ resid, double* __restrict__ obj64, double* __restrict__ kkt64) {
  extern __shared__ float4 smem_raw[];
  Smem<C> sm(reinterpret_cast<float*>(smem_raw));
  const long long items = (long long)H * W;
  for (long long it = blockIdx.x; it < items; it += gridDim.x)
    color_pixel<C, K, CH>(sm, img, H, W, pitch, cstride, S, inv_h2, ih2, prm, init_mode, it, out, iters_used, resid,
                          obj64, kkt64);
}

template <class C, int K, int CH>
int launch_color(const NlemColorLaunch& L) {
  if (L.S * L.S > C::CAP) return -1;
  if (CH * (L.S + K - 1) * (L.S + K - 1) > C::SZ_WRED) return -1;   // the tiles must fit their region
  auto kern = nlem_color_kernel<C, K, CH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  long long grid = (long long)L.H * L.W, cap = (long long)L.sm_count * C::MIN_BLOCKS * 64;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, C::NT, C::SMEM_BYTES, L.stream>>>(L.img, L.H, L.W, L.pitch, L.cstride, L.S, L.inv_h2,
                                                          L.inv_h2_exact, L.prm, L.init_mode, L.out, L.iters_used,
                                                          L.resid, L.obj64, L.kkt64);
  return (int)cudaGetLastError();
}

// three channels: 5x5 patches (d = 75, windows up to 21x21) and 7x7 patches (d = 147, windows up
// to 15x15, the 256 points one CTA's registers hold at this d)
using RGB5 = Cfg<75, 4, 19, 7, 8>;
using RGB7 = Cfg<147, 4, 37, 4, 8, 1>;

}  // namespace

int nlem_color_capacity(int channels, int patch) {
  if (channels == 3 && patch == 5) return RGB5::CAP;
  if (channels == 3 && patch == 7) return RGB7::CAP;
  return 0;
}

int launch_nlem_color(const NlemColorLaunch& L) {
  if (L.channels == 3 && L.patch == 5) return launch_color<RGB5, 5, 3>(L);
  if (L.channels == 3 && L.patch == 7) return launch_color<RGB7, 7, 3>(L);
  return -1;
}

}  // namespace nlemk
