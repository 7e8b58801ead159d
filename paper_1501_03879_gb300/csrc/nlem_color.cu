// NLEM on multichannel images (Sec. 3 with colour patches): the patch of pixel j is the CH
// channels' k x k patches stacked, coordinate q = c*k*k + r*k + s, so d = CH*k*k and
// ||P_i - P_j||^2 sums over every channel.  Each pixel's problem is solved by the same
// register-resident EM-ADMM core as grayscale NLEM; the output is the centre coordinate of every
// channel.
//
// One CTA holds 256 points of d = 147 in registers.  Larger windows split each problem over a
// cluster of two CTAs on neighbouring SMs: CTA r holds window points [256 r, 256 r + 256), both
// keep the full z, c and sum-g vectors, and after every block reduction warp 0 adds the peer's
// column totals, read from the peer's shared memory (distributed shared memory), so that both
// CTAs finalize the same sums and take the same branch at every residual check.
#include <cuda_runtime.h>

#include <type_traits>

#include "admm_core.cuh"
#include "kernels.h"

namespace nlemk {
namespace {

__device__ __forceinline__ int reflect_c(int x, int N) { return x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x); }

// ---- two-CTA clusters -------------------------------------------------------------------
__shared__ float4 x_buf[2][64];   // this CTA's column totals of the last two exchanges
__shared__ unsigned x_phase;      // exchanges so far; its parity picks the buffer

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of both CTAs: release this CTA's shared-memory writes, wait for the peer's.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// 16 bytes from the peer CTA's copy of a shared-memory location.
__device__ __forceinline__ float4 peer_load(const float4* local, unsigned peer) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(peer));
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(ra)
               : "memory");
  return v;
}

// Column totals over the two CTAs of a cluster, added in rank order so that both hold the same bits.
// The buffers alternate: the peer reads exchange k's buffer before it arrives at exchange k+1's
// barrier, which this CTA passes before it writes that buffer again at exchange k+2.
struct PairExchange {
  template <class C>
  __device__ static void combine(float4& t0, float4& t1) {
    static_assert(C::COLS <= 64, "exchange buffer holds 64 columns");
    const int t = threadIdx.x, lane = t & 31;
    const unsigned rank = cluster_rank();
    unsigned p = 0;
    if (t < 32) {
      p = x_phase & 1u;
      if (lane < C::COLS) x_buf[p][lane] = t0;
      if (lane + 32 < C::COLS) x_buf[p][lane + 32] = t1;
    }
    cluster_sync_all();
    if (t < 32) {
      const unsigned peer = rank ^ 1u;
      if (lane < C::COLS) {
        const float4 o = peer_load(&x_buf[p][lane], peer);
        t0 = rank == 0 ? f4add(t0, o) : f4add(o, t0);
      }
      if (lane + 32 < C::COLS) {
        const float4 o = peer_load(&x_buf[p][lane + 32], peer);
        t1 = rank == 0 ? f4add(t1, o) : f4add(o, t1);
      }
      __syncwarp();
      if (lane == 0) x_phase = x_phase + 1u;
      __syncwarp();
    }
  }
};

// One colour pixel solved by the whole CTA (NS = 1) or by the two CTAs of a cluster (NS = 2, this
// CTA holding window points [rank * CAP, rank * CAP + CAP)); ends with a barrier.  img is planar:
// channel c, row r, column s at img[c*cstride + r*pitch + s].
template <class C, int K, int CH, int NS>
__device__ void color_pixel(Smem<C>& sm, const float* __restrict__ img, int H, int W, int pitch, long long cstride,
                            int S, float inv_h2, double ih2, const SolveParams& prm, int init_mode, long long pix,
                            float* __restrict__ out, int* __restrict__ iters_used, float* __restrict__ resid,
                            double* __restrict__ obj64, double* __restrict__ kkt64) {
  static_assert(CH * K * K == C::D, "channels x patch^2 must match the compiled dimension");
  static_assert(NS == 1 || NS == 2, "one CTA or a pair");
  using X = typename std::conditional<NS == 2, PairExchange, NoExchange>::type;
  constexpr int KK = K * K;
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>();
  const bool last = (g == C::G - 1);
  constexpr int HK = (K - 1) / 2;
  const int R = (S - 1) / 2;
  const int ir = (int)(pix / W), ic = (int)(pix - (long long)ir * W);
  const int r0 = max(ir - R, 0), r1 = min(ir + R, H - 1);
  const int c0 = max(ic - R, 0), c1 = min(ic + R, W - 1);
  const int nwr = r1 - r0 + 1, nwc = c1 - c0 + 1, n_all = nwr * nwc;
  const int rank = NS == 2 ? (int)cluster_rank() : 0;
  const int jbase = rank * C::CAP;                               // this CTA's first window point
  const int n = min(max(n_all - jbase, 0), C::CAP);              // points this CTA holds
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
    const int jr = (jbase + j) / nwc, jc = (jbase + j) - jr * nwc;
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
    weighted_mean_start<C, X>(sm, wreg, n, C::D, prm);
  }
  admm_iterate<C, false, X>(sm, n_all, C::D, prm);
  if (t < CH && rank == 0) {
    const int q = t * KK + (KK - 1) / 2;
    out[(long long)t * H * W + pix] = sm.zv[(q / C::Q) * C::QA + (q % C::Q)];
  }
  if (t == 0 && rank == 0) {
    if (iters_used) iters_used[pix] = (int)sm.scal[2];
    if (resid) resid[pix] = sm.scal[3];
  }
  if (NS == 1 && (obj64 || kkt64)) {
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
    color_pixel<C, K, CH, 1>(sm, img, H, W, pitch, cstride, S, inv_h2, ih2, prm, init_mode, it, out, iters_used,
                             resid, obj64, kkt64);
}

// Two CTAs per pixel (a cluster of 2); the pixel loop runs over clusters, so both CTAs of a
// cluster take the same pixels and make the same number of exchanges.  The last cluster barrier
// keeps each CTA's shared memory alive until its peer's final reads are done.
template <class C, int K, int CH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(C::NT, 1)
nlem_color_pair_kernel(const float* __restrict__ img, int H, int W, int pitch, long long cstride, int S,
                       float inv_h2, double ih2, SolveParams prm, int init_mode, float* __restrict__ out,
                       int* __restrict__ iters_used, float* __restrict__ resid) {
  extern __shared__ float4 smem_raw[];
  Smem<C> sm(reinterpret_cast<float*>(smem_raw));
  if (threadIdx.x == 0) x_phase = 0u;
  __syncthreads();
  const long long items = (long long)H * W;
  const long long cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  for (long long it = cl; it < items; it += ncl)
    color_pixel<C, K, CH, 2>(sm, img, H, W, pitch, cstride, S, inv_h2, ih2, prm, init_mode, it, out, iters_used,
                             resid, nullptr, nullptr);
  cluster_sync_all();
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

template <class C, int K, int CH>
int launch_color_pair(const NlemColorLaunch& L) {
  if (L.S * L.S > 2 * C::CAP || L.obj64 || L.kkt64) return -1;
  if (CH * (L.S + K - 1) * (L.S + K - 1) > C::SZ_WRED) return -1;
  auto kern = nlem_color_pair_kernel<C, K, CH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  long long clusters = (long long)L.H * L.W, cap = (long long)L.sm_count * 32;
  if (clusters > cap) clusters = cap;
  if (clusters < 1) clusters = 1;
  kern<<<(unsigned)(2 * clusters), C::NT, C::SMEM_BYTES, L.stream>>>(L.img, L.H, L.W, L.pitch, L.cstride, L.S,
                                                                     L.inv_h2, L.inv_h2_exact, L.prm, L.init_mode,
                                                                     L.out, L.iters_used, L.resid);
  return (int)cudaGetLastError();
}

// three channels: 5x5 patches (d = 75, windows up to 21x21) and 7x7 patches (d = 147, windows up
// to 15x15, the 256 points one CTA's registers hold at this d)
using RGB5 = Cfg<75, 4, 19, 7, 8>;
using RGB7 = Cfg<147, 4, 37, 4, 8, 1>;

}  // namespace

int nlem_color_capacity(int channels, int patch) {
  if (channels == 3 && patch == 5) return RGB5::CAP;
  if (channels == 3 && patch == 7) return 2 * RGB7::CAP;
  return 0;
}

int nlem_color_single_cta_capacity(int channels, int patch) {
  if (channels == 3 && patch == 5) return RGB5::CAP;
  if (channels == 3 && patch == 7) return RGB7::CAP;
  return 0;
}

int launch_nlem_color(const NlemColorLaunch& L) {
  if (L.channels == 3 && L.patch == 5) return launch_color<RGB5, 5, 3>(L);
  if (L.channels == 3 && L.patch == 7)
    return L.S * L.S <= RGB7::CAP ? launch_color<RGB7, 7, 3>(L) : launch_color_pair<RGB7, 7, 3>(L);
  return -1;
}

}  // namespace nlemk
