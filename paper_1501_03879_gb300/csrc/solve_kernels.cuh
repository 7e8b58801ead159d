// EM-ADMM kernel templates: standalone batches of Euclidean-median problems (problem (1), Sec. 1) and
// fused NLEM denoising (Sec. 3, Eq. L1regression).  One CTA solves one problem at a time
// with the register-resident solver of admm_core.cuh and loops over problems.
#pragma once
#include <cuda_runtime.h>

#include "admm_core.cuh"
#include "debug.h"
#include "fast_core.cuh"
#include "irls_core.cuh"
#include "kernels.h"

namespace nlemk {

// ------------------------------------------------------------------------------------------
// standalone batch: points [B][n][d] and weights [B][n] streamed from HBM into the CTA's
// shared-memory point rows, one problem per CTA iteration
// ------------------------------------------------------------------------------------------
// PJ: the constraint set (ScalarBox = the box of SolveParams; CoordBoxes, Ball from admm_core.cuh).
// WPEN: per-point penalties mu_k = mu w_k (admm_iterate).  FAST: accelerated EM-ADMM
// (admm_fast_iterate, box only; the point rows then hold -a_j and its d-vectors follow the carve).
template <class C, class PJ = ScalarBox, bool WPEN = false, bool FAST = false>
__global__ void __launch_bounds__(C::NT, C::MIN_BLOCKS)
em_batch_kernel(const float* __restrict__ pts_g, const float* __restrict__ w_g, long long B, int n,
                int d, SolveParams prm, const float* __restrict__ x0, float* __restrict__ x_out,
                int* __restrict__ iters_used, float* __restrict__ resid, double* __restrict__ obj64,
                double* __restrict__ kkt64, PJ pj = PJ()) {
  constexpr bool kBox = std::is_same<PJ, ScalarBox>::value;
  static_assert(!FAST || (kBox && !WPEN), "the accelerated solver takes the box and one penalty");
  extern __shared__ float4 smem_raw[];
  Smem<C> sm(reinterpret_cast<float*>(smem_raw));
  const int t = threadIdx.x;
  const int dd = C::D > 0 ? C::D : d;
  for (long long b = blockIdx.x; b < B; b += gridDim.x) {
    const float* P = pts_g + (size_t)b * n * dd;
    const float* Wt = w_g + (size_t)b * n;
    // points -> [j][slice][QA] rows of a_j; inactive rows and (for runtime d) phantom slots zero
    int bad = 0;
    if (C::D == 0) {
      for (int i = t; i < C::CAP * C::DP; i += C::NT) sm.pts[i] = 0.f;
      __syncthreads();
    } else {
      for (int i = n * C::DP + t; i < C::CAP * C::DP; i += C::NT) sm.pts[i] = 0.f;
    }
    for (int idx = t; idx < n * dd; idx += C::NT) {
      const int j = idx / dd, q = idx - j * dd;
      const int sg = q / C::Q, i = q - sg * C::Q;
      const float v = __ldg(P + idx);
      bad |= !isfinite(v);
      const int r = j * C::DP + sg * C::QA + i;
      if (NLEM_DBG_OK(r, C::SZ_PTS, kDbgPointRow)) sm.pts[r] = FAST ? -v : v;
    }
    for (int j = t; j < C::CAP; j += C::NT) {
      float lam = 0.f;
      if (j < n) {
        const float w = __ldg(Wt + j);
        bad |= !(w >= 0.f) || !isfinite(w);
        lam = WPEN ? w : w * prm.inv_mu;
      }
      sm.lam[j] = lam;
    }
    bad = __syncthreads_or(bad);
    if (bad) {
      for (int q = t; q < dd; q += C::NT) x_out[(size_t)b * dd + q] = __int_as_float(0x7fc00000);
      if (t == 0) {
        if (iters_used) iters_used[b] = -1;
        if (resid) resid[b] = __int_as_float(0x7fc00000);
        if (obj64) obj64[b] = __longlong_as_double(0x7ff8000000000000ll);
        if (kkt64) kkt64[b] = __longlong_as_double(0x7ff8000000000000ll);
      }
      __syncthreads();
      continue;
    }
    if (x0) {
      for (int i = t; i < C::VEC; i += C::NT) {
        const int sg = i / C::QA, slot = i - sg * C::QA;
        const int real = slice_real<C>(sg, dd);
        const float xv = slot < real ? __ldg(x0 + (size_t)b * dd + sg * C::Q + slot) : 0.f;
        const float z = kBox ? clampf(xv, prm.lo, prm.hi) : xv;
        sm.zv[i] = z;
        sm.cv[i] = z;
        sm.sgv[i] = 0.f;
      }
      __syncthreads();
      if constexpr (!kBox) {   // any other set: warp 0 projects the whole start vector
        if (t < 32) project_zv<C>(sm, dd, pj);
        __syncthreads();
        for (int i = t; i < C::VEC; i += C::NT) sm.cv[i] = sm.zv[i];
        __syncthreads();
      }
    } else {
      float wreg[C::P];
      const int pg = lane_group<C>();
#pragma unroll
      for (int p = 0; p < C::P; ++p) {
        const int j = pg + p * C::NG;
        wreg[p] = j < n ? __ldg(Wt + j) : 0.f;
      }
      weighted_mean_start<C, NoExchange, PJ, FAST>(sm, wreg, n, dd, prm, pj);
    }
    if constexpr (FAST)
      admm_fast_iterate<C>(sm, FastVec<C>(sm.pts + C::TOTAL), n, dd, prm, prm.restart_every);
    else
      admm_iterate<C, C::G == 2, NoExchange, PJ, WPEN, false>(sm, n, dd, prm, pj);
    for (int q = t; q < dd; q += C::NT) {
      const int sg = q / C::Q, i = q - sg * C::Q;
      x_out[(size_t)b * dd + q] = sm.zv[sg * C::QA + i];
    }
    if (t == 0) {
      if (iters_used) iters_used[b] = (int)sm.scal[2];
      if (resid) resid[b] = sm.scal[3];
    }
    if (kBox && (obj64 || kkt64)) {   // the projected-gradient residual is the box's
      double F, R;
      auto wfun = [&](int j) { return (double)__ldg(Wt + j); };
      fp64_check<C, decltype(wfun), FAST>(sm, n, dd, prm, wfun, F, R);
      if (t == 0) {
        if (obj64) obj64[b] = F;
        if (kkt64) kkt64[b] = R;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// NLEM: one pixel per CTA iteration.  Tile of the reflect-padded image around the clipped
// search window -> patch rows in shared memory -> weights exp(-||P_i-P_j||^2/h^2) -> start
// point -> EM-ADMM -> centre coordinate.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int reflect_idx(int x, int N) {
  return x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x);
}

// One NLEM pixel (Sec. 3, Eq. L1regression) solved by the whole CTA: tile of the
// reflect-padded image around the clipped search window -> patch rows in shared memory ->
// weights exp(-||P_i-P_j||^2/h^2) -> start point -> EM-ADMM -> centre coordinate.
// IRLS: the surrogate solver of Eq. 2 in place of EM-ADMM (NLEM-IRLS, the comparison method of
// Sec. 3).  WPEN: EM-ADMM with per-point penalties mu_k = mu w_k (admm_iterate).  NEG: the point
// rows hold -a_j (admm_core.cuh).  FAST: accelerated EM-ADMM (admm_fast_iterate, rows of -a_j, its
// d-vectors after the carve: the launch adds FastVec<C>::BYTES of shared memory; SCATTER: its
// point norms by reduce-scatter, fast_norms).  Ends with a barrier, so the caller may start the next
// pixel at once.
template <class C, int K, bool IRLS = false, bool WPEN = false, bool NEG = false, bool FAST = false,
          bool SCATTER = false>
__device__ void nlem_pixel(Smem<C>& sm, const float* __restrict__ img, int H, int W, int pitch, int S,
                           float inv_h2, double ih2, const SolveParams& prm, int init_mode, long long pix,
                           float* __restrict__ out, int* __restrict__ iters_used, float* __restrict__ resid,
                           double* __restrict__ obj64, double* __restrict__ kkt64,
                           const float* __restrict__ wtab, const PixelExtra& ex) {
  static_assert(K * K == C::D, "patch size must match the compiled dimension");
  static_assert(!FAST || (NEG && !IRLS && !WPEN), "the accelerated solver reads rows of -a_j, one penalty");
  SolveParams pp = prm;   // the pixel's own penalty when the caller passes one
  if (ex.rho) {
    pp.mu = ex.rho[pix];
    pp.inv_mu = 1.f / pp.mu;
  }
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>();
  const bool last = (g == C::G - 1);
  constexpr int HK = (K - 1) / 2;
  const int R = (S - 1) / 2;
  const int ir = (int)(pix / W), ic = (int)(pix - (long long)ir * W);
  const int r0 = max(ir - R, 0), r1 = min(ir + R, H - 1);
  const int c0 = max(ic - R, 0), c1 = min(ic + R, W - 1);
  const int nwr = r1 - r0 + 1, nwc = c1 - c0 + 1, n = nwr * nwc;
  const int TR = nwr + 2 * HK, TC = nwc + 2 * HK;
  // tile rows r0-HK .. r1+HK, cols c0-HK .. c1+HK of the reflect-padded image (a warp per
  // row, lanes along it)
  {
    const int lane = t & 31, warp = t >> 5;
    for (int tr = warp; tr < TR; tr += C::NW) {
      const long long gr = (long long)reflect_idx(r0 - HK + tr, H) * pitch;
      for (int tc = lane; tc < TC; tc += 32) {
        const long long gi = gr + reflect_idx(c0 - HK + tc, W);
        const float v = NLEM_DBG_OK(gi, (long long)H * pitch, kDbgImageRead) ? __ldg(img + gi) : 0.f;
        if (NLEM_DBG_OK(tr * TC + tc, C::SZ_WRED, kDbgTileWrite)) sm.tile[tr * TC + tc] = v;
      }
    }
  }
  for (int i = n * C::DP + t; i < C::CAP * C::DP; i += C::NT) sm.pts[i] = 0.f;
  __syncthreads();
  // patch rows (of a_j, or -a_j with NEG): point j = window position (jr, jc) in row-major order,
  // coordinate q = (qr, qc); a thread per point, its row written as 16-byte quads (slots past Q or d
  // are zero)
  for (int j = t; j < n; j += C::NT) {
    const int jr = j / nwc, jc = j - jr * nwc;
    const float* tp = sm.tile + jr * TC + jc;
    float4* row = reinterpret_cast<float4*>(sm.pts + j * C::DP);
#pragma unroll
    for (int sg = 0; sg < C::G; ++sg) {
#pragma unroll
      for (int i4 = 0; i4 < C::NQA; ++i4) {
        if (sg * C::QA + 4 * i4 >= C::DP) continue;   // the last slice may be shorter
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int slot = 4 * i4 + c, q = sg * C::Q + slot;
          const int ti = (jr + q / K) * TC + jc + (q % K);
          const float tv = tp[(q / K) * TC + (q % K)];
          v[c] = (slot < C::Q && q < C::D && NLEM_DBG_OK(ti, TR * TC, kDbgTileRead)) ? (NEG ? -tv : tv) : 0.f;
        }
        if (NLEM_DBG_OK(j * C::DP + sg * C::QA + 4 * i4 + 3, C::SZ_PTS, kDbgPointRow))
          row[(sg * C::QA) / 4 + i4] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  }
  // centre patch in slice layout (phantom slots zero)
  for (int i = t; i < C::VEC; i += C::NT) {
    const int sg = i / C::QA, slot = i - sg * C::QA;
    float v = 0.f;
    if (slot < slice_real<C>(sg, C::D)) {
      const int q = sg * C::Q + slot;
      const int qr = q / K, qc = q - qr * K;
      const int ti = (ir - r0 + qr) * TC + (ic - c0 + qc);
      v = NLEM_DBG_OK(ti, TR * TC, kDbgTileRead) ? sm.tile[ti] : 0.f;
    }
    sm.pcv[i] = v;
  }
  __syncthreads();
  // weights (same lane layout as the solver): from the precomputed table in the mixed-precision
  // mode (the FP32 distances are then not formed at all), else exp(-||P_i - P_j||^2 / h^2)
  float wreg[C::P];
  if (wtab) {   // uniform over the CTA
#pragma unroll
    for (int p = 0; p < C::P; ++p) {
      const int j = pg + p * C::NG;
      const float w = j < n ? __ldg(wtab + pix * (long long)(S * S) + j) : 0.f;
      wreg[p] = w;
      if (g == 0) sm.lam[j] = (IRLS || WPEN) ? w : w * pp.inv_mu;
    }
  } else {
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
            const float e = NEG ? pc[q] + f4get(a4, c) : pc[q] - f4get(a4, c);
            if (c & 1) D1 = fmaf(e, e, D1); else D0 = fmaf(e, e, D0);
          }
        }
      }
      const float Dp = point_sum<C>(D0 + D1);
      const float w = j < n ? expf(-Dp * inv_h2) : 0.f;
      wreg[p] = w;
      if (g == 0) sm.lam[j] = (IRLS || WPEN) ? w : w * pp.inv_mu;
    }
  }
  if (ex.x0) {   // caller's start point, projected onto C
    for (int i = t; i < C::VEC; i += C::NT) {
      const int sg = i / C::QA, slot = i - sg * C::QA;
      const float zz = slot < slice_real<C>(sg, C::D)
                           ? clampf(__ldg(ex.x0 + pix * (long long)C::D + sg * C::Q + slot), pp.lo, pp.hi)
                           : 0.f;
      sm.zv[i] = zz;
      sm.cv[i] = zz;
      sm.sgv[i] = 0.f;
    }
    __syncthreads();
  } else if (init_mode == 1) {
    for (int i = t; i < C::VEC; i += C::NT) {
      const float z = clampf(sm.pcv[i], pp.lo, pp.hi);
      const int sg = i / C::QA, slot = i - sg * C::QA;
      const float zz = slot < slice_real<C>(sg, C::D) ? z : 0.f;
      sm.zv[i] = zz;
      sm.cv[i] = zz;
      sm.sgv[i] = 0.f;
    }
    __syncthreads();
  } else {
    __syncthreads();   // lam visible, tile no longer needed (wred aliases it)
    weighted_mean_start<C, NoExchange, ScalarBox, NEG>(sm, wreg, n, C::D, pp);
  }
  if constexpr (IRLS)
    irls_iterate<C, NEG>(sm, n, C::D, pp);
  else if constexpr (FAST)
    admm_fast_iterate<C, SCATTER>(sm, FastVec<C>(sm.pts + C::TOTAL), n, C::D, pp, pp.restart_every);
  else
    admm_iterate<C, false, NoExchange, ScalarBox, WPEN, NEG>(sm, n, C::D, pp);
  if (ex.z_out) {
    for (int q = t; q < C::D; q += C::NT)
      ex.z_out[pix * (long long)C::D + q] = sm.zv[(q / C::Q) * C::QA + (q % C::Q)];
  }
  if (t == 0) {
    constexpr int qc = (C::D - 1) / 2;
    constexpr int sg = qc / C::Q, slot = qc - sg * C::Q;
    out[pix] = sm.zv[sg * C::QA + slot];
    if (iters_used) iters_used[pix] = (int)sm.scal[2];
    if (resid) resid[pix] = sm.scal[3];
  }
  if (obj64 || kkt64) {
    double F, Rk;
    auto wfun = [&](int j) {
      double D = 0.0;
      for (int q = 0; q < C::D; ++q) {
        const int sg = q / C::Q, i = q - sg * C::Q;
        const double a = (double)sm.pts[j * C::DP + sg * C::QA + i];
        const double e = (double)sm.pcv[sg * C::QA + i] + (NEG ? a : -a);
        D += e * e;
      }
      return exp(-D * ih2);
    };
    fp64_check<C, decltype(wfun), NEG>(sm, n, C::D, pp, wfun, F, Rk);
    if (t == 0) {
      if (obj64) obj64[pix] = F;
      if (kkt64) kkt64[pix] = Rk;
    }
  }
  __syncthreads();
}

template <class C, int K, bool IRLS = false, bool WPEN = false, bool FAST = false>
__global__ void __launch_bounds__(C::NT, C::MIN_BLOCKS)
nlem_kernel(const float* __restrict__ img, int H, int W, int pitch, int S, float inv_h2, double ih2,
            SolveParams prm, int init_mode, float* __restrict__ out, int* __restrict__ iters_used,
            float* __restrict__ resid, double* __restrict__ obj64, double* __restrict__ kkt64,
            const float* __restrict__ wtab, const int* __restrict__ pix_list,
            const long long* __restrict__ n_list, PixelExtra ex) {
  extern __shared__ float4 smem_raw[];
  Smem<C> sm(reinterpret_cast<float*>(smem_raw));
  const long long items = pix_list ? *n_list : (long long)H * W;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const long long pix = pix_list ? (long long)pix_list[it] : it;
    // rows of -a_j for the 7-point EM-ADMM shapes of 7x7 patches, measured 3% faster that way (the
    // 4-point shape measured 18% slower and the 9x9 one 0.5%, so the others keep rows of a_j); the
    // accelerated solver always reads rows of -a_j.  Its norms by reduce-scatter measured 1.2% faster
    // here; in the standalone batch and the batched launch they raised register spills and were slower
    constexpr bool kNeg = FAST || (C::P >= 7 && C::D == 49 && !IRLS);
    nlem_pixel<C, K, IRLS, WPEN, kNeg, FAST, FAST>(sm, img, H, W, pitch, S, inv_h2, ih2, prm, init_mode, pix,
                                                   out, iters_used, resid, obj64, kkt64, wtab, ex);
  }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <class C, class PJ = ScalarBox, bool WPEN = false, bool FAST = false>
inline int launch_em(const EmLaunch& L, int grid_mult, const PJ& pj = PJ()) {
  auto kern = em_batch_kernel<C, PJ, WPEN, FAST>;
  const size_t smem = C::SMEM_BYTES + (FAST ? FastVec<C>::BYTES : 0);
  if (smem > 232448) return -1;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  long long grid = L.B;
  long long cap = (long long)L.sm_count * C::MIN_BLOCKS * grid_mult;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, C::NT, smem, L.stream>>>(L.pts, L.w, L.B, L.n, L.d, L.prm, L.x0, L.x_out, L.iters_used,
                                                 L.resid, L.obj64, L.kkt64, pj);
  return (int)cudaGetLastError();
}

template <class C, int K, bool IRLS = false, bool WPEN = false, bool FAST = false>
inline int launch_nlem(const NlemLaunch& L, int grid_mult) {
  if ((L.S + K - 1) * (L.S + K - 1) > C::SZ_WRED) return -1;   // tile must fit its region
  auto kern = nlem_kernel<C, K, IRLS, WPEN, FAST>;
  const size_t smem = C::SMEM_BYTES + (FAST ? FastVec<C>::BYTES : 0);
  if (smem > 232448) return -1;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  long long npix = L.pix_list ? L.max_items : (long long)L.H * L.W;
  long long grid = npix;
  long long cap = (long long)L.sm_count * C::MIN_BLOCKS * grid_mult;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, C::NT, smem, L.stream>>>(L.img, L.H, L.W, L.pitch, L.S, L.inv_h2, L.inv_h2_exact, L.prm,
                                                 L.init_mode, L.out, L.iters_used, L.resid, L.obj64, L.kkt64, L.wtab,
                                                 L.pix_list, L.n_list, L.ex);
  return (int)cudaGetLastError();
}

}  // namespace nlemk
