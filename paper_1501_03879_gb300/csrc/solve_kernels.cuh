// EM-ADMM kernel templates: standalone batches of Euclidean-median problems (problem (1), Sec. 1) and
// fused NLEM denoising (Sec. 3, Eq. L1regression).  One CTA solves one problem at a time
// with the register-resident solver of admm_core.cuh and loops over problems.
#pragma once
#include <cuda_runtime.h>

#include "admm_core.cuh"
#include "kernels.h"

namespace nlemk {

// ------------------------------------------------------------------------------------------
// standalone batch: points [B][n][d] and weights [B][n] streamed from HBM into the CTA's
// shared-memory point rows, one problem per CTA iteration
// ------------------------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(C::NT, C::MIN_BLOCKS)
em_batch_kernel(const float* __restrict__ pts_g, const float* __restrict__ w_g, long long B, int n,
                int d, SolveParams prm, const float* __restrict__ x0, float* __restrict__ x_out,
                int* __restrict__ iters_used, float* __restrict__ resid, double* __restrict__ obj64,
                double* __restrict__ kkt64) {
  extern __shared__ float4 smem_raw[];
  Smem<C> sm(reinterpret_cast<float*>(smem_raw));
  const int t = threadIdx.x;
  const int dd = C::D > 0 ? C::D : d;
  for (long long b = blockIdx.x; b < B; b += gridDim.x) {
    const float* P = pts_g + (size_t)b * n * dd;
    const float* Wt = w_g + (size_t)b * n;
    // points -> [j][slice][QA] rows; inactive rows and (for runtime d) phantom slots zero
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
      sm.pts[j * C::DP + sg * C::QA + i] = v;
    }
    for (int j = t; j < C::CAP; j += C::NT) {
      float lam = 0.f;
      if (j < n) {
        const float w = __ldg(Wt + j);
        bad |= !(w >= 0.f) || !isfinite(w);
        lam = w * prm.inv_mu;
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
        const float z = slot < real ? clampf(__ldg(x0 + (size_t)b * dd + sg * C::Q + slot), prm.lo, prm.hi) : 0.f;
        sm.zv[i] = z;
        sm.cv[i] = z;
        sm.sgv[i] = 0.f;
      }
      __syncthreads();
    } else {
      float wreg[C::P];
      const int pg = lane_group<C>();
#pragma unroll
      for (int p = 0; p < C::P; ++p) {
        const int j = pg + p * C::NG;
        wreg[p] = j < n ? __ldg(Wt + j) : 0.f;
      }
      weighted_mean_start<C>(sm, wreg, n, dd, prm);
    }
    admm_iterate<C>(sm, n, dd, prm);
    for (int q = t; q < dd; q += C::NT) {
      const int sg = q / C::Q, i = q - sg * C::Q;
      x_out[(size_t)b * dd + q] = sm.zv[sg * C::QA + i];
    }
    if (t == 0) {
      if (iters_used) iters_used[b] = (int)sm.scal[2];
      if (resid) resid[b] = sm.scal[3];
    }
    if (obj64 || kkt64) {
      double F, R;
      fp64_check<C>(sm, n, dd, prm, [&](int j) { return (double)__ldg(Wt + j); }, F, R);
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
// Ends with a barrier, so the caller may start the next pixel at once.
// Warm-start features of one NLEM problem: [m (d), q (d), H, pmax] with p = w / sum w,
// m = sum p a (not projected), q = coordinate-wise lower weighted median (the smallest value
// whose cumulative weight reaches half the total), H = -sum p ln p, pmax = max p.
//
// The medians use the structure of NLEM: coordinate c = (pr, pc) of window point j = (jr, jc)
// is the tile value at (jr + pr, jc + pc), so every coordinate's values are a shifted copy of
// one tile.  The tile is sorted once (bitonic on 64-bit keys: order-preserving value bits,
// then position); for each coordinate the weights are summed along that order by reading
// the window's weight map shifted by c (a zero border makes positions outside the shifted
// window weigh 0).  Weights are summed exactly, as 64-bit fixed point with 54 fraction bits
// (w <= 1 and n <= 441 keep every sum below 2^63): thread t sums ranks [RPT t, RPT t + RPT),
// a block-wide prefix scan gives each thread the weight before its run, and the one thread
// whose run crosses half the total re-walks it.  Scratch reuses the solver's carve (the
// reduction rows hold the keys, the point rows the weight map), so the caller's point rows,
// tile and reduction rows are overwritten.  Ends with a barrier.
constexpr int kFeatSort = 1024;                            // sorted entries (tile <= 32 x 32)

__device__ __forceinline__ unsigned long long feat_key(float v, int u) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // ascending float order
  return ((unsigned long long)o << 32) | (unsigned int)u;
}
__device__ __forceinline__ float feat_value(unsigned long long k) {
  const unsigned int o = (unsigned int)(k >> 32);
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Weighted medians of coordinates [C0, C0 + CN) from the sorted tile keys and the fixed-point
// weight map (see features_nlem): per-thread run sums, a block-wide prefix scan, and a
// re-walk of the run that crosses half the total.  scratch: (NW + 2) * CN 64-bit words.
// Starts and ends with a barrier.
template <class C, int K, int C0, int CN>
__device__ void feat_medians(const unsigned long long* __restrict__ keys, const unsigned long long* __restrict__ wmap,
                             unsigned long long* __restrict__ scratch, int NTILE, int TC, int MC,
                             float* __restrict__ fout) {
  constexpr int D = C::D;
  constexpr int RPT = kFeatSort / C::NT;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  __syncthreads();
  // this thread's run sums for every coordinate of the chunk
  unsigned long long acc[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) acc[c] = 0ull;
  for (int r = t * RPT; r < t * RPT + RPT; ++r) {
    const int u = (int)(unsigned int)keys[r];
    if (u >= NTILE) break;                                  // padding sorts last
    const int ur = u / TC, uc = u - ur * TC;
    // coordinate (pr, pc) reads map entry (ur - pr + K-1, uc - pc + K-1)
    const unsigned long long* base = wmap + (ur + K - 1) * MC + (uc + K - 1);
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[c] += base[-((C0 + c) / K) * MC - ((C0 + c) % K)];
  }
  // block-wide prefix of the run sums (warp shuffles, then warp totals)
  unsigned long long incl[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) incl[c] = acc[c];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const unsigned long long v = __shfl_up_sync(kFull, incl[c], o);
      if (lane >= o) incl[c] += v;
    }
  }
  unsigned long long* wtot = scratch;                       // [NW][CN]
  unsigned long long* xlo = scratch + C::NW * CN;           // [CN] weight before the crossing run
  int* xrun = reinterpret_cast<int*>(xlo + CN);              // [CN] thread owning that run
  if (lane == 31) {
#pragma unroll
    for (int c = 0; c < CN; ++c) wtot[warp * CN + c] = incl[c];
  }
  __syncthreads();
  // every coordinate sums the same n weights, so one total serves all; the thread whose run
  // crosses half records it (acc and incl are indexed at compile time only, so they stay in
  // registers)
  unsigned long long total = 0ull;
  for (int w = 0; w < C::NW; ++w) total += wtot[w * CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) {
    unsigned long long before = 0ull;
    for (int w = 0; w < warp; ++w) before += wtot[w * CN + c];
    const unsigned long long lo = before + incl[c] - acc[c];   // weight before this run
    const unsigned long long hi = before + incl[c];            // weight through this run
    if (2ull * lo < total && 2ull * hi >= total) {
      xlo[c] = lo;
      xrun[c] = t;
    }
  }
  __syncthreads();
  // one thread per coordinate re-walks the crossing run
  for (int c = t; c < CN; c += C::NT) {
    const int pr = (C0 + c) / K, pc = (C0 + c) % K, run = xrun[c];
    unsigned long long cum = xlo[c];
    float med = 0.f;
    for (int r = run * RPT; r < run * RPT + RPT; ++r) {
      const unsigned long long k = keys[r];
      const int u = (int)(unsigned int)k;
      if (u >= NTILE) break;
      const int ur = u / TC, uc = u - ur * TC;
      cum += wmap[(ur - pr + K - 1) * MC + (uc - pc + K - 1)];
      med = feat_value(k);
      if (2ull * cum >= total) break;
    }
    fout[D + C0 + c] = med;
  }
  __syncthreads();
}

template <class C, int K>
__device__ void features_nlem(Smem<C>& sm, const float (&wreg)[C::P], int n, int nwr, int nwc,
                              float* __restrict__ fout) {
  constexpr int D = C::D, HK = (K - 1) / 2;
  constexpr int RPT = kFeatSort / C::NT;                    // ranks per thread
  static_assert(kFeatSort % C::NT == 0, "ranks split evenly over the threads");
  static_assert(2 * kFeatSort <= C::SZ_WRED, "sort keys must fit the reduction rows");
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int TR = nwr + 2 * HK, TC = nwc + 2 * HK, NTILE = TR * TC;
  const int MC = nwc + 2 * (K - 1), MR = nwr + 2 * (K - 1);   // weight map [MR][MC]
  __shared__ unsigned int s_wmax;
  __shared__ float s_W, s_WlnW;
  if (t == 0) s_wmax = 0u;
  __syncthreads();
  // (1) weighted mean, entropy and largest weight
  {
    const int g = lane_slice<C>(), pg = lane_group<C>();
    const bool last = (g == C::G - 1);
    float acc[C::QR];
#pragma unroll
    for (int i = 0; i < C::QR; ++i) acc[i] = 0.f;
#pragma unroll
    for (int p = 0; p < C::P; ++p) {
      const int j = pg + p * C::NG;
      float a[C::Q];
      load_slice<C>(sm.pts + j * C::DP + g * C::QA, last, a);
      const float w = wreg[p];
#pragma unroll
      for (int q = 0; q < C::Q; ++q) acc[q] = fmaf(w, a[q], acc[q]);
      if (g == 0) {
        acc[C::Q] += w;
        acc[C::Q + 1] += w > 0.f ? w * logf(w) : 0.f;
        atomicMax(&s_wmax, __float_as_uint(w));   // w >= 0: integer order is float order
      }
    }
    float4 t0, t1;
    block_reduce<C>(sm, acc, t0, t1);
    if (warp == 0) {
      constexpr int cq = C::Q / 4;
      float vW = lane == cq ? f4get(t0, C::Q - 4 * cq) : 0.f;
      float vL = 0.f;
      {
        const int col1 = (C::Q + 1) / 4;
        const int sl1 = (C::Q + 1) - 4 * col1;
        if (lane == col1) vL = f4get(t0, sl1);
      }
      vW = warp_sum(vW);
      vL = warp_sum(vL);
      if (lane == 0) {
        s_W = vW;
        s_WlnW = vL;
      }
      __syncwarp();
      const float inv = 1.f / vW;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int col = lane + 32 * h2;
        if (col >= C::COLS) continue;
        const float4 tv = h2 == 0 ? t0 : t1;
        const int sg = col / C::NQR, quad = col - sg * C::NQR;
        const int real = slice_real<C>(sg, D);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int slot = 4 * quad + i;
          if (slot < real) fout[sg * C::Q + slot] = f4get(tv, i) * inv;
        }
      }
    }
    __syncthreads();
    if (t == 0) {
      const float W = s_W;
      fout[2 * D] = logf(W) - s_WlnW / W;
      fout[2 * D + 1] = __uint_as_float(s_wmax) / W;
    }
  }
  // (2) sort keys of the tile: tile position u = (ur, uc) is coordinate (ur - jr, uc - jc) of
  // window point (jr, jc) = (min(ur, nwr-1), min(uc, nwc-1)); values read from the point rows
  unsigned long long kv[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int u = t + i * C::NT;
    float v = __int_as_float(0x7f800000);                   // padding sorts last
    if (u < NTILE) {
      const int ur = u / TC, uc = u - ur * TC;
      const int jr = min(ur, nwr - 1), jc = min(uc, nwc - 1);
      const int q = (ur - jr) * K + (uc - jc);
      v = sm.pts[(jr * nwc + jc) * C::DP + (q / C::Q) * C::QA + (q % C::Q)];
    }
    kv[i] = feat_key(v, u);
  }
  __syncthreads();                                          // point rows and tile are now scratch
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(sm.wred);
  unsigned long long* wmap = reinterpret_cast<unsigned long long*>(sm.pts);
#pragma unroll
  for (int i = 0; i < RPT; ++i) keys[t + i * C::NT] = kv[i];
  for (int i = t; i < MR * MC; i += C::NT) wmap[i] = 0ull;
  __syncthreads();
  for (int j = t; j < n; j += C::NT) {
    const int jr = j / nwc, jc = j - jr * nwc;
    wmap[(jr + K - 1) * MC + jc + K - 1] = __float2ull_rz(sm.lam[j] * 18014398509481984.0f);   // w 2^54
  }
  // (3) bitonic sort, ascending
  for (int kk = 2; kk <= kFeatSort; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      __syncthreads();
      for (int pidx = t; pidx < kFeatSort / 2; pidx += C::NT) {
        const int i = ((pidx & ~(jj - 1)) << 1) | (pidx & (jj - 1)), partner = i + jj;   // jj: power of 2
        const bool asc = (i & kk) == 0;
        const unsigned long long a = keys[i], b = keys[partner];
        if ((a > b) == asc) {
          keys[i] = b;
          keys[partner] = a;
        }
      }
    }
  }
  __syncthreads();
  // (4)-(5) medians, in chunks of at most 49 coordinates (register budget)
  unsigned long long* scratch = wmap + MR * MC;
  feat_medians<C, K, 0, (D < 49 ? D : 49)>(keys, wmap, scratch, NTILE, TC, MC, fout);
  if constexpr (D > 49) feat_medians<C, K, 49, D - 49>(keys, wmap, scratch, NTILE, TC, MC, fout);
}

// FEAT: the features-only variant (its own kernel instance, so the solver's register
// allocation does not carry the feature code).
template <class C, int K, bool FEAT = false>
__device__ void nlem_pixel(Smem<C>& sm, const float* __restrict__ img, int H, int W, int pitch, int S,
                           float inv_h2, double ih2, const SolveParams& prm, int init_mode, long long pix,
                           float* __restrict__ out, int* __restrict__ iters_used, float* __restrict__ resid,
                           double* __restrict__ obj64, double* __restrict__ kkt64,
                           const float* __restrict__ wtab, const PixelExtra& ex, long long item = -1) {
  static_assert(K * K == C::D, "patch size must match the compiled dimension");
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
      const float* grow = img + (size_t)reflect_idx(r0 - HK + tr, H) * pitch;
      for (int tc = lane; tc < TC; tc += 32) sm.tile[tr * TC + tc] = __ldg(grow + reflect_idx(c0 - HK + tc, W));
    }
  }
  for (int i = n * C::DP + t; i < C::CAP * C::DP; i += C::NT) sm.pts[i] = 0.f;
  __syncthreads();
  // patch rows: point j = window position (jr, jc) in row-major order, coordinate q = (qr, qc);
  // a thread per point, its row written as 16-byte quads (slots past Q or d are zero)
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
          v[c] = (slot < C::Q && q < C::D) ? tp[(q / K) * TC + (q % K)] : 0.f;
        }
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
      v = sm.tile[(ir - r0 + qr) * TC + (ic - c0 + qc)];
    }
    sm.pcv[i] = v;
  }
  __syncthreads();
  // weights (same lane layout as the solver)
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
      float w = j < n ? expf(-Dp * inv_h2) : 0.f;
      if (wtab) w = j < n ? __ldg(wtab + pix * (long long)(S * S) + j) : 0.f;   // precomputed (BF16 mode)
      wreg[p] = w;
      if (g == 0) sm.lam[j] = w * pp.inv_mu;
    }
  }
  if constexpr (FEAT) {   // features only: no solve
    __syncthreads();
    // feature rows follow the pixel list (row = item), or the image when there is no list
    features_nlem<C, K>(sm, wreg, n, nwr, nwc, ex.feats + (item >= 0 ? item : pix) * (long long)(2 * C::D + 2));
    return;
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
    weighted_mean_start<C>(sm, wreg, n, C::D, pp);
  }
  admm_iterate<C>(sm, n, C::D, pp);
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
        const double e = (double)sm.pcv[sg * C::QA + i] - (double)sm.pts[j * C::DP + sg * C::QA + i];
        D += e * e;
      }
      return exp(-D * ih2);
    };
    fp64_check<C>(sm, n, C::D, pp, wfun, F, Rk);
    if (t == 0) {
      if (obj64) obj64[pix] = F;
      if (kkt64) kkt64[pix] = Rk;
    }
  }
  __syncthreads();
}

template <class C, int K, bool FEAT>
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
    nlem_pixel<C, K, FEAT>(sm, img, H, W, pitch, S, inv_h2, ih2, prm, init_mode, pix, out, iters_used, resid, obj64,
                           kkt64, wtab, ex, it);
  }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <class C>
inline int launch_em(const EmLaunch& L, int grid_mult) {
  auto kern = em_batch_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  long long grid = L.B;
  long long cap = (long long)L.sm_count * C::MIN_BLOCKS * grid_mult;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, C::NT, C::SMEM_BYTES, L.stream>>>(L.pts, L.w, L.B, L.n, L.d, L.prm, L.x0, L.x_out,
                                                          L.iters_used, L.resid, L.obj64, L.kkt64);
  return (int)cudaGetLastError();
}

template <class C, int K>
inline int launch_nlem(const NlemLaunch& L, int grid_mult) {
  if ((L.S + K - 1) * (L.S + K - 1) > C::SZ_WRED) return -1;   // tile must fit its region
  auto kern = L.ex.feats ? nlem_kernel<C, K, true> : nlem_kernel<C, K, false>;
  // the features mode sorts in shared memory past the solver's carve
  // features: the sorted tile and the weight map (+ warp totals) must fit the solver's carve
  if (L.ex.feats && ((L.S + K - 1) * (L.S + K - 1) > kFeatSort ||
                     2 * ((L.S + 2 * (K - 1)) * (L.S + 2 * (K - 1)) + (C::NW + 2) * 49) > C::CAP * C::DP))
    return -1;
  const size_t smem = C::SMEM_BYTES;
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
