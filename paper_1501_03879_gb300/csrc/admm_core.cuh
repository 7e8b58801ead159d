// Device core of EM-ADMM (Algorithm 1 of Chaudhury & Ramakrishnan, arXiv 1501.03879, Sec. 2)
// for one problem per CTA, with the per-point ADMM state held in registers.
//
// Reformulation (algebraically equal to Algorithm 1; FP32):
//   Algorithm 1 keeps x_k, y_k (n*d each) and z.  With u_k = y_k / mu, the prox of
//   Eq. (closed-form) at v_k = z - u_k with lam_k = w_k / mu is x_k = v_k - s_k e_k where
//   e_k = v_k - a_k and s_k = min(1, lam_k / ||e_k||).  Writing g_k = s_k e_k (the shrink
//   step), Eq. (updatez) becomes z+ = P_C(z - (1/n) sum_k g_k) and Eq. (updatey) becomes
//   u_k+ = z - z+ - g_k.  Substituting u_k into the next e_k gives
//       e_k(t+1) = c(t) + h_k(t),   c(t) = 2 z(t) - z(t-1),   h_k(t) = g_k(t) - a_k,
//   so the only per-point state is h_k (n*d floats), started at h_k = -a_k with
//   z(-1) = z(0).  One iteration per element is then: e = c + h, ||e||^2 += e*e,
//   sum_g += s*e, h = s*e - a: one FADD and three FFMA, issued as packed FP32 pairs
//   (FADD2 / FFMA2) over consecutive slots, so each instruction serves two coordinates.
//
// Layout: G consecutive lanes share a point; lane g of a group owns coordinate slice
// [g*Q, g*Q+Q) (the last slice may be shorter: phantom slots read as 0).  A lane owns P
// points j = pg + p*NG (pg = its group, NG = groups per CTA), so h[P][Q] lives in registers.
// Points sit in shared memory as [j][slice][QA] float rows (16-byte aligned slices) holding -a_j
// (NEG = true: the update h = s e - a then takes the loaded value as the FMA addend as it is) or
// a_j (NEG = false).  Both give the same arithmetic, bit for bit; the register allocation, and
// with it the speed, differs per kernel, so each kernel takes the sign it measured faster with.
// The d-vector sum over all points uses a two-level shared-memory column reduction; one warp
// then forms z+, c+ and, on check iterations, the relative residuals.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "solver_common.cuh"

namespace nlemk {


__host__ __device__ constexpr int rup4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr int pow2ceil(int x) { return x <= 1 ? 1 : 2 * pow2ceil((x + 1) / 2); }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// D_ > 0: compile-time dimension with the tight point layout; D_ == 0: runtime d <= G*Q
// with a zero-filled full layout.
// MB_ > 0 sets the CTAs per SM the register budget is sized for (default: 2 for 128 threads).
// PAD_: reduction rows RS float4 apart with RS odd, so that a warp's 16-byte row stores and the
// column reads fall in distinct bank quads (an even row stride conflicts).
template <int D_, int G_, int Q_, int P_, int NW_, int MB_ = 0, bool PAD_ = false>
struct Cfg {
  static constexpr int D = D_, G = G_, Q = Q_, P = P_, NW = NW_;
  static constexpr int NT = NW * 32;
  static constexpr int NG = NT / G;                 // point groups per CTA
  static constexpr int CAP = NG * P;                // largest n
  static constexpr int QA = rup4(Q);                // floats per full slice in a point row
  static constexpr int NQA = QA / 4;
  static constexpr int QL = (D > 0) ? (D - (G - 1) * Q) : Q;      // real slots, last slice
  static constexpr int DP0 = (D > 0) ? (G - 1) * QA + rup4(QL) : G * QA;
  // point row stride: DP/4 odd, so 8 consecutive rows read with 16-byte loads hit 8
  // different bank quads (conflict-free shared loads)
  static constexpr int DP = ((DP0 / 4) % 2 == 1) ? DP0 : DP0 + 4;
  static constexpr int LPG = 32 / G;                // lanes of a warp that share one slice
  static constexpr int QR = rup4(Q + 2);            // reduction row: Q sums + 2 scalars
  static constexpr int NQR = QR / 4;
  static constexpr int RS = (PAD_ && NQR % 2 == 0) ? NQR + 1 : NQR;   // reduction row stride (float4)
  static constexpr int COLS = G * NQR;              // float4 columns of a reduction
  static constexpr int VEC = G * QA;                // slice-layout vectors (z, c, ...)
  static constexpr int MIN_BLOCKS = MB_ > 0 ? MB_ : ((NT <= 128) ? 2 : 1);
  static_assert(32 % G == 0, "G must divide the warp");
  static_assert(G <= 4, "a slice must cover at least 8 consecutive lanes");
  static_assert(D == 0 || (QL > 0 && QL <= Q), "bad coordinate split");
  static_assert(COLS <= 64, "finalize handles at most two columns per lane");

  // shared-memory carve (in floats, every region 16-byte aligned)
  static constexpr int OFF_PTS = 0;
  static constexpr int SZ_PTS = CAP * DP + QA;      // + overread pad of the last slice
  static constexpr int OFF_LAM = rup4(OFF_PTS + SZ_PTS);
  static constexpr int OFF_ZV = rup4(OFF_LAM + CAP);
  static constexpr int OFF_CV = OFF_ZV + VEC;
  static constexpr int OFF_SGV = OFF_CV + VEC;
  static constexpr int OFF_PCV = OFF_SGV + VEC;
  static constexpr int OFF_WRED = OFF_PCV + VEC;
  static constexpr int SZ_WRED = NW * 32 * RS * 4;
  static constexpr int OFF_CRED = OFF_WRED + SZ_WRED;
  static constexpr int OFF_SCAL = OFF_CRED + NW * COLS * 4;
  static constexpr int TOTAL = OFF_SCAL + 16;
  static constexpr size_t SMEM_BYTES = (size_t)TOTAL * 4;
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB of shared memory a CTA may use");
  static_assert((CAP + 128) * 2 <= SZ_WRED, "FP64 check scratch must fit the reduction region");
};

template <class C>
struct Smem {
  float* pts;
  float* lam;
  float* zv;
  float* cv;
  float* sgv;
  float* pcv;
  float4* wred;
  float4* cred;
  float* scal;
  float* tile;   // aliases wred (only used before the first reduction)

  __device__ __forceinline__ explicit Smem(float* base)
      : pts(base + C::OFF_PTS), lam(base + C::OFF_LAM), zv(base + C::OFF_ZV), cv(base + C::OFF_CV),
        sgv(base + C::OFF_SGV), pcv(base + C::OFF_PCV),
        wred(reinterpret_cast<float4*>(base + C::OFF_WRED)),
        cred(reinterpret_cast<float4*>(base + C::OFF_CRED)), scal(base + C::OFF_SCAL),
        tile(base + C::OFF_WRED) {}
};

// Lane mapping: slice g = lane / LPG, point group pg = warp * LPG + lane % LPG, so the G lanes
// of a point are LPG apart and every 8-lane phase of a 16-byte shared load reads 8
// consecutive point rows of the same slice.
template <class C>
__device__ __forceinline__ int lane_slice() { return (threadIdx.x & 31) / C::LPG; }
template <class C>
__device__ __forceinline__ int lane_group() { return (threadIdx.x >> 5) * C::LPG + ((threadIdx.x & 31) % C::LPG); }
// sum over the G lanes that share a point
template <class C>
__device__ __forceinline__ float point_sum(float v) {
#pragma unroll
  for (int o = C::LPG; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Real slots of slice g (runtime d when C::D == 0).
template <class C>
__device__ __forceinline__ int slice_real(int g, int d) {
  if (C::D > 0) return g == C::G - 1 ? C::QL : C::Q;
  int r = d - g * C::Q;
  return r < 0 ? 0 : (r > C::Q ? C::Q : r);
}

// Load the Q slots of a slice row (16-byte aligned); phantom slots of the last slice -> 0.
template <class C>
__device__ __forceinline__ void load_slice(const float* row, bool last, float (&a)[C::Q]) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int i = 0; i < C::NQA; ++i) {
    float4 v = r4[i];
    if (4 * i + 0 < C::Q) a[4 * i + 0] = v.x;
    if (4 * i + 1 < C::Q) a[4 * i + 1] = v.y;
    if (4 * i + 2 < C::Q) a[4 * i + 2] = v.z;
    if (4 * i + 3 < C::Q) a[4 * i + 3] = v.w;
  }
  if (C::D > 0) {
#pragma unroll
    for (int i = (C::D > 0 ? C::QL : C::Q); i < C::Q; ++i) a[i] = last ? 0.f : a[i];
  }
}

// One float4 quad (slots 4i..4i+3) of a slice row, phantom slots of the last slice -> 0.
template <class C>
__device__ __forceinline__ float4 load_quad(const float* row, int i, bool last) {
  float4 v = reinterpret_cast<const float4*>(row)[i];
  if (C::D > 0) {
    if (4 * i + 0 >= C::QL && 4 * i + 0 < C::Q && last) v.x = 0.f;
    if (4 * i + 1 >= C::QL && 4 * i + 1 < C::Q && last) v.y = 0.f;
    if (4 * i + 2 >= C::QL && 4 * i + 2 < C::Q && last) v.z = 0.f;
    if (4 * i + 3 >= C::QL && 4 * i + 3 < C::Q && last) v.w = 0.f;
  }
  return v;
}

// Combining the column totals of the CTAs that share one problem.  The default is one CTA per
// problem: nothing to combine.  A type X with the same static member, called by every thread of
// the CTA after the block reduction, replaces warp 0's tot0 / tot1 with the totals over its CTAs.
struct NoExchange {
  template <class C>
  __device__ __forceinline__ static void combine(float4&, float4&) {}
};

// Two-level column reduction of every thread's acc[QR] row over the lanes that share a
// slice.  Returns, in warp 0, the totals of columns lane and lane+32 (float4 each).
// Contains one __syncthreads; wred/cred may be reused after the caller's next barrier.
// Variant for callers that already wrote their row (NQR float4) at wred[(warp*32+lane)*RS].
template <class C, class X = NoExchange>
__device__ __forceinline__ void block_reduce_rows(const Smem<C>& sm, float4& tot0, float4& tot1) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  __syncwarp();
  constexpr int LPG = C::LPG;                              // lanes per slice in a warp
  constexpr int CP2 = pow2ceil(C::COLS);
  constexpr int LPC = CP2 >= 32 ? 1 : 32 / CP2;            // reducer lanes per column
  constexpr int PER = LPG / LPC;                           // rows summed per reducer lane
  const float4* wbase = sm.wred + warp * 32 * C::RS;
#pragma unroll
  for (int c0 = 0; c0 < C::COLS; c0 += 32) {
    const int col = c0 + (CP2 >= 32 ? lane : (lane % CP2));
    const int part = CP2 >= 32 ? 0 : lane / CP2;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col < C::COLS) {
      const int g = col / C::NQR, quad = col - g * C::NQR;
      float4 s1 = s;   // two partial sums halve the dependent-add chain
#pragma unroll
      for (int m = 0; m < PER; m += 2) {
        const int l = g * LPG + part * PER + m;
        s = f4add(s, wbase[l * C::RS + quad]);
        if (m + 1 < PER) s1 = f4add(s1, wbase[(l + 1) * C::RS + quad]);
      }
      s = f4add(s, s1);
    }
#pragma unroll
    for (int o = CP2; o < 32; o <<= 1) {
      s.x += __shfl_xor_sync(kFull, s.x, o);
      s.y += __shfl_xor_sync(kFull, s.y, o);
      s.z += __shfl_xor_sync(kFull, s.z, o);
      s.w += __shfl_xor_sync(kFull, s.w, o);
    }
    if (part == 0 && col < C::COLS) sm.cred[warp * C::COLS + col] = s;
  }
  __syncthreads();
  tot0 = make_float4(0.f, 0.f, 0.f, 0.f);
  tot1 = tot0;
  if (warp == 0) {
#pragma unroll
    for (int w = 0; w < C::NW; ++w) {
      if (lane < C::COLS) tot0 = f4add(tot0, sm.cred[w * C::COLS + lane]);
      if (lane + 32 < C::COLS) tot1 = f4add(tot1, sm.cred[w * C::COLS + lane + 32]);
    }
  }
  X::template combine<C>(tot0, tot1);
}

template <class C, class X = NoExchange>
__device__ __forceinline__ void block_reduce(const Smem<C>& sm, const float (&acc)[C::QR],
                                             float4& tot0, float4& tot1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* my = sm.wred + (warp * 32 + lane) * C::RS;
#pragma unroll
  for (int i = 0; i < C::NQR; ++i)
    my[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
  block_reduce_rows<C, X>(sm, tot0, tot1);
}


// Projection onto the constraint set C of problem (1).  ScalarBox is the box [lo, hi]^d of Sec. 3
// (bounds in SolveParams), clamped per coordinate where each value is formed.  The other sets are
// projected by warp 0, eight values per lane (the lane's two reduction columns), with their
// parameters read through the read-only cache.
struct ScalarBox {};
struct CoordBoxes {                 // prod_q [lo[q], hi[q]] (device arrays of d floats)
  const float* lo;
  const float* hi;
};
struct Ball {                       // {x : ||x - c|| <= r} (device array of d floats, r >= 0)
  const float* c;
  float r;
};

// Warp 0: values v[k] of coordinates q[k] (where ok[k]) onto C; every lane of warp 0 calls it.
__device__ __forceinline__ void project_lane(const CoordBoxes& s, float (&v)[8], const int (&q)[8],
                                             const bool (&ok)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (ok[k]) v[k] = fminf(fmaxf(v[k], __ldg(s.lo + q[k])), __ldg(s.hi + q[k]));
}
__device__ __forceinline__ void project_lane(const Ball& s, float (&v)[8], const int (&q)[8], const bool (&ok)[8]) {
  float c[8], r2 = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c[k] = ok[k] ? __ldg(s.c + q[k]) : 0.f;
    const float e = ok[k] ? v[k] - c[k] : 0.f;
    r2 = fmaf(e, e, r2);
  }
  const float nr = sqrtf(warp_sum(r2));
  const float scale = nr > s.r ? s.r / nr : 1.f;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (ok[k]) v[k] = fmaf(v[k] - c[k], scale, c[k]);
}

// Warp 0: project the vector held in zv (slice layout, phantom slots zero) onto C in place.
template <class C, class PJ>
__device__ __forceinline__ void project_zv(const Smem<C>& sm, int d, const PJ& pj) {
  const int lane = threadIdx.x & 31;
  float v[8];
  int q[8];
  bool ok[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int col = lane + 32 * (k / 4), sg = col / C::NQR, slot = 4 * (col - sg * C::NQR) + (k % 4);
    ok[k] = col < C::COLS && slot < slice_real<C>(sg, d);
    q[k] = sg * C::Q + slot;
    v[k] = ok[k] ? sm.zv[sg * C::QA + slot] : 0.f;
  }
  project_lane(pj, v, q, ok);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int col = lane + 32 * (k / 4), sg = col / C::NQR, slot = 4 * (col - sg * C::NQR) + (k % 4);
    if (ok[k]) sm.zv[sg * C::QA + slot] = v[k];
  }
}

// Weighted sum of the points (sum_j w_j a_j) and sum_j w_j, with w_j = weight of point slot
// j taken from wreg[p] (0 for inactive slots).  Writes z0 = P_C(sum w a / sum w) into zv and
// cv (c(0) = z(0)), zeroes sgv.  If sum w == 0 the plain mean of the n points is used.
template <class C, class X = NoExchange, class PJ = ScalarBox, bool NEG = false>
__device__ void weighted_mean_start(const Smem<C>& sm, const float (&wreg)[C::P], int n, int d,
                                    const SolveParams& prm, const PJ& pj = PJ()) {
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>(), lane = t & 31;
  const bool last = (g == C::G - 1);
  for (int pass = 0; pass < 2; ++pass) {
    float acc[C::QR];
#pragma unroll
    for (int i = 0; i < C::QR; ++i) acc[i] = 0.f;
#pragma unroll
    for (int p = 0; p < C::P; ++p) {
      const int j = pg + p * C::NG;
      float a[C::Q];
      load_slice<C>(sm.pts + j * C::DP + g * C::QA, last, a);
      const float w = pass == 0 ? wreg[p] : (j < n ? 1.f : 0.f);
#pragma unroll
      for (int q = 0; q < C::Q; ++q) acc[q] = fmaf(NEG ? -w : w, a[q], acc[q]);
      if (g == 0) acc[C::Q] += w;
    }
    float4 t0, t1;
    block_reduce<C, X>(sm, acc, t0, t1);
    // every lane of warp 0 learns sum w from the column holding slot Q of slice 0
    __shared__ float s_wsum;
    if (t < 32) {
      constexpr int cq = C::Q / 4;           // column of slot Q in slice 0
      float v = (lane == cq) ? f4get(t0, C::Q - 4 * cq) : 0.f;
      v = warp_sum(v);
      if (lane == 0) s_wsum = v;
    }
    __syncwarp();
    if (t < 32) {
      const float wsum = s_wsum;
      if (pass == 0 && !(wsum > 0.f)) {
        // fall through to the unweighted pass (uniform decision across warp 0)
      } else if constexpr (!std::is_same<PJ, ScalarBox>::value) {
        const float inv = 1.f / wsum;
        float v[8];
        int q[8];
        bool ok[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int col = lane + 32 * (k / 4), sg = col / C::NQR, slot = 4 * (col - sg * C::NQR) + (k % 4);
          ok[k] = col < C::COLS && slot < slice_real<C>(sg, d);
          q[k] = sg * C::Q + slot;
          v[k] = ok[k] ? f4get(k < 4 ? t0 : t1, k % 4) * inv : 0.f;
        }
        project_lane(pj, v, q, ok);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int col = lane + 32 * (k / 4), sg = col / C::NQR, slot = 4 * (col - sg * C::NQR) + (k % 4);
          if (col < C::COLS && slot < C::QA) {
            sm.zv[sg * C::QA + slot] = v[k];
            sm.cv[sg * C::QA + slot] = v[k];
            sm.sgv[sg * C::QA + slot] = 0.f;
          }
        }
      } else {
        const float inv = 1.f / wsum;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int col = lane + 32 * h2;
          if (col >= C::COLS) continue;
          const float4 tv = h2 == 0 ? t0 : t1;
          const int sg = col / C::NQR, quad = col - sg * C::NQR;
          const int real = slice_real<C>(sg, d);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int slot = 4 * quad + i;
            if (slot >= C::QA) continue;
            const float z = slot < real ? clampf(f4get(tv, i) * inv, prm.lo, prm.hi) : 0.f;
            sm.zv[sg * C::QA + slot] = z;
            sm.cv[sg * C::QA + slot] = z;
            sm.sgv[sg * C::QA + slot] = 0.f;
          }
        }
      }
    }
    if (t == 0) sm.scal[1] = (pass == 0 && !(s_wsum > 0.f)) ? 1.f : 0.f;
    __syncthreads();
    if (sm.scal[1] == 0.f) break;
  }
}

// Algorithm 1 from the state set up by the caller: pts (inactive slots zero), lam
// (lam_j = w_j / mu, zero for inactive slots), zv = cv = z(0) (phantom slots zero) and
// sgv = 0.  On return zv holds z; scal[2] = iterations run; scal[3] = last residual.
// SPLIT (two lanes per point only): thread 0 publishes each iteration's check flag, and the two
// lanes of a point split the rsqrt of the step s.  The standalone batch kernel measured 3.6%
// faster with it; the NLEM kernels of one pixel per CTA measured 2-5% slower, so they do not
// take it (the register allocation decides).
// WPEN: per-point penalties mu_k = mu w_k (a penalty per constraint in the augmented Lagrangian
// of Sec. 2).  lam then holds the weights w_j (zero for inactive slots) instead of w_j / mu:
//   s_k = min(1, (1/mu) / ||e_k||) (the prox radius w_k / mu_k = 1/mu; 0 where w_k = 0, whose
//   terms carry weight 0 everywhere), z+ = P_C(z - sum_k w_k g_k / W) with W = sum_k w_k, and
//   the residuals of the stopping rule in the w-weighted norm (n -> W, each point's terms
//   times w_k), so the reformulation above holds with every sum over k weighted by w_k.
// If every weight is zero the weights are taken as 1.
template <class C, bool SPLIT = false, class X = NoExchange, class PJ = ScalarBox, bool WPEN = false, bool NEG = false>
__device__ void admm_iterate(const Smem<C>& sm, int n, int d, const SolveParams& prm, const PJ& pj = PJ()) {
  static_assert(!SPLIT || C::G == 2, "the split rsqrt pairs the two lanes of a point");
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>(), lane = t & 31, warp = t >> 5;
  const bool last = (g == C::G - 1);
  float inv_n = 1.f / (float)n;
  float fn = (float)n;
  if constexpr (WPEN) {   // W = sum_k w_k, the count the weighted sums divide by
    __syncthreads();
    if (t < 32) {
      float sw = 0.f;
      for (int j = lane; j < C::CAP; j += 32) sw += sm.lam[j];
      sw = warp_sum(sw);
      if (lane == 0) sm.scal[8] = sw;
    }
    __syncthreads();
    float W = sm.scal[8];
    if (!(W > 0.f)) {
      for (int j = t; j < n; j += C::NT) sm.lam[j] = 1.f;
      W = (float)n;
      __syncthreads();
    }
    inv_n = 1.f / W;
    fn = W;
  }

  // state h as coordinate pairs (packed FP32: one FADD2 / FFMA2 serves two slots) plus the
  // single last slot when Q is odd
  constexpr int NP2 = C::Q / 2;
  float2 h2[C::P][NP2];
  float h1[C::P];
#pragma unroll
  for (int p = 0; p < C::P; ++p) {
    const int j = pg + p * C::NG;
    float a[C::Q];
    load_slice<C>(sm.pts + j * C::DP + g * C::QA, last, a);
#pragma unroll
    for (int k = 0; k < NP2; ++k) h2[p][k] = NEG ? make_float2(a[2 * k], a[2 * k + 1]) : make_float2(-a[2 * k], -a[2 * k + 1]);
    h1[p] = (C::Q % 2) ? (NEG ? a[C::Q - 1] : -a[C::Q - 1]) : 0.f;
  }

  int it = 0;
  float resid = 0.f;
  // the check schedule (the cap, and every check_every-th iteration with a tolerance).  With
  // SPLIT, thread 0 keeps a countdown in shared memory and publishes each next iteration's flag,
  // so the other threads read a flag instead of each computing a remainder.
  int* si = reinterpret_cast<int*>(sm.scal);
  if constexpr (SPLIT) {
    if (t == 0) {
      const bool periodic = prm.check_every == 1;
      si[7] = periodic ? prm.check_every : prm.check_every - 1;
      si[6] = (1 == prm.iters || (prm.tol > 0.f && periodic)) ? 1 : 0;
    }
    __syncthreads();
  }
  for (it = 1; it <= prm.iters; ++it) {
    const bool check = SPLIT ? si[6] != 0 : (it == prm.iters) || (prm.tol > 0.f && (it % prm.check_every) == 0);
    // phase 1: e = c + h (in place) and squared norms, one float4 of c at a time; the
    // points are innermost so that consecutive FFMA2s feed different norm accumulators
    float s[C::P];
    {
      float2 s2[C::P];
#pragma unroll
      for (int p = 0; p < C::P; ++p) s2[p] = make_float2(0.f, 0.f);
      const float* crow = sm.cv + g * C::QA;
#pragma unroll
      for (int i = 0; i < C::NQA; ++i) {
        const float4 c4 = load_quad<C>(crow, i, last);
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
          const int q0 = 4 * i + 2 * jh;
          if (q0 + 1 < C::Q) {
            const float2 c2 = jh == 0 ? make_float2(c4.x, c4.y) : make_float2(c4.z, c4.w);
#pragma unroll
            for (int p = 0; p < C::P; ++p) {
              h2[p][q0 / 2] = __fadd2_rn(h2[p][q0 / 2], c2);
              s2[p] = __ffma2_rn(h2[p][q0 / 2], h2[p][q0 / 2], s2[p]);
            }
          } else if (q0 < C::Q) {
            const float c1 = jh == 0 ? c4.x : c4.z;
#pragma unroll
            for (int p = 0; p < C::P; ++p) {
              h1[p] += c1;
              s2[p].x = fmaf(h1[p], h1[p], s2[p].x);
            }
          }
        }
      }
#pragma unroll
      for (int p = 0; p < C::P; ++p) s[p] = s2[p].x + s2[p].y;
    }
    // s = min(1, lam / ||e||); r2 = 0 gives lam*inf (or NaN when lam = 0), and fminf then
    // yields 1, which is harmless because e = 0 there.
    float gs = 0.f;
    if constexpr (SPLIT) {
      // the two lanes of a point split the points: a reduce-scatter of the partial norms leaves
      // lane g with the full norm of points 2k+g, which it alone turns into s; the s values are
      // then exchanged (4 rsqrt per lane instead of 7)
      constexpr int PH = (C::P + 1) / 2;
      const bool up = g != 0;
      float sh[PH];
#pragma unroll
      for (int k = 0; k < PH; ++k) {
        const float lo = s[2 * k], hi = 2 * k + 1 < C::P ? s[2 * k + 1] : 0.f;
        const float r2 = (up ? hi : lo) + __shfl_xor_sync(kFull, up ? lo : hi, C::LPG);
        const int p = 2 * k + (up ? 1 : 0);
        const bool valid = p < C::P;
        const float lj = sm.lam[pg + (valid ? p : 0) * C::NG];
        const float lam_k = WPEN ? (lj > 0.f ? prm.inv_mu : 0.f) : lj;
        sh[k] = valid ? fminf(1.f, lam_k * rsqrtf(r2)) : 0.f;
        // each point's ||g_k||^2 once, by its owner (times w_k with per-point penalties)
        gs = fmaf((WPEN ? lj : 1.f) * sh[k] * sh[k], valid ? r2 : 0.f, gs);
      }
#pragma unroll
      for (int k = 0; k < PH; ++k) {
        const float other = __shfl_xor_sync(kFull, sh[k], C::LPG);
        s[2 * k] = up ? other : sh[k];
        if (2 * k + 1 < C::P) s[2 * k + 1] = up ? sh[k] : other;
      }
    } else {
#pragma unroll
      for (int p = 0; p < C::P; ++p) s[p] = point_sum<C>(s[p]);
#pragma unroll
      for (int p = 0; p < C::P; ++p) {
        const float r2 = s[p];
        const float lj = sm.lam[pg + p * C::NG];
        s[p] = fminf(1.f, (WPEN ? (lj > 0.f ? prm.inv_mu : 0.f) : lj) * rsqrtf(r2));
        gs = fmaf((WPEN ? lj : 1.f) * s[p] * s[p], r2, gs);
      }
      if (g != 0) gs = 0.f;    // each point's ||g_k||^2 counted once, by its slice-0 lane
    }
    // the factor of g_k in the sums over k: s_k, or w_k s_k with per-point penalties
    float ws[C::P];
#pragma unroll
    for (int p = 0; p < C::P; ++p) ws[p] = WPEN ? sm.lam[pg + p * C::NG] * s[p] : s[p];
    float dd = 0.f;            // sum_k ||h_k(t) - h_k(t+1)||^2 over this lane's slots
    if (check) {
      // ||(1-s) e + a - c||^2 in a pass of its own; the fences keep the compiler from
      // carrying these loads (or phase 1's) into phase 2, which would exhaust registers
      asm volatile("" ::: "memory");
      const float* crow = sm.cv + g * C::QA;
#pragma unroll
      for (int p = 0; p < C::P; ++p) {
        const float* arow = sm.pts + (pg + p * C::NG) * C::DP + g * C::QA;
        const float oms = 1.f - s[p];
        const float2 oms2 = make_float2(oms, oms), noms2 = make_float2(-oms, -oms);
        float2 dd2 = make_float2(0.f, 0.f);
        float dd1 = 0.f;
#pragma unroll
        for (int i = 0; i < C::NQA; ++i) {
          const float4 a4 = load_quad<C>(arow, i, last);
          const float4 c4 = load_quad<C>(crow, i, last);
#pragma unroll
          for (int jh = 0; jh < 2; ++jh) {
            const int q0 = 4 * i + 2 * jh;
            const float2 a2 = jh == 0 ? make_float2(a4.x, a4.y) : make_float2(a4.z, a4.w);
            const float2 c2 = jh == 0 ? make_float2(c4.x, c4.y) : make_float2(c4.z, c4.w);
            // with rows of -a, (-(1-s)) e + (c - a) is the negated difference, with the same square
            if (q0 + 1 < C::Q) {
              const float2 dq2 = NEG ? __ffma2_rn(noms2, h2[p][q0 / 2], __fadd2_rn(a2, c2))
                                     : __ffma2_rn(oms2, h2[p][q0 / 2], __fadd2_rn(a2, make_float2(-c2.x, -c2.y)));
              dd2 = __ffma2_rn(dq2, dq2, dd2);
            } else if (q0 < C::Q) {
              const float dq = NEG ? fmaf(-oms, h1[p], a2.x + c2.x) : fmaf(oms, h1[p], a2.x - c2.x);
              if constexpr (WPEN)
                dd1 = fmaf(dq, dq, dd1);
              else
                dd = fmaf(dq, dq, dd);
            }
          }
        }
        // per-point penalties weight the point's term by w_k
        if constexpr (WPEN)
          dd = fmaf(sm.lam[pg + p * C::NG], dd1 + (dd2.x + dd2.y), dd);
        else
          dd += dd2.x + dd2.y;
        asm volatile("" ::: "memory");
      }
    }
    // phase 2, one float4 column at a time: sum_k g_k into this lane's reduction row and
    // h = s e - a; only four accumulators are live at once
    {
      float4* my = sm.wred + (warp * 32 + lane) * C::RS;
      const float* abase = sm.pts + pg * C::DP + g * C::QA;
      // two point quads in flight ahead of their use (linear order: quad-major, point-minor)
      float4 a_n1 = load_quad<C>(abase, 0, last);
      float4 a_n2 = C::P > 1 ? load_quad<C>(abase + C::NG * C::DP, 0, last) : load_quad<C>(abase, 1, last);
#pragma unroll
      for (int i = 0; i < C::NQR; ++i) {
        float acc4[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < C::NQA) {
          float2 accp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          float acc1 = 0.f;
#pragma unroll
          for (int p = 0; p < C::P; ++p) {
            const float4 a4 = a_n1;
            a_n1 = a_n2;
            {
              const int lin = i * C::P + p + 2;          // the quad two steps ahead
              const int ni = lin / C::P, np = lin % C::P;
              if (ni < C::NQA) a_n2 = load_quad<C>(abase + np * C::NG * C::DP, ni, last);
            }
            const float2 sp2 = make_float2(s[p], s[p]), wp2 = make_float2(ws[p], ws[p]);
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
              const int q0 = 4 * i + 2 * jh;
              const float2 a2 = jh == 0 ? make_float2(a4.x, a4.y) : make_float2(a4.z, a4.w);
              const float2 na2 = NEG ? a2 : make_float2(-a2.x, -a2.y);
              if (q0 + 1 < C::Q) {
                accp[jh] = __ffma2_rn(wp2, h2[p][q0 / 2], accp[jh]);
                h2[p][q0 / 2] = __ffma2_rn(sp2, h2[p][q0 / 2], na2);
              } else if (q0 < C::Q) {
                acc1 = fmaf(ws[p], h1[p], acc1);
                h1[p] = fmaf(s[p], h1[p], na2.x);
              }
            }
          }
#pragma unroll
          for (int jh = 0; jh < 2; ++jh) {
            const int q0 = 4 * i + 2 * jh;
            if (q0 + 1 < C::Q) {
              acc4[2 * jh] = accp[jh].x;
              acc4[2 * jh + 1] = accp[jh].y;
            } else if (q0 < C::Q) {
              acc4[2 * jh] = acc1;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (4 * i + c == C::Q) acc4[c] = dd;
          if (4 * i + c == C::Q + 1) acc4[c] = gs;
        }
        my[i] = make_float4(acc4[0], acc4[1], acc4[2], acc4[3]);
      }
    }
    float4 t0, t1;
    block_reduce_rows<C, X>(sm, t0, t1);
    // finalize (warp 0): z+ = P_C(z - sum g / n), c+ = 2 z+ - z, residuals on checks
    if (t < 32) {
      if (SPLIT && t == 0) {   // the next iteration's check flag (read by every thread after the barrier)
        const int cnt = si[7];
        const bool periodic = cnt == 1;
        si[7] = periodic ? prm.check_every : cnt - 1;
        si[6] = (it + 1 == prm.iters || (prm.tol > 0.f && periodic)) ? 1 : 0;
      }
      float p_dd = 0.f, p_dS = 0.f, p_zz = 0.f, p_zx = 0.f, p_dz = 0.f, p_dzA = 0.f, p_E = 0.f, p_G = 0.f;
      if constexpr (std::is_same<PJ, ScalarBox>::value) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int col = lane + 32 * h2;
          if (col >= C::COLS) continue;
          const float4 tv = h2 == 0 ? t0 : t1;
          const int sg = col / C::NQR, quad = col - sg * C::NQR;
          const int real = slice_real<C>(sg, d);
          // this lane's four slots of z, c and sum g as one 16-byte access each (slots past the
          // slice's real coordinates stay zero)
          const bool has_z = quad < C::NQA;
          const int vi0 = sg * C::QA + 4 * quad;
          float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f), c4o = z4, s4o = z4;
          if (has_z) {
            z4 = *reinterpret_cast<const float4*>(sm.zv + vi0);
            if (check) {
              c4o = *reinterpret_cast<const float4*>(sm.cv + vi0);
              s4o = *reinterpret_cast<const float4*>(sm.sgv + vi0);
            }
          }
          float zn[4], cn[4], sn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int slot = 4 * quad + i;
            const float A = f4get(tv, i);
            zn[i] = cn[i] = sn[i] = 0.f;
            if (slot < real) {
              const float z = f4get(z4, i);
              const float znew = clampf(fmaf(-A, inv_n, z), prm.lo, prm.hi);
              if (check) {
                const float c = f4get(c4o, i);
                const float sgp = f4get(s4o, i);
                const float del = c - znew;          // delta = c(t) - z(t+1)
                const float SD = sgp - A;            // sum_k (g_k(t) - g_k(t+1))
                const float dz = z - znew;
                p_dd = fmaf(del, del, p_dd);
                p_dS = fmaf(del, SD, p_dS);
                p_zz = fmaf(znew, znew, p_zz);
                p_zx = fmaf(znew, fmaf(fn, del, SD), p_zx);
                p_dz = fmaf(dz, dz, p_dz);
                p_dzA = fmaf(dz, A, p_dzA);
              }
              zn[i] = znew;
              cn[i] = 2.f * znew - z;
              sn[i] = A;
            } else if (slot == C::Q) {
              p_E += A;
            } else if (slot == C::Q + 1) {
              p_G += A;
            }
          }
          if (has_z) {
            *reinterpret_cast<float4*>(sm.zv + vi0) = make_float4(zn[0], zn[1], zn[2], zn[3]);
            *reinterpret_cast<float4*>(sm.cv + vi0) = make_float4(cn[0], cn[1], cn[2], cn[3]);
            *reinterpret_cast<float4*>(sm.sgv + vi0) = make_float4(sn[0], sn[1], sn[2], sn[3]);
          }
        }
      } else {
        // any other set: form v = z - sum g / n for the lane's eight values, project them together,
        // then the same residual terms and stores as above
        float v[8], zo[8], co[8], so[8], Av[8];
        int q[8];
        bool ok[8];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int col = lane + 32 * h2;
          const bool colok = col < C::COLS;
          const float4 tv = h2 == 0 ? t0 : t1;
          const int sg = colok ? col / C::NQR : 0, quad = colok ? col - sg * C::NQR : 0;
          const int real = slice_real<C>(sg, d);
          const bool has_z = colok && quad < C::NQA;
          const int vi0 = sg * C::QA + 4 * quad;
          float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f), c4o = z4, s4o = z4;
          if (has_z) {
            z4 = *reinterpret_cast<const float4*>(sm.zv + vi0);
            if (check) {
              c4o = *reinterpret_cast<const float4*>(sm.cv + vi0);
              s4o = *reinterpret_cast<const float4*>(sm.sgv + vi0);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = 4 * h2 + i, slot = 4 * quad + i;
            const float A = f4get(tv, i);
            ok[k] = colok && slot < real;
            q[k] = sg * C::Q + slot;
            zo[k] = f4get(z4, i);
            co[k] = f4get(c4o, i);
            so[k] = f4get(s4o, i);
            Av[k] = A;
            v[k] = ok[k] ? fmaf(-A, inv_n, zo[k]) : 0.f;
            if (colok && !ok[k]) {
              if (slot == C::Q) p_E += A;
              else if (slot == C::Q + 1) p_G += A;
            }
          }
        }
        project_lane(pj, v, q, ok);
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int col = lane + 32 * h2;
          const bool colok = col < C::COLS;
          const int sg = colok ? col / C::NQR : 0, quad = colok ? col - sg * C::NQR : 0;
          const bool has_z = colok && quad < C::NQA;
          float zn[4], cn[4], sn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = 4 * h2 + i;
            zn[i] = cn[i] = sn[i] = 0.f;
            if (ok[k]) {
              const float znew = v[k], z = zo[k], A = Av[k];
              if (check) {
                const float del = co[k] - znew;
                const float SD = so[k] - A;
                const float dz = z - znew;
                p_dd = fmaf(del, del, p_dd);
                p_dS = fmaf(del, SD, p_dS);
                p_zz = fmaf(znew, znew, p_zz);
                p_zx = fmaf(znew, fmaf(fn, del, SD), p_zx);
                p_dz = fmaf(dz, dz, p_dz);
                p_dzA = fmaf(dz, A, p_dzA);
              }
              zn[i] = znew;
              cn[i] = 2.f * znew - z;
              sn[i] = A;
            }
          }
          if (has_z) {
            const int vi0 = sg * C::QA + 4 * quad;
            *reinterpret_cast<float4*>(sm.zv + vi0) = make_float4(zn[0], zn[1], zn[2], zn[3]);
            *reinterpret_cast<float4*>(sm.cv + vi0) = make_float4(cn[0], cn[1], cn[2], cn[3]);
            *reinterpret_cast<float4*>(sm.sgv + vi0) = make_float4(sn[0], sn[1], sn[2], sn[3]);
          }
        }
      }
      if (check) {
        p_dd = warp_sum(p_dd);
        p_dS = warp_sum(p_dS);
        p_zz = warp_sum(p_zz);
        p_zx = warp_sum(p_zx);
        p_dz = warp_sum(p_dz);
        p_dzA = warp_sum(p_dzA);
        p_E = warp_sum(p_E);
        p_G = warp_sum(p_G);
        if (lane == 0) {
          // sum_k ||x_k - z+||^2 = n||delta||^2 + 2 delta . sum Delta + sum ||Delta_k||^2
          const float spr = fmaxf(fn * p_dd + 2.f * p_dS + p_E, 0.f);
          // sum_k ||x_k||^2 = spr + 2 z+ . (n delta + sum Delta) + n ||z+||^2
          const float sx = fmaxf(spr + 2.f * p_zx + fn * p_zz, 0.f);
          // sum_k ||u_k+||^2 = n ||dz||^2 - 2 dz . sum g + sum ||g_k||^2
          const float su = fmaxf(fn * p_dz - 2.f * p_dzA + p_G, 0.f);
          const float den_p = fmaxf(fmaxf(sqrtf(sx), sqrtf(fn * p_zz)), 1e-30f);
          const float den_d = fmaxf(sqrtf(su), 1e-30f);
          const float rp = sqrtf(spr) / den_p;
          const float rd = sqrtf(fn * p_dz) / den_d;
          sm.scal[3] = fmaxf(rp, rd);
          sm.scal[4] = rp;
          sm.scal[5] = rd;
          sm.scal[0] = (prm.tol > 0.f && rp < prm.tol && rd < prm.tol) ? 1.f : 0.f;
        }
      }
    }
    __syncthreads();
    if (check) {
      resid = sm.scal[3];
      if (sm.scal[0] != 0.f) break;
    }
  }
  if (it > prm.iters) it = prm.iters;
  __syncthreads();
  if (t == 0) {
    sm.scal[2] = (float)it;
    sm.scal[3] = resid;
  }
  __syncthreads();
}

// FP64 objective of problem (1) and projected-gradient optimality residual at z (zv), both
// accumulated in double on the GPU.  Uses the wred region as scratch (CAP doubles for the
// distances).  wfun(j) returns the weight of point j in double: the caller's input weight for
// standalone problems, exp(-||P_i - P_j||^2 / h^2) recomputed in double for NLEM.
template <class C, class WF, bool NEG = false>
__device__ void fp64_check(const Smem<C>& sm, int n, int d, const SolveParams& prm, const WF& wfun,
                           double& F, double& R) {
  const int t = threadIdx.x;
  double* coef = reinterpret_cast<double*>(sm.wred);   // w_j / ||z - a_j|| (0 inside tau)
  double* gvec = coef + C::CAP;                           // the d-vector g
  __shared__ double s_F[C::NW], s_wb[C::NW], s_ws[C::NW], s_g2[C::NW];
  __shared__ double s_R, s_Fo;
  const double tau = 1e-9 * fmax(1.0, (double)prm.hi - (double)prm.lo);
  double f = 0.0, wb = 0.0, ws = 0.0;
  for (int j = t; j < n; j += C::NT) {
    double r2 = 0.0;
    for (int q = 0; q < d; ++q) {
      const int sg = q / C::Q, i = q - sg * C::Q;
      const double a = (double)sm.pts[j * C::DP + sg * C::QA + i];
      const double e = (double)sm.zv[sg * C::QA + i] + (NEG ? a : -a);   // z - a
      r2 += e * e;
    }
    const double r = sqrt(r2);
    const double w = wfun(j);
    f += w * r;
    ws += w;
    if (r <= tau) {
      wb += w;
      coef[j] = 0.0;
    } else {
      coef[j] = w / r;
    }
  }
  __syncthreads();
  double g2 = 0.0;
  for (int q = t; q < d; q += C::NT) {
    const int sg = q / C::Q, i = q - sg * C::Q;
    const double z = (double)sm.zv[sg * C::QA + i];
    double gq = 0.0;
    for (int j = 0; j < n; ++j) {
      const double a = (double)sm.pts[j * C::DP + sg * C::QA + i];
      gq += coef[j] * (z + (NEG ? a : -a));
    }
    gvec[q] = gq;
    g2 += gq * gq;
  }
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(kFull, f, o);
    wb += __shfl_xor_sync(kFull, wb, o);
    ws += __shfl_xor_sync(kFull, ws, o);
    g2 += __shfl_xor_sync(kFull, g2, o);
  }
  if ((t & 31) == 0) {
    s_F[t >> 5] = f;
    s_wb[t >> 5] = wb;
    s_ws[t >> 5] = ws;
    s_g2[t >> 5] = g2;
  }
  __syncthreads();
  if (t == 0) {
    double FF = 0, WB = 0, WS = 0, G2 = 0;
    for (int w = 0; w < C::NW; ++w) {
      FF += s_F[w];
      WB += s_wb[w];
      WS += s_ws[w];
      G2 += s_g2[w];
    }
    const double gn = sqrt(G2);
    const double scale = gn > 0.0 ? fmax(gn - WB, 0.0) / gn : 0.0;
    double RR = 0.0;
    if (WS > 0.0) {
      for (int q = 0; q < d; ++q) {
        const int sg = q / C::Q, i = q - sg * C::Q;
        const double z = (double)sm.zv[sg * C::QA + i];
        double tq = z - scale * gvec[q] / WS;
        tq = fmin(fmax(tq, (double)prm.lo), (double)prm.hi);
        RR += (z - tq) * (z - tq);
      }
    }
    s_R = sqrt(RR);
    s_Fo = FF;
  }
  __syncthreads();
  F = s_Fo;
  R = s_R;
}

}  // namespace nlemk
