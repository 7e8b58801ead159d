// Accelerated EM-ADMM for one problem per CTA: the steps of Algorithm 1 (Sec. 2 of Chaudhury &
// Ramakrishnan, arXiv 1501.03879) taken at an extrapolated point, with restart.  Sec. 4 names
// accelerated ADMM as future work; the scheme is fast ADMM with restart of Goldstein, O'Donoghue,
// Setzer and Baraniuk (2014), the variant for objectives that are not strongly convex.
//
// Method (scaled multipliers u_k = y_k / mu).  Step t runs Algorithm 1 once from (z^, u^_k):
//   e_k = z^ - u^_k - a_k,  f_k = min(1, lam_k / ||e_k||),  g_k = f_k e_k,  x_k = a_k + e_k - g_k,
//   z = P_C(z^ - (1/n) sum_k g_k),  u_k = u^_k + x_k - z = D - g_k   with D = z^ - z.
// Then c = n ||z - z^||^2, the z-part of Goldstein's combined residual (divided by mu), decides: if
// c < eta c_prev, alpha+ = (1 + sqrt(1 + 4 alpha^2)) / 2, beta = (alpha - 1) / alpha+,
// z^ = z + beta (z - z_old), u^ = u + beta (u - u_old), c_prev = c; otherwise (restart) alpha = 1,
// z^ = z_old, u^ = u_old, c_prev = c_prev / eta.  With a fixed period k > 0 (the fixed restart of
// O'Donoghue and Candes 2015) the step after iteration t restarts when t % k == 0 instead.  The
// combined residual's other part, sum_k ||x_k - z||^2, lies below what the FP32 state resolves near
// convergence (per-element rounding of about 1e-5 on values near 100 outweighs it), while
// n ||D||^2 is exact to FP32's relative precision (D = (1/n) sum_k g_k where the clamp is
// inactive); on NLEM and standalone problems at mu >= 0.01 the two tests take the same decisions in
// FP64.
//
// State form.  With h_k(t) = g_k(t) - a_k, the next shrink input is
//   e_k = C + p h_k(t) + q h_k(t-1):
//   momentum: p = 1 + beta, q = -beta, C = z^+ - (1 + beta) D(t) + beta D(t-1);
//   restart:  p = 0,        q = 1,     C = z(t-1) - D(t-1)
// (u_k = D - g_k, and the a_k terms cancel because p + q = 1).  Two per-point banks h(t), h(t-1)
// live in registers; the new h overwrites the older bank, and the banks swap roles each step.
// Per element and step: e (2 FFMA), ||e||^2 (FFMA), sum g (FFMA) and h = f e - a (FFMA): five FP32
// operations, issued as packed pairs (Algorithm 1's core takes four).
//
// Stopping rule.  Algorithm 1's relative primal and dual residuals at the step's x, u, z, with the
// step's own z-change z - z^ = -D in place of z - z_prev (the same when nothing is extrapolated;
// after a restart the step starts from z(t-1) and can land next to z(t) far from the optimum, which
// z - z_prev would take for convergence).  On check iterations a pass of its own forms
// W2 = sum_k ||x_k - r||^2 per element as (f - 1) e + (r - a) = -(x_k - r), with r = z^ - D(t-1) a
// close guess of z (FADD, FFMA, FFMA per element); the rest comes from d-vector sums:
//   sum_k (x_k - r) = n (z^ - r) - sum_k u^_k - G,  G = sum_k g_k,
//   sum_k u^_k = p (n D(t) - G(t)) + q (n D(t-1) - G(t-1)),
//   sum_k ||x_k - z||^2 = W2 + 2 (r - z) . sum (x_k - r) + n ||r - z||^2,
//   sum_k ||x_k||^2 = W2 + 2 r . sum (x_k - r) + n ||r||^2,
//   sum_k ||u_k||^2 = n ||D||^2 - 2 D . G + sum_k ||g_k||^2.
//
// Inactive point slots (j >= n) have zero rows and lam = 0, so g = 0 and h stays 0; their share of W2
// is left out per point.  Rows hold -a_j (the point rows of the NEG layout of admm_core.cuh).
#pragma once

#include "admm_core.cuh"
#include "debug.h"

namespace nlemk {

// The accelerated solver's d-vectors beyond the core's carve (zv = z, cv = C, sgv = G(t-1)), each in
// the slice layout (VEC floats): z^ of the next step, its residual reference r = z^ - D(t), D(t - 1),
// sum_k u^_k and dl = z^ - z(t-1).
template <class C>
struct FastVec {
  static constexpr int FLOATS = 5 * C::VEC;
  static constexpr size_t BYTES = (size_t)FLOATS * 4;
  float* zh;
  float* zr;
  float* dv;
  float* uh;
  float* dl;
  __device__ __forceinline__ explicit FastVec(float* base)
      : zh(base), zr(base + C::VEC), dv(base + 2 * C::VEC), uh(base + 3 * C::VEC), dl(base + 4 * C::VEC) {}
};

// Phase 1: e = C + p L + q O for the lane's points and slots, written into O, and the lane's share
// of each ||e_k||^2.
template <class C>
__device__ __forceinline__ void fast_phase1(const Smem<C>& sm, int g, bool last, float p, float q,
                                            const float2 (&L2)[C::P][C::Q / 2], const float (&L1)[C::P],
                                            float2 (&O2)[C::P][C::Q / 2], float (&O1)[C::P], float (&s)[C::P]) {
  float2 s2[C::P];
#pragma unroll
  for (int k = 0; k < C::P; ++k) s2[k] = make_float2(0.f, 0.f);
  const float2 p2 = make_float2(p, p), q2 = make_float2(q, q);
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
        for (int k = 0; k < C::P; ++k) {
          const float2 e = __ffma2_rn(q2, O2[k][q0 / 2], __ffma2_rn(p2, L2[k][q0 / 2], c2));
          O2[k][q0 / 2] = e;
          s2[k] = __ffma2_rn(e, e, s2[k]);
        }
      } else if (q0 < C::Q) {
        const float c1 = jh == 0 ? c4.x : c4.z;
#pragma unroll
        for (int k = 0; k < C::P; ++k) {
          const float e = fmaf(q, O1[k], fmaf(p, L1[k], c1));
          O1[k] = e;
          s2[k].x = fmaf(e, e, s2[k].x);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < C::P; ++k) s[k] = s2[k].x + s2[k].y;
}

// On check iterations, between the factors f and phase 2 (e still in O): the lane's share of
// W2 = sum_k ||x_k - r||^2 over its active points, with x_k - r = -(f e - a - e + r) and r = fv.zr.  The
// fences keep the compiler from carrying these loads into phase 2, where they would cost registers.
template <class C>
__device__ __forceinline__ float fast_check_w2(const Smem<C>& sm, const FastVec<C>& fv, int g, int pg, bool last,
                                              const float (&f)[C::P], int n, const float2 (&O2)[C::P][C::Q / 2],
                                              const float (&O1)[C::P]) {
  asm volatile("" ::: "memory");
  const float* zrow = fv.zr + g * C::QA;
  float2 ww2 = make_float2(0.f, 0.f);
  float ww1 = 0.f;
#pragma unroll
  for (int k = 0; k < C::P; ++k) {
    const bool act = pg + k * C::NG < n;
    const float* arow = sm.pts + (pg + k * C::NG) * C::DP + g * C::QA;
    const float fm = f[k] - 1.f;
    float2 pw2 = make_float2(0.f, 0.f);
    float pw1 = 0.f;
    const float2 fm2 = make_float2(fm, fm);
#pragma unroll
    for (int i = 0; i < C::NQA; ++i) {
      const float4 a4 = load_quad<C>(arow, i, last);
      const float4 r4 = load_quad<C>(zrow, i, last);
#pragma unroll
      for (int jh = 0; jh < 2; ++jh) {
        const int q0 = 4 * i + 2 * jh;
        const float2 na2 = jh == 0 ? make_float2(a4.x, a4.y) : make_float2(a4.z, a4.w);
        const float2 r2 = jh == 0 ? make_float2(r4.x, r4.y) : make_float2(r4.z, r4.w);
        if (q0 + 1 < C::Q) {
          const float2 w = __ffma2_rn(fm2, O2[k][q0 / 2], __fadd2_rn(r2, na2));
          pw2 = __ffma2_rn(w, w, pw2);
        } else if (q0 < C::Q) {
          const float w = fmaf(fm, O1[k], r2.x + na2.x);
          pw1 = fmaf(w, w, pw1);
        }
      }
    }
    if (act) ww1 += pw2.x + pw2.y + pw1;
    asm volatile("" ::: "memory");
  }
  return ww2.x + ww2.y + ww1;
}

// One quad of a point row for phase 2.  A last quad holding a single slot (Q = 4m + 1) is read as one float:
// a lane then reads 4Q + 4 bytes of its row instead of 4Q + 12, which cuts phase 2's shared-memory
// wavefronts by 3 of 16 per point.
template <class C>
__device__ __forceinline__ float4 load_row_quad(const float* row, int i, bool last) {
  if (C::Q % 4 == 1 && i == C::NQA - 1) return make_float4((C::D > 0 && last && 4 * i >= C::QL) ? 0.f : row[4 * i], 0.f, 0.f, 0.f);
  return load_quad<C>(row, i, last);
}

// Phase 2: from e (in O) and the factors f: h = f e - a back into O, and the first level of the block
// reduction.  Each quad's column sums of g = f e over the lane's points (plus W2 and sum ||g||^2 in the
// two slots after the last column) are summed over the slice's lanes by shuffles, and the warp's
// partial goes to cred, one float4 per warp and column; warp 0's finalize adds the warps' partials.
template <class C>
__device__ __forceinline__ void fast_phase2(const Smem<C>& sm, int g, int pg, bool last, const float (&f)[C::P],
                                            float w2, float gs, float2 (&O2)[C::P][C::Q / 2], float (&O1)[C::P]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* abase = sm.pts + pg * C::DP + g * C::QA;

#pragma unroll
  for (int i = 0; i < C::NQR; ++i) {
    float acc4[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < C::NQA) {
      float2 accp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float acc1 = 0.f;
#pragma unroll
      for (int k = 0; k < C::P; ++k) {
        const float4 a4 = load_row_quad<C>(abase + k * C::NG * C::DP, i, last);
        const float2 f2 = make_float2(f[k], f[k]);
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
          const int q0 = 4 * i + 2 * jh;
          const float2 na2 = jh == 0 ? make_float2(a4.x, a4.y) : make_float2(a4.z, a4.w);
          if (q0 + 1 < C::Q) {
            const float2 e = O2[k][q0 / 2];
            accp[jh] = __ffma2_rn(f2, e, accp[jh]);
            O2[k][q0 / 2] = __ffma2_rn(f2, e, na2);
          } else if (q0 < C::Q) {
            const float e = O1[k];
            acc1 = fmaf(f[k], e, acc1);
            O1[k] = fmaf(f[k], e, na2.x);
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
      if (4 * i + c == C::Q) acc4[c] = w2;
      if (4 * i + c == C::Q + 1) acc4[c] = gs;
    }
    {
      // sum over the slice's LPG lanes (8 or 16, consecutive), reduce-scattered: after xor LPG/2 a lane
      // keeps two of the four values, after xor LPG/4 one, and the remaining levels complete it in every
      // lane of a group of LPG/4
      static_assert(C::LPG == 8 || C::LPG == 16, "the fused reduction takes 8 or 16 lanes per slice");
      constexpr int H1 = C::LPG / 2, H2 = C::LPG / 4;
      const bool b2 = (lane & H1) != 0, b1 = (lane & H2) != 0;
      const float s0 = b2 ? acc4[0] : acc4[2], s1 = b2 ? acc4[1] : acc4[3];
      const float k0 = (b2 ? acc4[2] : acc4[0]) + __shfl_xor_sync(kFull, s0, H1);
      const float k1 = (b2 ? acc4[3] : acc4[1]) + __shfl_xor_sync(kFull, s1, H1);
      float k = (b1 ? k1 : k0) + __shfl_xor_sync(kFull, b1 ? k0 : k1, H2);
#pragma unroll
      for (int o = H2 / 2; o >= 1; o >>= 1) k += __shfl_xor_sync(kFull, k, o);
      const int ci = (warp * C::COLS + g * C::NQR + i) * 4 + (b2 ? 2 : 0) + (b1 ? 1 : 0);
      if ((lane & (H2 - 1)) == 0 && NLEM_DBG_OK(ci, C::NW * C::COLS * 4, kDbgFastPartial))
        reinterpret_cast<float*>(sm.cred)[ci] = k;
    }
  }
}

// Warp 0 state of the momentum / restart rule, identical in every lane.  The countdowns to the next
// periodic check and the next fixed-period restart (in place of a remainder per iteration) live in
// shared memory, scal[6] and scal[7] as integers.
struct FastRule {
  float alpha, c_prev;
  int restarts;
};

// The z-update of one coordinate, z = P_C(z^ - A / n), and the step D = z^ - z.  Where the clamp is
// inactive D is A / n itself, not the difference of two rounded values near z: the step is resolved
// to FP32's relative precision even when it is a few ulps of z.
__device__ __forceinline__ void fast_zstep(float zh, float A, float inv_n, float lo, float hi, float& z, float& D) {
  const float zu = fmaf(-A, inv_n, zh);
  z = fminf(fmaxf(zu, lo), hi);
  D = z == zu ? A * inv_n : zh - z;
}

// Warp 0, after the block reduction of step `it`: z, the residuals on check iterations, the
// momentum-or-restart decision and the next step's vectors; publishes the stop flag, p, q and the next
// step's check flag.
// The check pass measured w~_k = x_k - r against r = z^ - D(t-1), a close guess of z (D changes slowly), so
// that sum_k ||x_k - z||^2 = W2 + 2 (D - D(t-1)) . sum w~ + n ||D - D(t-1)||^2 keeps small terms, with
// sum_k w~_k = n D(t-1) - sum_k u^_k - G.  The iterate's step s = z(t) - z(t-1) is carried exactly as
// s = dl - D, dl = z^(t) - z(t-1) being beta s (momentum) or -s (restart) of the step before.
// CHECK: a check iteration (residuals and the stopping test); the instance without them carries none of
// their code, which otherwise lengthens the step's critical path.  The next-step vectors of both outcomes
// (momentum and restart) are formed before the decision's warp sum and selected after it: the finalize
// is one warp's dependent chain, and this takes them off it.
template <class C, bool CHECK>
__device__ __forceinline__ void fast_finalize(const Smem<C>& sm, const FastVec<C>& fv, int d, int it, float inv_n,
                                              float fn, const SolveParams& prm, int restart_every, FastRule& R) {
  static_assert(C::COLS <= 16, "the finalize gives each lane of warp 0 two slots of one column");
  constexpr float kEta = 0.999f;
  const int lane = threadIdx.x & 31;
  int* si = reinterpret_cast<int*>(sm.scal);
  const int ccnt = si[6], rcnt = si[7];
  // the momentum coefficients, formed before the decision that may not need them
  const float ua = fmaf(4.f * R.alpha, R.alpha, 1.f);
  const float a1 = 0.5f * fmaf(ua, rsqrtf(ua), 1.f);   // (1 + sqrt(1 + 4 alpha^2)) / 2
  const float beta_m = __fdividef(R.alpha - 1.f, a1);
  // lane l takes slots 2 (l & 1) and 2 (l & 1) + 1 of column l / 2: its totals are the sum of the
  // NW per-warp partials
  const int col = lane >> 1, hh = lane & 1;
  const bool colok = col < C::COLS;
  const int sg = colok ? col / C::NQR : 0, quad = colok ? col - sg * C::NQR : 0;
  const bool has = colok && quad < C::NQA &&     // the pair lies in the d-vectors
                   NLEM_DBG_OK(sg * C::QA + 4 * quad + 2 * hh + 1, C::VEC, kDbgFastVec);
  const int real = slice_real<C>(sg, d);
  const int slot0 = 4 * quad + 2 * hh;
  const int vi = sg * C::QA + slot0;
  float2 Aa = make_float2(0.f, 0.f), Ab = Aa;
  if (colok) {
    const float2* cr = reinterpret_cast<const float2*>(sm.cred) + 2 * col + hh;
#pragma unroll
    for (int w = 0; w < C::NW; w += 2) {
      const float2 va = cr[2 * C::COLS * w];
      Aa = make_float2(Aa.x + va.x, Aa.y + va.y);
      if (w + 1 < C::NW) {
        const float2 vb = cr[2 * C::COLS * (w + 1)];
        Ab = make_float2(Ab.x + vb.x, Ab.y + vb.y);
      }
    }
  }
  const float A0 = Aa.x + Ab.x, A1 = Aa.y + Ab.y;
  float2 zh2 = make_float2(0.f, 0.f), zo2 = zh2, do2 = zh2, go2 = zh2, dl2 = zh2;
  if (has) {
    zh2 = *reinterpret_cast<const float2*>(fv.zh + vi);
    zo2 = *reinterpret_cast<const float2*>(sm.zv + vi);
    do2 = *reinterpret_cast<const float2*>(fv.dv + vi);
    go2 = *reinterpret_cast<const float2*>(sm.sgv + vi);
    dl2 = *reinterpret_cast<const float2*>(fv.dl + vi);
  }
  float z[2] = {0.f, 0.f}, D[2] = {0.f, 0.f};
  float p_W2 = 0.f, p_gs = 0.f, p_DD = 0.f, p_eD = 0.f, p_eSw = 0.f, p_rSw = 0.f, p_rr = 0.f, p_zz = 0.f, p_DA = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int slot = slot0 + i;
    const float A = i ? A1 : A0;
    if (has && slot < real) {
      const float zh = i ? zh2.y : zh2.x;
      fast_zstep(zh, A, inv_n, prm.lo, prm.hi, z[i], D[i]);
      p_DD = fmaf(D[i], D[i], p_DD);
      if constexpr (CHECK) {
        const float Do = i ? do2.y : do2.x;
        const float Sw = fmaf(fn, Do, -fv.uh[vi + i] - A);   // sum_k (x_k - r)
        const float eD = D[i] - Do;
        const float r = zh - Do;
        p_eD = fmaf(eD, eD, p_eD);
        p_eSw = fmaf(eD, Sw, p_eSw);
        p_rSw = fmaf(r, Sw, p_rSw);
        p_rr = fmaf(r, r, p_rr);
        p_zz = fmaf(z[i], z[i], p_zz);
        p_DA = fmaf(D[i], A, p_DA);
      }
    } else if (colok && slot == C::Q) {
      p_W2 += A;
    } else if (colok && slot == C::Q + 1) {
      p_gs += A;
    }
  }
  // both outcomes' next-step vectors, formed before the decision so that they overlap its warp sum
  const float bpm = 1.f + beta_m;
  float zhm[2], cnm[2], uhm[2], dlm[2], zhr[2], cnr[2], uhr[2], dlr[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float A = i ? A1 : A0;
    const float zo = i ? zo2.y : zo2.x, Do = i ? do2.y : do2.x, Go = i ? go2.y : go2.x;
    const float st = (i ? dl2.y : dl2.x) - D[i];   // z(t) - z(t-1)
    const float uo = fmaf(fn, Do, -Go);
    zhm[i] = fmaf(beta_m, st, z[i]);
    cnm[i] = fmaf(beta_m, Do, fmaf(-bpm, D[i], zhm[i]));
    uhm[i] = fmaf(bpm, fmaf(fn, D[i], -A), -beta_m * uo);
    dlm[i] = beta_m * st;
    zhr[i] = zo;
    cnr[i] = zo - Do;
    uhr[i] = uo;
    dlr[i] = -st;
  }
  p_DD = warp_sum(p_DD);
  const float cc = fn * p_DD;   // the z-part of the combined residual, divided by mu
  bool stop = false;
  if constexpr (CHECK) {
    p_W2 = warp_sum(p_W2);
    p_gs = warp_sum(p_gs);
    p_eD = warp_sum(p_eD);
    p_eSw = warp_sum(p_eSw);
    p_rSw = warp_sum(p_rSw);
    p_rr = warp_sum(p_rr);
    p_zz = warp_sum(p_zz);
    p_DA = warp_sum(p_DA);
    const float spr = fmaxf(fmaf(fn, p_eD, fmaf(2.f, p_eSw, p_W2)), 0.f);   // sum_k ||x_k - z||^2
    const float sx = fmaxf(fmaf(fn, p_rr, fmaf(2.f, p_rSw, p_W2)), 0.f);    // sum_k ||x_k||^2
    const float su = fmaxf(fmaf(fn, p_DD, fmaf(-2.f, p_DA, p_gs)), 0.f);    // sum_k ||u_k||^2
    const float den_p = fmaxf(fmaxf(sqrtf(sx), sqrtf(fn * p_zz)), 1e-30f);
    const float den_d = fmaxf(sqrtf(su), 1e-30f);
    const float rp = sqrtf(spr) / den_p;
    const float rd = sqrtf(fn * p_DD) / den_d;
    stop = prm.tol > 0.f && rp < prm.tol && rd < prm.tol;
    if (lane == 0) {
      sm.scal[3] = fmaxf(rp, rd);
      sm.scal[4] = rp;
      sm.scal[5] = rd;
    }
  }
  // the momentum-or-restart step (also taken after the last iteration, where it only counts)
  bool mom = true;
  float beta = 0.f;
  if (!stop) {
    mom = restart_every > 0 ? rcnt != 1 : cc < kEta * R.c_prev;
    if (mom) {
      beta = beta_m;
      R.alpha = a1;
      R.c_prev = cc;
    } else {
      R.alpha = 1.f;
      R.c_prev = R.c_prev / kEta;
      ++R.restarts;
    }
  }
  const float bp = 1.f + beta;
  // the next step's vectors for the lane's two slots (phantom slots stay zero)
  if (has) {
    float zhn[2], zrn[2], cn[2], uhn[2], dln[2], gn[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const bool ok = slot0 + i < real;
      zhn[i] = ok ? (mom ? zhm[i] : zhr[i]) : 0.f;
      cn[i] = ok ? (mom ? cnm[i] : cnr[i]) : 0.f;
      uhn[i] = ok ? (mom ? uhm[i] : uhr[i]) : 0.f;
      dln[i] = ok ? (mom ? dlm[i] : dlr[i]) : 0.f;
      zrn[i] = ok ? zhn[i] - D[i] : 0.f;
      gn[i] = ok ? (i ? A1 : A0) : 0.f;
    }
    *reinterpret_cast<float2*>(sm.zv + vi) = make_float2(z[0], z[1]);
    if (!stop) {
      *reinterpret_cast<float2*>(fv.zh + vi) = make_float2(zhn[0], zhn[1]);
      *reinterpret_cast<float2*>(fv.zr + vi) = make_float2(zrn[0], zrn[1]);
      *reinterpret_cast<float2*>(sm.cv + vi) = make_float2(cn[0], cn[1]);
      *reinterpret_cast<float2*>(fv.uh + vi) = make_float2(uhn[0], uhn[1]);
      *reinterpret_cast<float2*>(fv.dv + vi) = make_float2(D[0], D[1]);
      *reinterpret_cast<float2*>(fv.dl + vi) = make_float2(dln[0], dln[1]);
      *reinterpret_cast<float2*>(sm.sgv + vi) = make_float2(gn[0], gn[1]);
    }
  }
  if (lane == 0) {
    // the next step's check flag, then one 16-byte store: stop, p, q, check; the countdowns advance
    const bool chk = it + 1 == prm.iters || (prm.tol > 0.f && ccnt == 1);
    *reinterpret_cast<float4*>(sm.scal + 12) = make_float4(stop ? 1.f : 0.f, mom ? bp : 0.f, mom ? -beta : 1.f,
                                                           chk ? 1.f : 0.f);
    si[6] = ccnt == 1 ? prm.check_every : ccnt - 1;
    si[7] = rcnt == 1 ? restart_every : rcnt - 1;
  }
}

// The norms ||e_k|| of this lane's points (sums of its slices' partial squares s), the factors
// f_k = min(1, lam_k / ||e_k||) and gs = the lane's share of sum_k ||g_k||^2 = sum_k f_k^2 ||e_k||^2.
// SCATTER (shapes with G = 4 slices on lanes xor 8 / xor 16 and P = 7): the 4 lanes of a point group
// reduce-scatter the 7 sums so that each forms f for 2 points only, then gather the f values back
// (fewer shuffles and reciprocal square roots than a full all-reduce per point).
template <class C, bool SCATTER>
__device__ __forceinline__ void fast_norms(const Smem<C>& sm, int g, int pg, float (&s)[C::P], float (&f)[C::P],
                                           float& gs) {
  gs = 0.f;
  if constexpr (SCATTER && C::G == 4 && C::LPG == 8 && C::P == 7) {
    const int lane = threadIdx.x & 31;
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    // after the xor-16 and xor-8 halvings lane (b4, b3) holds points 4*b4 + 2*b3 + {0, 1} (the 8th a pad)
    float k4[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const float lo = s[jj], hi = jj + 4 < C::P ? s[jj + 4] : 0.f;
      k4[jj] = (b4 ? hi : lo) + __shfl_xor_sync(kFull, b4 ? lo : hi, 16);
    }
    float fo[2];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const float r2 = (b3 ? k4[jj + 2] : k4[jj]) + __shfl_xor_sync(kFull, b3 ? k4[jj] : k4[jj + 2], 8);
      const int idx = (b4 ? 4 : 0) + (b3 ? 2 : 0) + jj;
      const bool real = idx < C::P;
      // r2 = 0 gives lam*inf (or NaN when lam = 0) and fminf then yields 1, harmless because e = 0 there
      const float lam = real ? sm.lam[pg + (real ? idx : 0) * C::NG] : 0.f;
      fo[jj] = fminf(1.f, lam * rsqrtf(r2));
      if (real) gs = fmaf(fo[jj] * fo[jj], r2, gs);   // each point counted once, by the lane that owns it
    }
    float f4[4];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const float other = __shfl_xor_sync(kFull, fo[jj], 8);
      f4[jj] = b3 ? other : fo[jj];
      f4[jj + 2] = b3 ? fo[jj] : other;
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const float other = __shfl_xor_sync(kFull, f4[jj], 16);
      f[jj] = b4 ? other : f4[jj];
      if (jj + 4 < C::P) f[jj + 4] = b4 ? f4[jj] : other;
    }
  } else {
#pragma unroll
    for (int k = 0; k < C::P; ++k) s[k] = point_sum<C>(s[k]);
#pragma unroll
    for (int k = 0; k < C::P; ++k) {
      const float r2 = s[k];
      // r2 = 0 gives lam*inf (or NaN when lam = 0) and fminf then yields 1, harmless because e = 0 there
      f[k] = fminf(1.f, sm.lam[pg + k * C::NG] * rsqrtf(r2));
      gs = fmaf(f[k] * f[k], r2, gs);
    }
    if (g != 0) gs = 0.f;   // each point's ||g_k||^2 counted once, by its slice-0 lane
  }
}

// One step with bank L = h(t-1) (latest) and O = h(t-2) (older, overwritten by h(t)).  Returns true
// when the solve ends after this step.
template <class C, bool SCATTER>
__device__ __forceinline__ bool fast_step(const Smem<C>& sm, const FastVec<C>& fv, int n, int d, int it,
                                          const SolveParams& prm, int restart_every, float inv_n, float fn,
                                          const float2 (&L2)[C::P][C::Q / 2], const float (&L1)[C::P],
                                          float2 (&O2)[C::P][C::Q / 2], float (&O1)[C::P], FastRule& R) {
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>();
  const bool last = (g == C::G - 1);
  const float4 pq = *reinterpret_cast<const float4*>(sm.scal + 12);   // stop, p, q, check
  const bool check = pq.w != 0.f;
  const float p = pq.y, q = pq.z;
  float s[C::P];
  fast_phase1<C>(sm, g, last, p, q, L2, L1, O2, O1, s);
  float f[C::P];
  float gs;
  fast_norms<C, SCATTER>(sm, g, pg, s, f, gs);
  const float w2 = check ? fast_check_w2<C>(sm, fv, g, pg, last, f, n, O2, O1) : 0.f;
  fast_phase2<C>(sm, g, pg, last, f, w2, gs, O2, O1);
  __syncthreads();
  if (t < 32) {
    if (check)
      fast_finalize<C, true>(sm, fv, d, it, inv_n, fn, prm, restart_every, R);
    else
      fast_finalize<C, false>(sm, fv, d, it, inv_n, fn, prm, restart_every, R);
  }
  __syncthreads();
  return sm.scal[12] != 0.f || it >= prm.iters;
}

// Accelerated EM-ADMM from the state set up by the caller, as for admm_iterate: pts (rows of
// -a_j, inactive slots zero), lam (w_j / mu), zv = cv = z(0) (phantom slots zero) and sgv = 0.
// On return zv holds z; scal[2] = iterations run, scal[3] = last residual, scal[9] = restarts.
template <class C, bool SCATTER = false>
__device__ void admm_fast_iterate(const Smem<C>& sm, const FastVec<C>& fv, int n, int d, const SolveParams& prm,
                                  int restart_every) {
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>();
  const bool last = (g == C::G - 1);
  const float inv_n = 1.f / (float)n, fn = (float)n;
  constexpr int NP2 = C::Q / 2;
  // bank A starts as h(0) = -a (g = 0, u = 0), bank B as zeros (its weight q is 0 in step 1)
  float2 hA[C::P][NP2], hB[C::P][NP2];
  float hA1[C::P], hB1[C::P];
#pragma unroll
  for (int k = 0; k < C::P; ++k) {
    const int j = pg + k * C::NG;
    float a[C::Q];
    load_slice<C>(sm.pts + j * C::DP + g * C::QA, last, a);
#pragma unroll
    for (int i = 0; i < NP2; ++i) {
      hA[k][i] = make_float2(a[2 * i], a[2 * i + 1]);
      hB[k][i] = make_float2(0.f, 0.f);
    }
    hA1[k] = (C::Q % 2) ? a[C::Q - 1] : 0.f;
    hB1[k] = 0.f;
  }
  for (int i = t; i < C::VEC; i += C::NT) {
    fv.zh[i] = sm.zv[i];
    fv.zr[i] = sm.zv[i];
    fv.dv[i] = 0.f;
    fv.uh[i] = 0.f;
    fv.dl[i] = 0.f;
  }
  // countdowns: iteration t is a periodic check when the check countdown reads 1 as its flag is formed,
  // and a fixed-period restart when the restart countdown reads 1 in its finalize
  FastRule R{1.f, __int_as_float(0x7f800000), 0};
  if (t == 0) {
    const bool chk1 = prm.iters == 1 || (prm.tol > 0.f && prm.check_every == 1);
    int* si = reinterpret_cast<int*>(sm.scal);
    si[6] = prm.check_every == 1 ? 1 : prm.check_every - 1;
    si[7] = restart_every;
    sm.scal[3] = 0.f;
    *reinterpret_cast<float4*>(sm.scal + 12) = make_float4(0.f, 1.f, 0.f, chk1 ? 1.f : 0.f);   // stop, p, q, check
  }
  __syncthreads();
  int it = 0;
  if (prm.iters > 0) {
    for (;;) {
      ++it;
      if (fast_step<C, SCATTER>(sm, fv, n, d, it, prm, restart_every, inv_n, fn, hA, hA1, hB, hB1, R)) break;
      ++it;
      if (fast_step<C, SCATTER>(sm, fv, n, d, it, prm, restart_every, inv_n, fn, hB, hB1, hA, hA1, R)) break;
    }
  }
  if (t == 0) {
    sm.scal[2] = (float)it;
    sm.scal[9] = (float)R.restarts;
  }
  __syncthreads();
}

}  // namespace nlemk
