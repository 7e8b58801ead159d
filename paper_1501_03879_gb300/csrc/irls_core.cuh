// Device core of IRLS on the smooth surrogate of problem (1) (Eq. 2 of Chaudhury & Ramakrishnan,
// arXiv 1501.03879, Sec. 1): minimise sum_k w_k (||x - a_k||^2 + eps)^(1/2) over C.
//
// Setting the gradient of the surrogate to zero gives the fixed point x = sum_k om_k a_k / sum_k om_k
// with om_k = w_k (||x - a_k||^2 + eps)^(-1/2); one IRLS step evaluates the right-hand side at
// the current x.  The box C is enforced by projecting after every step (the same reading as the
// FP64 reference).  It is the comparison method of Sec. 3 (NLEM-IRLS, Table 1 and Figs. 1-2).
//
// The step is taken in residual form, x+ = P_C(x - sum_k om_k e_k / sum_k om_k) with e_k = x - a_k,
// which equals the weighted mean above.  From the noisy patch the pixel's own patch sits at
// distance ~0 with weight w/sqrt(eps), so the plain weighted sum adds a 1000x term to the rest
// and its FP32 rounding (about 1e-4 of x) then decides the next weight 1/||x - a_i||; the residual
// form keeps the error at the FP32 storage of x.  Each lane keeps e_k for its P points in
// registers (packed FP32 pairs, started at -a_k) and adds the last step dx = x - x_prev before
// use, as the ADMM core adds c to h: one step per coordinate pair is e += dx (FADD2),
// ||e||^2 (FFMA2) and sum om e (FFMA2), three packed instructions against the ADMM's four.
// Same CTA layout as admm_core.cuh: G lanes share a point, lane g owns slice g of the coordinates.
#pragma once

#include "admm_core.cuh"

namespace nlemk {

// IRLS from the state set up by the caller: pts (inactive slots zero), lam = w_j (zero for
// inactive slots) and zv = cv = x(0) (phantom slots zero).  Runs exactly prm.iters steps.  On
// return zv holds x and cv the last step; scal[2] = steps run; scal[3] = ||x(T) - x(T-1)|| /
// ||x(T)|| of the last step (0 when no step ran).
template <class C, bool NEG = false>
__device__ void irls_iterate(const Smem<C>& sm, int n, int d, const SolveParams& prm) {
  const int t = threadIdx.x, g = lane_slice<C>(), pg = lane_group<C>(), lane = t & 31, warp = t >> 5;
  const bool last = (g == C::G - 1);
  const float eps = prm.eps;

  constexpr int NP2 = C::Q / 2;
  float2 e2[C::P][NP2];    // e_k = x - a_k, two slots per register pair (started at -a_k)
  float e1[C::P];          // the single last slot when Q is odd
  float lam[C::P];
#pragma unroll
  for (int p = 0; p < C::P; ++p) {
    const int j = pg + p * C::NG;
    float a[C::Q];
    load_slice<C>(sm.pts + j * C::DP + g * C::QA, last, a);
#pragma unroll
    // e = -a: the rows hold -a (NEG) or a
    for (int k = 0; k < NP2; ++k) e2[p][k] = NEG ? make_float2(a[2 * k], a[2 * k + 1]) : make_float2(-a[2 * k], -a[2 * k + 1]);
    e1[p] = (C::Q % 2) ? (NEG ? a[C::Q - 1] : -a[C::Q - 1]) : 0.f;
    lam[p] = sm.lam[j];
  }

  float resid = 0.f;
  for (int it = 1; it <= prm.iters; ++it) {
    const bool check = it == prm.iters;
    // phase 1: e += dx (cv holds x(0) before the first step, then the last step) and the squared
    // distances ||e||^2, one float4 of dx at a time
    float om[C::P];
    {
      float2 s2[C::P];
#pragma unroll
      for (int p = 0; p < C::P; ++p) s2[p] = make_float2(0.f, 0.f);
      const float* drow = sm.cv + g * C::QA;
#pragma unroll
      for (int i = 0; i < C::NQA; ++i) {
        const float4 d4 = load_quad<C>(drow, i, last);
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
          const int q0 = 4 * i + 2 * jh;
          if (q0 + 1 < C::Q) {
            const float2 d2 = jh == 0 ? make_float2(d4.x, d4.y) : make_float2(d4.z, d4.w);
#pragma unroll
            for (int p = 0; p < C::P; ++p) {
              e2[p][q0 / 2] = __fadd2_rn(e2[p][q0 / 2], d2);
              s2[p] = __ffma2_rn(e2[p][q0 / 2], e2[p][q0 / 2], s2[p]);
            }
          } else if (q0 < C::Q) {
            const float d1 = jh == 0 ? d4.x : d4.z;
#pragma unroll
            for (int p = 0; p < C::P; ++p) {
              e1[p] += d1;
              s2[p].x = fmaf(e1[p], e1[p], s2[p].x);
            }
          }
        }
      }
#pragma unroll
      for (int p = 0; p < C::P; ++p) om[p] = point_sum<C>(s2[p].x + s2[p].y);
#pragma unroll
      for (int p = 0; p < C::P; ++p) om[p] = lam[p] * rsqrtf(om[p] + eps);
    }
    // phase 2: sum_k om_k e_k into this lane's reduction row, sum_k om_k in slot Q (counted by
    // the slice-0 lane of each point)
    {
      float den = 0.f;
#pragma unroll
      for (int p = 0; p < C::P; ++p) den += om[p];
      if (g != 0) den = 0.f;
      float4* my = sm.wred + (warp * 32 + lane) * C::RS;
#pragma unroll
      for (int i = 0; i < C::NQR; ++i) {
        float acc4[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < C::NQA) {
          float2 accp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          float acc1 = 0.f;
#pragma unroll
          for (int p = 0; p < C::P; ++p) {
            const float2 om2 = make_float2(om[p], om[p]);
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
              const int q0 = 4 * i + 2 * jh;
              if (q0 + 1 < C::Q) accp[jh] = __ffma2_rn(om2, e2[p][q0 / 2], accp[jh]);
              else if (q0 < C::Q) acc1 = fmaf(om[p], e1[p], acc1);
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
        for (int c = 0; c < 4; ++c)
          if (4 * i + c == C::Q) acc4[c] = den;
        my[i] = make_float4(acc4[0], acc4[1], acc4[2], acc4[3]);
      }
    }
    float4 t0, t1;
    block_reduce_rows<C>(sm, t0, t1);
    // finalize (warp 0): x+ = P_C(x - sum om e / sum om), dx = x+ - x; x is kept if every weight is
    // zero
    if (t < 32) {
      __shared__ float s_den;
      {
        constexpr int cq = C::Q / 4;      // column holding slot Q of slice 0
        float v = (lane == cq) ? f4get(t0, C::Q - 4 * cq) : 0.f;
        v = warp_sum(v);
        if (lane == 0) s_den = v;
      }
      __syncwarp();
      const float den = s_den;
      const bool upd = den > 0.f;
      const float inv = upd ? 1.f / den : 0.f;
      float p_dx = 0.f, p_xx = 0.f;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int col = lane + 32 * h2;
        if (col >= C::COLS) continue;
        const int sg = col / C::NQR, quad = col - sg * C::NQR;
        if (quad >= C::NQA) continue;
        const float4 tv = h2 == 0 ? t0 : t1;
        const int real = slice_real<C>(sg, d);
        const int vi0 = sg * C::QA + 4 * quad;
        const float4 x4 = *reinterpret_cast<const float4*>(sm.zv + vi0);
        float xn[4], dn[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int slot = 4 * quad + i;
          const float x = f4get(x4, i);
          xn[i] = dn[i] = 0.f;
          if (slot < real) {
            xn[i] = upd ? clampf(fmaf(-f4get(tv, i), inv, x), prm.lo, prm.hi) : x;
            dn[i] = xn[i] - x;
            p_dx = fmaf(dn[i], dn[i], p_dx);
            p_xx = fmaf(xn[i], xn[i], p_xx);
          }
        }
        *reinterpret_cast<float4*>(sm.zv + vi0) = make_float4(xn[0], xn[1], xn[2], xn[3]);
        *reinterpret_cast<float4*>(sm.cv + vi0) = make_float4(dn[0], dn[1], dn[2], dn[3]);
      }
      if (check) {
        p_dx = warp_sum(p_dx);
        p_xx = warp_sum(p_xx);
        if (lane == 0) sm.scal[3] = sqrtf(p_dx) / fmaxf(sqrtf(p_xx), 1e-30f);
      }
    }
    __syncthreads();
    if (check) resid = sm.scal[3];
  }
  __syncthreads();
  if (t == 0) {
    sm.scal[2] = (float)(prm.iters > 0 ? prm.iters : 0);
    sm.scal[3] = resid;
  }
  __syncthreads();
}

}  // namespace nlemk
