/*
 * FP64 CPU oracle for constrained Euclidean medians (EM-ADMM) and NLEM denoising.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the CPU-baseline /
 * reference arm of bench.py load this library.  It shares no code, header or table with the
 * CUDA library; the two meet only through the seeded inputs of the `synth` module.
 *
 * Source: K. N. Chaudhury and K. R. Ramakrishnan, "A new ADMM algorithm for the Euclidean
 * median and its application to robust patch regression" (arXiv 1501.03879).
 *   problem (1)             Sec. 1, Eq. (1):  min_{x in C} sum_k w_k ||x - a_k||_2
 *   prox of lam*||x-u||     Sec. 2, Eqs. (prox), (defprox), (closed-form)
 *   conjugate prox          Sec. 2, Eqs. (CF), (proxfstar): projection onto the lam-ball
 *   EM-ADMM                 Sec. 2, Algorithm 1 with Eqs. (updatex), (updatez), (updatey)
 *   box projection          Sec. 3, coordinate-wise clamp to [l, u]
 *   accelerated EM-ADMM     Sec. 4 names accelerated ADMM as future work; orc_em_admm_fast
 *                           follows Goldstein, O'Donoghue, Setzer and Baraniuk (2014), fast ADMM
 *                           with restart for problems that are not strongly convex
 *   NLEM                    Sec. 3, Eq. (L1regression): patches, weights exp(-||Pi-Pj||^2/h^2),
 *                           window S(i), centre pixel of the denoised patch
 *
 * Readings where the paper is silent (all also listed in the design notes):
 *   - zero distance in the prox (0/0 in Eq. closed-form): the limit value v;
 *   - z-average over N = n terms, unweighted, exactly as Algorithm 1 writes it;
 *   - y_k = 0 and z = P_C(weighted mean) or the noisy patch at start (Sec. 3 text);
 *   - stopping: scaled-form relative primal/dual residuals (Boyd et al. 2011) checked every
 *     m iterations and at the cap;
 *   - borders: search window clipped to in-image centres, patches reflect-padded (no edge
 *     repeat);
 *   - weights use the raw squared distance, not divided by k^2, and w_ii = 1 is kept.
 *
 * Arithmetic is plain double, summed in index order; built with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---------------------------------------------------------------------------------------
 * Sec. 2, Eq. (closed-form):  Psi_lam(v, u) = v - min(lam, ||v-u||) (v-u)/||v-u||.
 * At ||v-u|| = 0 the fraction is 0/0; the limit (and the argmin of Eq. defprox) is v.
 * lam = +inf gives u.
 * ------------------------------------------------------------------------------------- */
void orc_prox(const double *v, const double *u, double lam, int d, double *out) {
  double r2 = 0.0;
  for (int q = 0; q < d; ++q) {
    double e = v[q] - u[q];
    r2 += e * e;
  }
  double r = sqrt(r2);
  if (r == 0.0) {
    for (int q = 0; q < d; ++q) out[q] = v[q];
    return;
  }
  double m = lam < r ? lam : r;
  double f = m / r;
  for (int q = 0; q < d; ++q) out[q] = v[q] - f * (v[q] - u[q]);
}

/* Sec. 2, Eq. (proxfstar): prox of the conjugate = projection of v-u onto the lam-ball. */
void orc_prox_conj(const double *v, const double *u, double lam, int d, double *out) {
  double r2 = 0.0;
  for (int q = 0; q < d; ++q) {
    double e = v[q] - u[q];
    r2 += e * e;
  }
  double r = sqrt(r2);
  if (r == 0.0) {
    for (int q = 0; q < d; ++q) out[q] = 0.0;
    return;
  }
  double m = lam < r ? lam : r;
  for (int q = 0; q < d; ++q) out[q] = m * (v[q] - u[q]) / r;
}

/* Sec. 3: projection onto C = [lo, hi]^d, coordinate by coordinate. */
void orc_project_box(const double *x, int d, double lo, double hi, double *out) {
  for (int q = 0; q < d; ++q) {
    double t = x[q];
    if (t < lo) t = lo;
    if (t > hi) t = hi;
    out[q] = t;
  }
}

/* Sec. 1, Eq. (1): F(z) = sum_k w_k ||z - a_k||. */
double orc_objective(const double *z, const double *pts, const double *w, int n, int d) {
  double F = 0.0;
  for (int k = 0; k < n; ++k) {
    double r2 = 0.0;
    for (int q = 0; q < d; ++q) {
      double e = z[q] - pts[(size_t)k * d + q];
      r2 += e * e;
    }
    F += w[k] * sqrt(r2);
  }
  return F;
}

/* Optimality residual of problem (1) with C a box, in the units of z.
 * g = sum over points farther than tau of w_k (z-a_k)/||z-a_k||; points within tau add the
 * subgradient ball of radius sum w_k, so ||g|| is reduced by that radius (floored at 0).
 * R = || z - P_C(z - g / sum_k w_k) ||  (projected-gradient form of 0 in dF(z) + N_C(z)). */
double orc_kkt_residual(const double *z, const double *pts, const double *w, int n, int d,
                        double lo, double hi, double tau) {
  double *g = (double *)calloc((size_t)d, sizeof(double));
  double wsum = 0.0, wball = 0.0;
  for (int k = 0; k < n; ++k) {
    wsum += w[k];
    double r2 = 0.0;
    for (int q = 0; q < d; ++q) {
      double e = z[q] - pts[(size_t)k * d + q];
      r2 += e * e;
    }
    double r = sqrt(r2);
    if (r <= tau) {
      wball += w[k];
      continue;
    }
    for (int q = 0; q < d; ++q) g[q] += w[k] * (z[q] - pts[(size_t)k * d + q]) / r;
  }
  double gn = 0.0;
  for (int q = 0; q < d; ++q) gn += g[q] * g[q];
  gn = sqrt(gn);
  double scale = 0.0;
  if (gn > 0.0) scale = (gn > wball ? gn - wball : 0.0) / gn;
  double R = 0.0;
  if (wsum > 0.0) {
    for (int q = 0; q < d; ++q) {
      double t = z[q] - scale * g[q] / wsum;
      if (t < lo) t = lo;
      if (t > hi) t = hi;
      double e = z[q] - t;
      R += e * e;
    }
  }
  free(g);
  return sqrt(R);
}

/* Start point: P_C(sum w_k a_k / sum w_k) (the NLM patch of Sec. 3); plain mean if all
 * weights vanish. */
void orc_weighted_mean_start(const double *pts, const double *w, int n, int d, double lo,
                             double hi, double *z) {
  double ws = 0.0;
  for (int k = 0; k < n; ++k) ws += w[k];
  for (int q = 0; q < d; ++q) {
    double s = 0.0;
    if (ws > 0.0) {
      for (int k = 0; k < n; ++k) s += w[k] * pts[(size_t)k * d + q];
      s /= ws;
    } else {
      for (int k = 0; k < n; ++k) s += pts[(size_t)k * d + q];
      s /= (double)n;
    }
    z[q] = s;
  }
  orc_project_box(z, d, lo, hi, z);
}

/* ---------------------------------------------------------------------------------------
 * Algorithm 1 (EM-ADMM), Sec. 2, in its own order and notation:
 *   loop: r = 0;  for k: x_k = Psi_{w_k/mu}(z - y_k/mu, a_k);  r += x_k + y_k/mu
 *         z = P_C(r / N)                      (N = n, Eq. updatez)
 *         for k: y_k += mu (x_k - z)          (Eq. updatey)
 * y_k starts at 0 (Sec. 3).  z0 == NULL starts from P_C(weighted mean).
 * tol > 0 stops at the first check iteration t (t % check_every == 0, or t == iters) where
 * both relative residuals are below tol:
 *   r_pri  = sqrt(sum_k ||x_k - z||^2) / max(sqrt(sum_k ||x_k||^2), sqrt(n) ||z||, 1e-30)
 *   r_dual = sqrt(n) ||z - z_prev|| / max(sqrt(sum_k ||y_k/mu||^2), 1e-30)
 * The residuals of the last iteration run are always returned (0 if iters == 0).
 * Returns 0, or -1 if memory runs out.
 * ------------------------------------------------------------------------------------- */
/* Algorithm 1 with a penalty per constraint, mu_k = mu * w_k (the augmented Lagrangian of Sec. 2
 * with (mu_k / 2) ||x_k - z||^2 in place of (mu / 2) ||x_k - z||^2; Sec. 4 leaves the choice of
 * penalty open).  The steps are those of Algorithm 1 with mu replaced by mu_k:
 *   x_k = Psi_{w_k / mu_k}(z - y_k / mu_k, a_k)        prox radius w_k / mu_k = 1 / mu for every k
 *   z   = P_C(sum_k mu_k (x_k + y_k / mu_k) / sum_k mu_k)   a weighted mean, weights w_k
 *   y_k = y_k + mu_k (x_k - z)
 * kept in the scaled multipliers u_k = y_k / mu_k (y_k = 0 at the start, so u_k = 0), which stay
 * defined where w_k = 0: such a point has no penalty and no say in z.  If every weight is 0 the
 * weights are taken as 1 (any z is then optimal).
 * The stopping rule is the one of orc_em_admm in the norm the penalties define (each point's
 * terms weighted by mu_k / mu = w_k, and n replaced by W = sum_k w_k):
 *   r_pri  = sqrt(sum_k w_k ||x_k - z||^2) / max(sqrt(sum_k w_k ||x_k||^2), sqrt(W) ||z||, 1e-30)
 *   r_dual = sqrt(W) ||z - z_prev|| / max(sqrt(sum_k w_k ||u_k||^2), 1e-30)
 * Start, check schedule and outputs as orc_em_admm.  Returns 0, or -1 if memory runs out. */
int orc_em_admm_wpen(const double *pts, const double *w, int n, int d, double lo, double hi, double mu,
                     int iters, const double *z0, double tol, int check_every, double *z, int *iters_used,
                     double *rpri, double *rdual) {
  const size_t nd = (size_t)n * d;
  double *x = (double *)malloc(sizeof(double) * nd);
  double *u = (double *)calloc(nd, sizeof(double));
  double *om = (double *)malloc(sizeof(double) * (size_t)n);
  double *r = (double *)malloc(sizeof(double) * (size_t)d);
  double *v = (double *)malloc(sizeof(double) * (size_t)d);
  double *zprev = (double *)malloc(sizeof(double) * (size_t)d);
  if (!x || !u || !om || !r || !v || !zprev) {
    free(x); free(u); free(om); free(r); free(v); free(zprev);
    return -1;
  }
  double W = 0.0;
  for (int k = 0; k < n; ++k) W += w[k];
  for (int k = 0; k < n; ++k) om[k] = W > 0.0 ? w[k] : 1.0;
  if (!(W > 0.0)) W = (double)n;
  if (z0) {
    for (int q = 0; q < d; ++q) z[q] = z0[q];
  } else {
    orc_weighted_mean_start(pts, w, n, d, lo, hi, z);
  }
  if (check_every < 1) check_every = 1;
  int t_done = 0;
  double rp = 0.0, rd = 0.0;
  for (int t = 1; t <= iters; ++t) {
    for (int q = 0; q < d; ++q) r[q] = 0.0;
    for (int k = 0; k < n; ++k) {
      double *xk = x + (size_t)k * d;
      const double *uk = u + (size_t)k * d;
      for (int q = 0; q < d; ++q) v[q] = z[q] - uk[q];
      orc_prox(v, pts + (size_t)k * d, 1.0 / mu, d, xk);
      for (int q = 0; q < d; ++q) r[q] += om[k] * (xk[q] + uk[q]);
    }
    for (int q = 0; q < d; ++q) {
      zprev[q] = z[q];
      z[q] = r[q] / W;
    }
    orc_project_box(z, d, lo, hi, z);
    for (int k = 0; k < n; ++k) {
      double *uk = u + (size_t)k * d;
      const double *xk = x + (size_t)k * d;
      for (int q = 0; q < d; ++q) uk[q] += xk[q] - z[q];
    }
    t_done = t;
    int check = (t == iters) || (tol > 0.0 && (t % check_every) == 0);
    if (check) {
      double spr = 0.0, sx = 0.0, su = 0.0, zz = 0.0, dz = 0.0;
      for (int k = 0; k < n; ++k) {
        double pe = 0.0, px = 0.0, pu = 0.0;
        for (int q = 0; q < d; ++q) {
          double xq = x[(size_t)k * d + q];
          double e = xq - z[q];
          double uq = u[(size_t)k * d + q];
          pe += e * e;
          px += xq * xq;
          pu += uq * uq;
        }
        spr += om[k] * pe;
        sx += om[k] * px;
        su += om[k] * pu;
      }
      for (int q = 0; q < d; ++q) {
        zz += z[q] * z[q];
        double e = z[q] - zprev[q];
        dz += e * e;
      }
      double den_p = sqrt(sx);
      double wzn = sqrt(W) * sqrt(zz);
      if (wzn > den_p) den_p = wzn;
      if (den_p < 1e-30) den_p = 1e-30;
      double den_d = sqrt(su);
      if (den_d < 1e-30) den_d = 1e-30;
      rp = sqrt(spr) / den_p;
      rd = sqrt(W) * sqrt(dz) / den_d;
      if (tol > 0.0 && rp < tol && rd < tol) break;
    }
  }
  if (iters_used) *iters_used = t_done;
  if (rpri) *rpri = rp;
  if (rdual) *rdual = rd;
  free(x); free(u); free(om); free(r); free(v); free(zprev);
  return 0;
}

/* Algorithm 1 with Nesterov-type momentum and restart (fast ADMM with restart; Goldstein et al.
 * 2014, the variant for objectives that are not strongly convex).  Steps (x, z, y) are those of
 * Algorithm 1, taken at the extrapolated z_hat and y_hat.  After each step a residual c decides:
 * with combined != 0 Goldstein's combined residual c = ||y - y_hat||^2 / mu + mu * n * ||z - z_hat||^2,
 * with combined == 0 its z-part c = mu * n * ||z - z_hat||^2 (the dual residual of the step).  If
 * c < eta * c_prev the momentum
 * grows, alpha+ = (1 + sqrt(1 + 4 alpha^2)) / 2, and z_hat, y_hat step beyond the new iterate by
 * (alpha - 1) / alpha+ times its change; otherwise alpha = 1, z_hat and y_hat restart from the
 * previous iterate and c_prev is divided by eta.  With alpha = 1 at the start, the first two
 * iterations equal Algorithm 1's.  The stopping rule and residuals are those of orc_em_admm,
 * evaluated at the step's x, y and z, with the step's own z-change z - z_hat in place of
 * z - z_prev (the same when nothing is extrapolated, z_hat = z_prev; after a restart, a step from
 * z(t-1) can land next to z(t) while far from the optimum).  *restarts (if not NULL)
 * counts the restarts.  *margin (if not NULL) is the smallest |c / (eta c_prev) - 1| over the
 * momentum-or-restart decisions taken with a finite c_prev (+inf if there were none): how close
 * the run came to deciding the other way.
 * restart_every = k > 0 replaces the residual test by a fixed period (the fixed restart of
 * O'Donoghue and Candes 2015): the step after iteration t restarts when t % k == 0 and takes the
 * momentum otherwise; c is then not consulted (margin stays +inf). */
int orc_em_admm_fast(const double *pts, const double *w, int n, int d, double lo, double hi, double mu,
                     int iters, const double *z0, double tol, int check_every, double eta, int restart_every,
                     int combined, double *z, int *iters_used, double *rpri, double *rdual, int *restarts,
                     double *margin) {
  const size_t nd = (size_t)n * d;
  double *x = (double *)malloc(sizeof(double) * nd);
  double *y = (double *)calloc(nd, sizeof(double));
  double *yh = (double *)calloc(nd, sizeof(double));
  double *yo = (double *)calloc(nd, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * (size_t)d);
  double *v = (double *)malloc(sizeof(double) * (size_t)d);
  double *zh = (double *)malloc(sizeof(double) * (size_t)d);
  double *zo = (double *)malloc(sizeof(double) * (size_t)d);
  if (!x || !y || !yh || !yo || !r || !v || !zh || !zo) {
    free(x); free(y); free(yh); free(yo); free(r); free(v); free(zh); free(zo);
    return -1;
  }
  if (z0) {
    for (int q = 0; q < d; ++q) z[q] = z0[q];
  } else {
    orc_weighted_mean_start(pts, w, n, d, lo, hi, z);
  }
  for (int q = 0; q < d; ++q) zh[q] = zo[q] = z[q];
  if (check_every < 1) check_every = 1;
  double alpha = 1.0, c_prev = INFINITY, rp = 0.0, rd = 0.0, marg = INFINITY;
  int t_done = 0, nrest = 0;
  for (int t = 1; t <= iters; ++t) {
    /* Algorithm 1's step at (z_hat, y_hat) */
    for (int q = 0; q < d; ++q) r[q] = 0.0;
    for (int k = 0; k < n; ++k) {
      double *xk = x + (size_t)k * d;
      const double *yk = yh + (size_t)k * d;
      for (int q = 0; q < d; ++q) v[q] = zh[q] - yk[q] / mu;
      orc_prox(v, pts + (size_t)k * d, w[k] / mu, d, xk);
      for (int q = 0; q < d; ++q) r[q] += xk[q] + yk[q] / mu;
    }
    for (int q = 0; q < d; ++q) z[q] = r[q] / (double)n;
    orc_project_box(z, d, lo, hi, z);
    double cy = 0.0, cz = 0.0;
    for (size_t i = 0; i < nd; ++i) {
      y[i] = yh[i] + mu * (x[i] - z[i % (size_t)d]);
      cy += (y[i] - yh[i]) * (y[i] - yh[i]);
    }
    for (int q = 0; q < d; ++q) cz += (z[q] - zh[q]) * (z[q] - zh[q]);
    t_done = t;
    /* the stopping rule of orc_em_admm at this step's iterate */
    int check = (t == iters) || (tol > 0.0 && (t % check_every) == 0);
    if (check) {
      double spr = 0.0, sx = 0.0, su = 0.0, zz = 0.0, dz = 0.0;
      for (size_t i = 0; i < nd; ++i) {
        double e = x[i] - z[i % (size_t)d], u = y[i] / mu;
        spr += e * e;
        sx += x[i] * x[i];
        su += u * u;
      }
      for (int q = 0; q < d; ++q) {
        zz += z[q] * z[q];
        dz += (z[q] - zh[q]) * (z[q] - zh[q]);
      }
      double den_p = sqrt(sx), nzn = sqrt((double)n) * sqrt(zz);
      if (nzn > den_p) den_p = nzn;
      if (den_p < 1e-30) den_p = 1e-30;
      double den_d = sqrt(su);
      if (den_d < 1e-30) den_d = 1e-30;
      rp = sqrt(spr) / den_p;
      rd = sqrt((double)n) * sqrt(dz) / den_d;
      if (tol > 0.0 && rp < tol && rd < tol) break;
    }
    /* momentum or restart */
    const double c = (combined ? cy / mu : 0.0) + mu * (double)n * cz;
    if (restart_every <= 0 && isfinite(c_prev)) {
      const double m = fabs(c / (eta * c_prev) - 1.0);
      if (m < marg) marg = m;
    }
    const int momentum = restart_every > 0 ? (t % restart_every) != 0 : c < eta * c_prev;
    if (momentum) {
      const double a1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * alpha * alpha));
      const double beta = (alpha - 1.0) / a1;
      for (int q = 0; q < d; ++q) zh[q] = z[q] + beta * (z[q] - zo[q]);
      for (size_t i = 0; i < nd; ++i) yh[i] = y[i] + beta * (y[i] - yo[i]);
      alpha = a1;
      c_prev = c;
    } else {
      alpha = 1.0;
      for (int q = 0; q < d; ++q) zh[q] = zo[q];
      for (size_t i = 0; i < nd; ++i) yh[i] = yo[i];
      c_prev = c_prev / eta;
      ++nrest;
    }
    for (int q = 0; q < d; ++q) zo[q] = z[q];
    for (size_t i = 0; i < nd; ++i) yo[i] = y[i];
  }
  if (iters_used) *iters_used = t_done;
  if (rpri) *rpri = rp;
  if (rdual) *rdual = rd;
  if (restarts) *restarts = nrest;
  if (margin) *margin = marg;
  free(x); free(y); free(yh); free(yo); free(r); free(v); free(zh); free(zo);
  return 0;
}

/* Constraint sets other than the box of Sec. 3 (the method needs only a closed convex C with a
 * simple projection, Sec. 2).  kind 1: per-coordinate boxes prod_q [pa[q], pb[q]], projected by
 * clamping each coordinate; kind 2: the ball ||x - pa|| <= r, projected by pulling x radially
 * onto the sphere when it lies outside.  Any other kind leaves x as it is. */
void orc_project_set(const double *x, int d, int kind, const double *pa, const double *pb, double r,
                     double *out) {
  if (kind == 1) {
    for (int q = 0; q < d; ++q) {
      double t = x[q];
      if (t < pa[q]) t = pa[q];
      if (t > pb[q]) t = pb[q];
      out[q] = t;
    }
  } else if (kind == 2) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s += (x[q] - pa[q]) * (x[q] - pa[q]);
    const double nr = sqrt(s);
    const double f = nr > r ? r / nr : 1.0;
    for (int q = 0; q < d; ++q) out[q] = pa[q] + f * (x[q] - pa[q]);
  } else {
    for (int q = 0; q < d; ++q) out[q] = x[q];
  }
}

/* Algorithm 1 with the z-update's projection onto the box [lo, hi]^d (kind 0) or onto the set of
 * orc_project_set (kind 1, 2); the start is z0 as given, else the weighted mean projected onto C. */
static int em_admm_impl(const double *pts, const double *w, int n, int d, int kind, double lo, double hi,
                        const double *pa, const double *pb, double rad, double mu, int iters,
                        const double *z0, double tol, int check_every, double *z, int *iters_used,
                        double *rpri, double *rdual);

int orc_em_admm(const double *pts, const double *w, int n, int d, double lo, double hi,
                double mu, int iters, const double *z0, double tol, int check_every,
                double *z, int *iters_used, double *rpri, double *rdual) {
  return em_admm_impl(pts, w, n, d, 0, lo, hi, NULL, NULL, 0.0, mu, iters, z0, tol, check_every, z,
                      iters_used, rpri, rdual);
}

int orc_em_admm_set(const double *pts, const double *w, int n, int d, int kind, const double *pa,
                    const double *pb, double rad, double mu, int iters, const double *z0, double tol,
                    int check_every, double *z, int *iters_used, double *rpri, double *rdual) {
  return em_admm_impl(pts, w, n, d, kind, 0.0, 0.0, pa, pb, rad, mu, iters, z0, tol, check_every, z,
                      iters_used, rpri, rdual);
}

static int em_admm_impl(const double *pts, const double *w, int n, int d, int kind, double lo, double hi,
                        const double *pa, const double *pb, double rad, double mu, int iters,
                        const double *z0, double tol, int check_every, double *z, int *iters_used,
                        double *rpri, double *rdual) {
  double *x = (double *)malloc(sizeof(double) * (size_t)n * d);
  double *y = (double *)calloc((size_t)n * d, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * (size_t)d);
  double *v = (double *)malloc(sizeof(double) * (size_t)d);
  double *zprev = (double *)malloc(sizeof(double) * (size_t)d);
  if (!x || !y || !r || !v || !zprev) {
    free(x); free(y); free(r); free(v); free(zprev);
    return -1;
  }
  if (z0) {
    for (int q = 0; q < d; ++q) z[q] = z0[q];
  } else if (kind == 0) {
    orc_weighted_mean_start(pts, w, n, d, lo, hi, z);
  } else {
    orc_weighted_mean_start(pts, w, n, d, -INFINITY, INFINITY, z);
    orc_project_set(z, d, kind, pa, pb, rad, z);
  }
  if (check_every < 1) check_every = 1;
  int t_done = 0;
  double rp = 0.0, rd = 0.0;
  for (int t = 1; t <= iters; ++t) {
    for (int q = 0; q < d; ++q) r[q] = 0.0;
    for (int k = 0; k < n; ++k) {
      double *xk = x + (size_t)k * d;
      const double *yk = y + (size_t)k * d;
      for (int q = 0; q < d; ++q) v[q] = z[q] - yk[q] / mu;
      orc_prox(v, pts + (size_t)k * d, w[k] / mu, d, xk);
      for (int q = 0; q < d; ++q) r[q] += xk[q] + yk[q] / mu;
    }
    for (int q = 0; q < d; ++q) {
      zprev[q] = z[q];
      z[q] = r[q] / (double)n;
    }
    if (kind == 0)
      orc_project_box(z, d, lo, hi, z);
    else
      orc_project_set(z, d, kind, pa, pb, rad, z);
    for (int k = 0; k < n; ++k) {
      double *yk = y + (size_t)k * d;
      const double *xk = x + (size_t)k * d;
      for (int q = 0; q < d; ++q) yk[q] += mu * (xk[q] - z[q]);
    }
    t_done = t;
    int check = (t == iters) || (tol > 0.0 && (t % check_every) == 0);
    if (check) {
      double spr = 0.0, sx = 0.0, su = 0.0, zz = 0.0, dz = 0.0;
      for (int k = 0; k < n; ++k) {
        for (int q = 0; q < d; ++q) {
          double xq = x[(size_t)k * d + q];
          double e = xq - z[q];
          double u = y[(size_t)k * d + q] / mu;
          spr += e * e;
          sx += xq * xq;
          su += u * u;
        }
      }
      for (int q = 0; q < d; ++q) {
        zz += z[q] * z[q];
        double e = z[q] - zprev[q];
        dz += e * e;
      }
      double den_p = sqrt(sx);
      double nzn = sqrt((double)n) * sqrt(zz);
      if (nzn > den_p) den_p = nzn;
      if (den_p < 1e-30) den_p = 1e-30;
      double den_d = sqrt(su);
      if (den_d < 1e-30) den_d = 1e-30;
      rp = sqrt(spr) / den_p;
      rd = sqrt((double)n) * sqrt(dz) / den_d;
      if (tol > 0.0 && rp < tol && rd < tol) break;
    }
  }
  if (iters_used) *iters_used = t_done;
  if (rpri) *rpri = rp;
  if (rdual) *rdual = rd;
  free(x); free(y); free(r); free(v); free(zprev);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * Cross-checks used by the tests (not part of the paper's method).
 * ------------------------------------------------------------------------------------- */

/* Weiszfeld iteration for the unconstrained weighted EM (Weiszfeld 1937, cited in Sec. 1):
 * x <- sum (w_k/||x-a_k||) a_k / sum (w_k/||x-a_k||).  Stops early if x lands on a point.
 * Writes the objective after every iteration into F_hist (nullable, length iters). */
void orc_weiszfeld(const double *pts, const double *w, int n, int d, const double *x0,
                   int iters, double *x, double *F_hist) {
  double *nx = (double *)malloc(sizeof(double) * (size_t)d);
  for (int q = 0; q < d; ++q) x[q] = x0[q];
  for (int t = 0; t < iters; ++t) {
    double den = 0.0;
    int on_point = 0;
    for (int q = 0; q < d; ++q) nx[q] = 0.0;
    for (int k = 0; k < n; ++k) {
      double r2 = 0.0;
      for (int q = 0; q < d; ++q) {
        double e = x[q] - pts[(size_t)k * d + q];
        r2 += e * e;
      }
      double r = sqrt(r2);
      if (r < 1e-300) { on_point = 1; break; }
      double c = w[k] / r;
      den += c;
      for (int q = 0; q < d; ++q) nx[q] += c * pts[(size_t)k * d + q];
    }
    if (!on_point && den > 0.0)
      for (int q = 0; q < d; ++q) x[q] = nx[q] / den;
    if (F_hist) F_hist[t] = orc_objective(x, pts, w, n, d);
  }
  free(nx);
}

/* IRLS on the smooth surrogate (2), sum w_k (||x-a_k||^2 + eps)^{1/2} (Sec. 1): the
 * stationarity condition gives x = sum om_k a_k / sum om_k with
 * om_k = w_k (||x-a_k||^2 + eps)^{-1/2}; C is enforced by projecting after every step. */
void orc_irls(const double *pts, const double *w, int n, int d, double lo, double hi,
              const double *x0, double eps, int iters, double *x, double *F_hist) {
  double *nx = (double *)malloc(sizeof(double) * (size_t)d);
  for (int q = 0; q < d; ++q) x[q] = x0[q];
  for (int t = 0; t < iters; ++t) {
    double den = 0.0;
    for (int q = 0; q < d; ++q) nx[q] = 0.0;
    for (int k = 0; k < n; ++k) {
      double r2 = 0.0;
      for (int q = 0; q < d; ++q) {
        double e = x[q] - pts[(size_t)k * d + q];
        r2 += e * e;
      }
      double c = w[k] / sqrt(r2 + eps);
      den += c;
      for (int q = 0; q < d; ++q) nx[q] += c * pts[(size_t)k * d + q];
    }
    if (den > 0.0)
      for (int q = 0; q < d; ++q) x[q] = nx[q] / den;
    orc_project_box(x, d, lo, hi, x);
    if (F_hist) F_hist[t] = orc_objective(x, pts, w, n, d);
  }
  free(nx);
}

/* ---------------------------------------------------------------------------------------
 * Batch driver: problems b = 0..B-1, float32 inputs, each solved by orc_em_admm.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  const float *pts, *w, *z0;
  long long B;
  int n, d, iters, check_every, nthreads, tid;
  double lo, hi, mu, tol;
  double *z;
  int *iters_used;
  double *rpri, *rdual;
  int status;
  int penalty;   /* 0: Algorithm 1; 1: per-point penalties mu_k = mu w_k (orc_em_admm_wpen);
                    2: accelerated Algorithm 1 (orc_em_admm_fast, eta = 0.999, the z-part test) */
  int *restarts;
  double *margin;
  int restart_every;   /* orc_em_admm_fast's fixed restart period (0: the residual test) */
} batch_job;

static void *batch_worker(void *arg) {
  batch_job *J = (batch_job *)arg;
  int n = J->n, d = J->d;
  double *a = (double *)malloc(sizeof(double) * (size_t)n * d);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *z0 = (double *)malloc(sizeof(double) * (size_t)d);
  if (!a || !w || !z0) { J->status = -1; free(a); free(w); free(z0); return NULL; }
  for (long long b = J->tid; b < J->B; b += J->nthreads) {
    for (size_t i = 0; i < (size_t)n * d; ++i) a[i] = (double)J->pts[(size_t)b * n * d + i];
    for (int k = 0; k < n; ++k) w[k] = (double)J->w[(size_t)b * n + k];
    const double *zs = NULL;
    if (J->z0) {
      for (int q = 0; q < d; ++q) z0[q] = (double)J->z0[(size_t)b * d + q];
      zs = z0;
    }
    int used = 0, nrest = 0;
    double rp = 0, rd = 0, marg = INFINITY;
    int rc;
    if (J->penalty == 2)
      rc = orc_em_admm_fast(a, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every, 0.999,
                            J->restart_every, 0, J->z + (size_t)b * d, &used, &rp, &rd, &nrest, &marg);
    else if (J->penalty == 1)
      rc = orc_em_admm_wpen(a, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every,
                            J->z + (size_t)b * d, &used, &rp, &rd);
    else
      rc = orc_em_admm(a, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every,
                       J->z + (size_t)b * d, &used, &rp, &rd);
    if (rc != 0) {
      J->status = -1;
      break;
    }
    if (J->restarts) J->restarts[b] = nrest;
    if (J->margin) J->margin[b] = marg;
    if (J->iters_used) J->iters_used[b] = used;
    if (J->rpri) J->rpri[b] = rp;
    if (J->rdual) J->rdual[b] = rd;
  }
  free(a); free(w); free(z0);
  return NULL;
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

int orc_num_cores(void) { return resolve_threads(0); }

int orc_em_admm_batch(const float *pts, const float *w, long long B, int n, int d, double lo,
                      double hi, double mu, int iters, const float *z0, double tol,
                      int check_every, double *z, int *iters_used, double *rpri,
                      double *rdual, int nthreads, int penalty, int *restarts, double *margin,
                      int restart_every) {
  int T = resolve_threads(nthreads);
  if ((long long)T > B) T = (int)(B > 0 ? B : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  batch_job *jobs = (batch_job *)malloc(sizeof(batch_job) * (size_t)T);
  for (int i = 0; i < T; ++i) {
    batch_job J = {pts, w, z0, B, n, d, iters, check_every, T, i, lo, hi, mu, tol,
                   z, iters_used, rpri, rdual, 0, penalty, restarts, margin, restart_every};
    jobs[i] = J;
    pthread_create(&th[i], NULL, batch_worker, &jobs[i]);
  }
  int status = 0;
  for (int i = 0; i < T; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].status) status = jobs[i].status;
  }
  free(th);
  free(jobs);
  return status;
}

/* ---------------------------------------------------------------------------------------
 * NLEM (Sec. 3).  For pixel i: P_j = k x k patch of g centred at j (reflect-padded, no edge
 * repeat), S(i) = pixels of the S x S window centred at i that lie in the image (row-major
 * order), w_ij = exp(-||P_i - P_j||^2 / h^2), solve problem (L1regression) over
 * C = [lo,hi]^{k^2} with Algorithm 1 and output the centre coordinate of the solution.
 *
 * weight_mode 0: squared distance in double from the float image.
 * weight_mode 1: mixed-precision model: ||P_i||^2 + ||P_j||^2 - 2 <bf16(P_i), bf16(P_j)>,
 *                norms from the float values, the cross term from values rounded to bfloat16
 *                (round to nearest even), everything else in double.
 * init_mode 0: z0 = P_C(weighted mean of the patches) (the NLM patch); 1: z0 = P_C(P_i).
 * pix == NULL processes every pixel (row-major); otherwise the npix listed linear indices.
 * out[i], iters_used[i], rpri/rdual[i] refer to the i-th processed pixel.
 * ------------------------------------------------------------------------------------- */
static inline int reflect_index(int x, int N) {
  if (x < 0) return -x;
  if (x >= N) return 2 * N - 2 - x;
  return x;
}

static double round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (double)f;  /* inf / nan unchanged */
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return (double)r;
}

typedef struct {
  const float *img;
  int H, W, k, S, iters, check_every, init_mode, weight_mode, nthreads, tid;
  double h, mu, lo, hi, tol;
  const long long *pix;
  long long npix;
  double *out, *rpri, *rdual, *wsum_out;
  int *iters_used, *n_out;
  int status;
  int penalty;   /* 0: Algorithm 1; 1: per-point penalties mu_k = mu w_k (orc_em_admm_wpen);
                    2: accelerated Algorithm 1 (orc_em_admm_fast, eta = 0.999, the z-part test) */
  int *restarts;
  double *margin;
  int restart_every;   /* orc_em_admm_fast's fixed restart period (0: the residual test) */
} nlem_job;

/* Patch of g centred at (r, c), reflect-padded, row-major k x k, as double. */
static void extract_patch(const float *img, int H, int W, int k, int r, int c, double *p) {
  int hk = (k - 1) / 2;
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b)
      p[a * k + b] = (double)img[(size_t)reflect_index(r - hk + a, H) * W +
                                 reflect_index(c - hk + b, W)];
}

static void *nlem_worker(void *arg) {
  nlem_job *J = (nlem_job *)arg;
  int k = J->k, d = k * k, S = J->S, R = (S - 1) / 2;
  int nmax = S * S;
  double *pts = (double *)malloc(sizeof(double) * (size_t)nmax * d);
  double *w = (double *)malloc(sizeof(double) * (size_t)nmax);
  double *pc = (double *)malloc(sizeof(double) * (size_t)d);
  double *z = (double *)malloc(sizeof(double) * (size_t)d);
  double *z0 = (double *)malloc(sizeof(double) * (size_t)d);
  float *pcf = (float *)malloc(sizeof(float) * (size_t)d);
  if (!pts || !w || !pc || !z || !z0 || !pcf) { J->status = -1; goto done; }
  long long total = J->pix ? J->npix : (long long)J->H * J->W;
  for (long long t = J->tid; t < total; t += J->nthreads) {
    long long lin = J->pix ? J->pix[t] : t;
    int ir = (int)(lin / J->W), ic = (int)(lin % J->W);
    extract_patch(J->img, J->H, J->W, k, ir, ic, pc);
    int r0 = ir - R < 0 ? 0 : ir - R, r1 = ir + R > J->H - 1 ? J->H - 1 : ir + R;
    int c0 = ic - R < 0 ? 0 : ic - R, c1 = ic + R > J->W - 1 ? J->W - 1 : ic + R;
    int n = 0;
    for (int jr = r0; jr <= r1; ++jr) {
      for (int jc = c0; jc <= c1; ++jc) {
        double *pj = pts + (size_t)n * d;
        extract_patch(J->img, J->H, J->W, k, jr, jc, pj);
        double D;
        if (J->weight_mode == 0) {
          D = 0.0;
          for (int q = 0; q < d; ++q) {
            double e = pc[q] - pj[q];
            D += e * e;
          }
        } else {
          double ni = 0.0, nj = 0.0, x = 0.0;
          for (int q = 0; q < d; ++q) {
            ni += pc[q] * pc[q];
            nj += pj[q] * pj[q];
            x += round_bf16((float)pc[q]) * round_bf16((float)pj[q]);
          }
          D = ni + nj - 2.0 * x;
          if (D < 0.0) D = 0.0;
        }
        w[n] = exp(-D / (J->h * J->h));
        ++n;
      }
    }
    const double *zs = NULL;
    if (J->init_mode == 1) {
      orc_project_box(pc, d, J->lo, J->hi, z0);
      zs = z0;
    }
    int used = 0, nrest = 0;
    double rp = 0, rd = 0, marg = INFINITY;
    int rc;
    if (J->penalty == 2)
      rc = orc_em_admm_fast(pts, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every, 0.999,
                            J->restart_every, 0, z, &used, &rp, &rd, &nrest, &marg);
    else if (J->penalty == 1)
      rc = orc_em_admm_wpen(pts, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every, z, &used,
                            &rp, &rd);
    else
      rc = orc_em_admm(pts, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every, z, &used, &rp,
                       &rd);
    if (rc != 0) {
      J->status = -1;
      break;
    }
    if (J->restarts) J->restarts[t] = nrest;
    if (J->margin) J->margin[t] = marg;
    J->out[t] = z[(d - 1) / 2];
    if (J->iters_used) J->iters_used[t] = used;
    if (J->rpri) J->rpri[t] = rp;
    if (J->rdual) J->rdual[t] = rd;
    if (J->n_out) J->n_out[t] = n;
    if (J->wsum_out) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += w[j];
      J->wsum_out[t] = s;
    }
  }
done:
  free(pts); free(w); free(pc); free(z); free(z0); free(pcf);
  return NULL;
}

int orc_nlem(const float *img, int H, int W, int k, int S, double h, double mu, int iters,
             double lo, double hi, double tol, int check_every, int init_mode, int weight_mode,
             const long long *pix, long long npix, double *out, int *iters_used, double *rpri,
             double *rdual, int *n_out, double *wsum_out, int nthreads, int penalty, int *restarts,
             double *margin, int restart_every) {
  int T = resolve_threads(nthreads);
  long long total = pix ? npix : (long long)H * W;
  if ((long long)T > total) T = (int)(total > 0 ? total : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  nlem_job *jobs = (nlem_job *)malloc(sizeof(nlem_job) * (size_t)T);
  for (int i = 0; i < T; ++i) {
    nlem_job J = {img, H, W, k, S, iters, check_every, init_mode, weight_mode, T, i,
                  h, mu, lo, hi, tol, pix, npix, out, rpri, rdual, wsum_out, iters_used, n_out, 0, penalty,
                  restarts, margin, restart_every};
    jobs[i] = J;
    pthread_create(&th[i], NULL, nlem_worker, &jobs[i]);
  }
  int status = 0;
  for (int i = 0; i < T; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].status) status = jobs[i].status;
  }
  free(th);
  free(jobs);
  return status;
}

/* The problem (points, weights) the NLEM driver builds for one pixel; used by tests that
 * check the NLEM assembly separately from the solver.  pts must hold S*S*k*k doubles and
 * w S*S; returns n. */
int orc_nlem_problem(const float *img, int H, int W, int k, int S, double h, long long lin,
                     int weight_mode, double *pts, double *w, double *pc) {
  int d = k * k, R = (S - 1) / 2;
  int ir = (int)(lin / W), ic = (int)(lin % W);
  extract_patch(img, H, W, k, ir, ic, pc);
  int r0 = ir - R < 0 ? 0 : ir - R, r1 = ir + R > H - 1 ? H - 1 : ir + R;
  int c0 = ic - R < 0 ? 0 : ic - R, c1 = ic + R > W - 1 ? W - 1 : ic + R;
  int n = 0;
  for (int jr = r0; jr <= r1; ++jr)
    for (int jc = c0; jc <= c1; ++jc) {
      double *pj = pts + (size_t)n * d;
      extract_patch(img, H, W, k, jr, jc, pj);
      double D = 0.0;
      if (weight_mode == 0) {
        for (int q = 0; q < d; ++q) { double e = pc[q] - pj[q]; D += e * e; }
      } else {
        double ni = 0.0, nj = 0.0, x = 0.0;
        for (int q = 0; q < d; ++q) {
          ni += pc[q] * pc[q];
          nj += pj[q] * pj[q];
          x += round_bf16((float)pc[q]) * round_bf16((float)pj[q]);
        }
        D = ni + nj - 2.0 * x;
        if (D < 0.0) D = 0.0;
      }
      w[n] = exp(-D / (h * h));
      ++n;
    }
  return n;
}

/* ---------------------------------------------------------------------------------------
 * Learned warm start (not in the paper): problem features and a small MLP, for checking the
 * GPU feature, forward and backward kernels.
 * ------------------------------------------------------------------------------------- */

typedef struct {
  double v, w;
} vw_pair;

static int cmp_vw(const void *a, const void *b) {
  double x = ((const vw_pair *)a)->v, y = ((const vw_pair *)b)->v;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Features of problem (1): f = [m (d), q (d), H, pmax] with p_k = w_k / sum w,
 * m = sum p_k a_k (weighted mean, not projected), q_c = lower weighted median of coordinate c
 * (the smallest value whose cumulative weight in ascending order reaches half the total),
 * H = -sum_{p_k > 0} p_k log p_k, pmax = max p_k.  All weights zero: p uniform. */
void orc_features(const double *pts, const double *w, int n, int d, double *f) {
  double W = 0.0;
  for (int k = 0; k < n; ++k) W += w[k];
  vw_pair *buf = (vw_pair *)malloc(sizeof(vw_pair) * (size_t)n);
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += (W > 0.0 ? w[k] / W : 1.0 / n) * pts[(size_t)k * d + c];
    f[c] = s;
    for (int k = 0; k < n; ++k) {
      buf[k].v = pts[(size_t)k * d + c];
      buf[k].w = W > 0.0 ? w[k] : 1.0;
    }
    qsort(buf, (size_t)n, sizeof(vw_pair), cmp_vw);
    double tot = 0.0, cum = 0.0;
    for (int k = 0; k < n; ++k) tot += buf[k].w;
    double med = buf[n - 1].v;
    for (int k = 0; k < n; ++k) {
      cum += buf[k].w;
      if (cum >= 0.5 * tot) {
        med = buf[k].v;
        break;
      }
    }
    f[d + c] = med;
  }
  double H = 0.0, pmax = 0.0;
  for (int k = 0; k < n; ++k) {
    double p = W > 0.0 ? w[k] / W : 1.0 / n;
    if (p > 0.0) H -= p * log(p);
    if (p > pmax) pmax = p;
  }
  f[2 * d] = H;
  f[2 * d + 1] = pmax;
  free(buf);
}

/* MLP  x = normalise(f);  h1 = relu(W1 x + b1);  h2 = relu(W2 h1 + b2);  y = W3 h2 + b3
 * with F = 2d+2 inputs, Hd hidden units, O = d+1 outputs.  normalise: coordinates of m and q
 * -> (v - 127.5) / 64, H -> H / log(nref), pmax unchanged.
 * Parameter vector (row-major): W1 [Hd][F], b1 [Hd], W2 [Hd][Hd], b2 [Hd], W3 [O][Hd], b3 [O].
 * Loss of a batch: L = (1/B) sum_b [ (1/d) sum_{c<d} (y_bc - t_bc)^2 + (y_bd - t_bd)^2 ]. */
static void mlp_normalise(const double *f, int d, double nref, double *x) {
  for (int c = 0; c < 2 * d; ++c) x[c] = (f[c] - 127.5) / 64.0;
  x[2 * d] = f[2 * d] / log(nref);
  x[2 * d + 1] = f[2 * d + 1];
}

void orc_mlp_forward(const double *prm, int d, int Hd, double nref, const double *f, long long B, double *y) {
  int F = 2 * d + 2, O = d + 1;
  const double *W1 = prm, *b1 = W1 + (size_t)Hd * F, *W2 = b1 + Hd, *b2 = W2 + (size_t)Hd * Hd;
  const double *W3 = b2 + Hd, *b3 = W3 + (size_t)O * Hd;
  double *x = (double *)malloc(sizeof(double) * (size_t)F);
  double *h1 = (double *)malloc(sizeof(double) * (size_t)Hd);
  double *h2 = (double *)malloc(sizeof(double) * (size_t)Hd);
  for (long long b = 0; b < B; ++b) {
    mlp_normalise(f + (size_t)b * F, d, nref, x);
    for (int i = 0; i < Hd; ++i) {
      double s = b1[i];
      for (int j = 0; j < F; ++j) s += W1[(size_t)i * F + j] * x[j];
      h1[i] = s > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < Hd; ++i) {
      double s = b2[i];
      for (int j = 0; j < Hd; ++j) s += W2[(size_t)i * Hd + j] * h1[j];
      h2[i] = s > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < O; ++i) {
      double s = b3[i];
      for (int j = 0; j < Hd; ++j) s += W3[(size_t)i * Hd + j] * h2[j];
      y[(size_t)b * O + i] = s;
    }
  }
  free(x); free(h1); free(h2);
}

/* Loss and its gradient with respect to every parameter (backpropagation, FP64). */
double orc_mlp_loss_grad(const double *prm, int d, int Hd, double nref, const double *f, const double *t,
                         long long B, double *grad) {
  int F = 2 * d + 2, O = d + 1;
  size_t P = (size_t)Hd * F + Hd + (size_t)Hd * Hd + Hd + (size_t)O * Hd + O;
  const double *W1 = prm, *b1 = W1 + (size_t)Hd * F, *W2 = b1 + Hd, *b2 = W2 + (size_t)Hd * Hd;
  const double *W3 = b2 + Hd, *b3 = W3 + (size_t)O * Hd;
  double *gW1 = grad, *gb1 = gW1 + (size_t)Hd * F, *gW2 = gb1 + Hd, *gb2 = gW2 + (size_t)Hd * Hd;
  double *gW3 = gb2 + Hd, *gb3 = gW3 + (size_t)O * Hd;
  for (size_t i = 0; i < P; ++i) grad[i] = 0.0;
  double *x = (double *)malloc(sizeof(double) * (size_t)F);
  double *a1 = (double *)malloc(sizeof(double) * (size_t)Hd), *h1 = (double *)malloc(sizeof(double) * (size_t)Hd);
  double *a2 = (double *)malloc(sizeof(double) * (size_t)Hd), *h2 = (double *)malloc(sizeof(double) * (size_t)Hd);
  double *y = (double *)malloc(sizeof(double) * (size_t)O), *dy = (double *)malloc(sizeof(double) * (size_t)O);
  double *dh2 = (double *)malloc(sizeof(double) * (size_t)Hd), *dh1 = (double *)malloc(sizeof(double) * (size_t)Hd);
  double L = 0.0;
  for (long long b = 0; b < B; ++b) {
    mlp_normalise(f + (size_t)b * F, d, nref, x);
    for (int i = 0; i < Hd; ++i) {
      double s = b1[i];
      for (int j = 0; j < F; ++j) s += W1[(size_t)i * F + j] * x[j];
      a1[i] = s;
      h1[i] = s > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < Hd; ++i) {
      double s = b2[i];
      for (int j = 0; j < Hd; ++j) s += W2[(size_t)i * Hd + j] * h1[j];
      a2[i] = s;
      h2[i] = s > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < O; ++i) {
      double s = b3[i];
      for (int j = 0; j < Hd; ++j) s += W3[(size_t)i * Hd + j] * h2[j];
      y[i] = s;
    }
    const double *tb = t + (size_t)b * O;
    for (int i = 0; i < O; ++i) {
      double e = y[i] - tb[i];
      double wgt = i < d ? 1.0 / d : 1.0;
      L += wgt * e * e;
      dy[i] = 2.0 * wgt * e / (double)B;
    }
    for (int j = 0; j < Hd; ++j) dh2[j] = 0.0;
    for (int i = 0; i < O; ++i) {
      gb3[i] += dy[i];
      for (int j = 0; j < Hd; ++j) {
        gW3[(size_t)i * Hd + j] += dy[i] * h2[j];
        dh2[j] += W3[(size_t)i * Hd + j] * dy[i];
      }
    }
    for (int j = 0; j < Hd; ++j) dh1[j] = 0.0;
    for (int i = 0; i < Hd; ++i) {
      double da = a2[i] > 0.0 ? dh2[i] : 0.0;
      gb2[i] += da;
      for (int j = 0; j < Hd; ++j) {
        gW2[(size_t)i * Hd + j] += da * h1[j];
        dh1[j] += W2[(size_t)i * Hd + j] * da;
      }
    }
    for (int i = 0; i < Hd; ++i) {
      double da = a1[i] > 0.0 ? dh1[i] : 0.0;
      gb1[i] += da;
      for (int j = 0; j < F; ++j) gW1[(size_t)i * F + j] += da * x[j];
    }
  }
  free(x); free(a1); free(h1); free(a2); free(h2); free(y); free(dy); free(dh2); free(dh1);
  return L / (double)B;
}
