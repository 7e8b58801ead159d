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
int orc_em_admm(const double *pts, const double *w, int n, int d, double lo, double hi,
                double mu, int iters, const double *z0, double tol, int check_every,
                double *z, int *iters_used, double *rpri, double *rdual) {
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
      const double *yk = y + (size_t)k * d;
      for (int q = 0; q < d; ++q) v[q] = z[q] - yk[q] / mu;
      orc_prox(v, pts + (size_t)k * d, w[k] / mu, d, xk);
      for (int q = 0; q < d; ++q) r[q] += xk[q] + yk[q] / mu;
    }
    for (int q = 0; q < d; ++q) {
      zprev[q] = z[q];
      z[q] = r[q] / (double)n;
    }
    orc_project_box(z, d, lo, hi, z);
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
    int used = 0;
    double rp = 0, rd = 0;
    if (orc_em_admm(a, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every,
                    J->z + (size_t)b * d, &used, &rp, &rd) != 0) {
      J->status = -1;
      break;
    }
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
                      double *rdual, int nthreads) {
  int T = resolve_threads(nthreads);
  if ((long long)T > B) T = (int)(B > 0 ? B : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  batch_job *jobs = (batch_job *)malloc(sizeof(batch_job) * (size_t)T);
  for (int i = 0; i < T; ++i) {
    batch_job J = {pts, w, z0, B, n, d, iters, check_every, T, i, lo, hi, mu, tol,
                   z, iters_used, rpri, rdual, 0};
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
    int used = 0;
    double rp = 0, rd = 0;
    if (orc_em_admm(pts, w, n, d, J->lo, J->hi, J->mu, J->iters, zs, J->tol, J->check_every,
                    z, &used, &rp, &rd) != 0) {
      J->status = -1;
      break;
    }
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
             double *rdual, int *n_out, double *wsum_out, int nthreads) {
  int T = resolve_threads(nthreads);
  long long total = pix ? npix : (long long)H * W;
  if ((long long)T > total) T = (int)(total > 0 ? total : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)T);
  nlem_job *jobs = (nlem_job *)malloc(sizeof(nlem_job) * (size_t)T);
  for (int i = 0; i < T; ++i) {
    nlem_job J = {img, H, W, k, S, iters, check_every, init_mode, weight_mode, T, i,
                  h, mu, lo, hi, tol, pix, npix, out, rpri, rdual, wsum_out, iters_used, n_out, 0};
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
