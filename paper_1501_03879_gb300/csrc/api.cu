// C ABI of libnlem.so (declared in include/nlem.h): argument validation, context and
// workspace ownership, dispatch to the kernels, and error reporting without exceptions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/nlem.h"
#include "batch.h"
#include "kernels.h"
#include "trace.h"

#include "ctx.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(NLEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite(float x) { return std::isfinite(x); }

int check_common(nlem_ctx* ctx, nlem_box box, float rho, int iters, const nlem_options* opt) {
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  if (!(rho > 0.f) || !finite(rho)) return fail(NLEM_ERR_INVALID, "rho must be finite and > 0 (got %g)", rho);
  if (iters < 0) return fail(NLEM_ERR_INVALID, "iters must be >= 0 (got %d)", iters);
  if (!finite(box.lo) || !finite(box.hi) || box.lo > box.hi)
    return fail(NLEM_ERR_INVALID, "box must satisfy lo <= hi, both finite (got [%g, %g])", box.lo, box.hi);
  if (opt) {
    if (opt->check_every < 1) return fail(NLEM_ERR_INVALID, "check_every must be >= 1");
    if (!std::isfinite(opt->tol)) return fail(NLEM_ERR_INVALID, "tol must be finite");
    if (opt->precision != NLEM_PREC_FP32 && opt->precision != NLEM_PREC_BF16)
      return fail(NLEM_ERR_INVALID, "unknown precision %d", opt->precision);
    if (opt->init != NLEM_INIT_WEIGHTED_MEAN && opt->init != NLEM_INIT_NOISY_PATCH)
      return fail(NLEM_ERR_INVALID, "unknown init %d", opt->init);
    if (opt->layout < NLEM_LAYOUT_AUTO || opt->layout > NLEM_LAYOUT_PAIR)
      return fail(NLEM_ERR_INVALID, "unknown layout %d", opt->layout);
    if (opt->solver != NLEM_SOLVER_ADMM && opt->solver != NLEM_SOLVER_IRLS && opt->solver != NLEM_SOLVER_FAST)
      return fail(NLEM_ERR_INVALID, "unknown solver %d", opt->solver);
    if (opt->restart_every < 0)
      return fail(NLEM_ERR_INVALID, "restart_every must be >= 0 (got %d)", opt->restart_every);
    if (opt->solver == NLEM_SOLVER_IRLS) {
      if (!(opt->irls_eps >= 1e-30f) || !finite(opt->irls_eps))
        return fail(NLEM_ERR_INVALID, "irls_eps must be finite and >= 1e-30 (got %g)", opt->irls_eps);
      if (opt->tol > 0.f) return fail(NLEM_ERR_INVALID, "IRLS runs a fixed number of steps: tol must be <= 0");
    }
    if (opt->penalty != NLEM_PENALTY_UNIFORM && opt->penalty != NLEM_PENALTY_WEIGHTED)
      return fail(NLEM_ERR_INVALID, "unknown penalty %d", opt->penalty);
    if (opt->penalty == NLEM_PENALTY_WEIGHTED && opt->solver == NLEM_SOLVER_IRLS)
      return fail(NLEM_ERR_INVALID, "per-point penalties belong to EM-ADMM, not IRLS");
    if (opt->penalty == NLEM_PENALTY_WEIGHTED && opt->solver == NLEM_SOLVER_FAST)
      return fail(NLEM_ERR_UNSUPPORTED, "the accelerated solver takes one penalty for every point");
  }
  return NLEM_OK;
}

// Entry points of standalone problems: EM-ADMM or its accelerated form (IRLS is nlem_denoise's).
int no_irls(const nlem_options* opt, const char* who) {
  if (opt && opt->solver == NLEM_SOLVER_IRLS)
    return fail(NLEM_ERR_INVALID, "%s runs EM-ADMM only (plain or accelerated), not IRLS", who);
  return NLEM_OK;
}

// The accelerated solver's shapes: d = 49, at most nlemk::fast_capacity() points.
int fast_shape(const nlem_options* opt, int n, int d) {
  if (opt && opt->solver == NLEM_SOLVER_FAST && (d != 49 || n > nlemk::fast_capacity()))
    return fail(NLEM_ERR_UNSUPPORTED, "the accelerated solver is compiled for d = 49 and n <= %d (got n = %d, d = %d)",
                nlemk::fast_capacity(), n, d);
  return NLEM_OK;
}

// Entry points whose kernels take one penalty for every point (Algorithm 1) only.
int uniform_penalty_only(const nlem_options* opt, const char* who) {
  if (opt && opt->penalty != NLEM_PENALTY_UNIFORM)
    return fail(NLEM_ERR_UNSUPPORTED, "%s solves with one penalty for every point only", who);
  return NLEM_OK;
}

// Entry points whose kernels run EM-ADMM only.
int admm_only(const nlem_options* opt, const char* who) {
  if (opt && opt->solver != NLEM_SOLVER_ADMM)
    return fail(NLEM_ERR_INVALID, "%s runs EM-ADMM only (solver %d)", who, opt->solver);
  return NLEM_OK;
}

nlemk::SolveParams make_params(nlem_box box, float rho, int iters, const nlem_options* opt, int d) {
  nlemk::SolveParams p;
  p.lo = box.lo;
  p.hi = box.hi;
  p.mu = rho;
  p.inv_mu = 1.f / rho;
  p.iters = iters;
  p.tol = opt ? opt->tol : 0.f;
  p.check_every = opt ? opt->check_every : 1;
  p.d = d;
  p.solver = opt ? opt->solver : NLEM_SOLVER_ADMM;
  p.eps = opt ? opt->irls_eps : 1e-6f;
  p.restart_every = opt ? opt->restart_every : 0;
  return p;
}

int set_device(nlem_ctx* ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return NLEM_OK;
}

}  // namespace

namespace nlemk {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace nlemk

extern "C" {

void nlem_options_default(nlem_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tol = 0.f;
  opt->check_every = 1;
  opt->precision = NLEM_PREC_FP32;
  opt->init = NLEM_INIT_WEIGHTED_MEAN;
  opt->fp64_check = 0;
  opt->layout = NLEM_LAYOUT_AUTO;
  opt->solver = NLEM_SOLVER_ADMM;
  opt->irls_eps = 1e-6f;
  opt->penalty = NLEM_PENALTY_UNIFORM;
  opt->restart_every = 0;
}

const char* nlem_last_error(void) { return g_err.c_str(); }

const char* nlem_version(void) { return "nlem-gb300 0.1 (sm_103a)"; }

int nlem_ctx_create(nlem_ctx** ctx, int device) {
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx out-pointer is NULL");
  *ctx = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(NLEM_ERR_INVALID, "device %d out of range (%d devices)", device, count);
  nlem_ctx* c = new (std::nothrow) nlem_ctx();
  if (!c) return fail(NLEM_ERR_OOM, "out of host memory");
  c->device = device;
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute(MultiProcessorCount)");
  }
  *ctx = c;
  return NLEM_OK;
}

int nlem_ctx_destroy(nlem_ctx* ctx) {
  if (!ctx) return NLEM_OK;
  cudaSetDevice(ctx->device);
  if (ctx->have_plan && ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  cudaFree(ctx->ws_img);
  cudaFree(ctx->ws_out);
  cudaFree(ctx->ws_iters);
  cudaFree(ctx->ws_batch);
  cudaFree(ctx->ws_queue);
  cudaFree(ctx->ws_wtab);
  cudaFree(ctx->ws_err);
  cudaFree(ctx->ws_feats);
  cudaFree(ctx->ws_y);
  cudaFree(ctx->ws_x0);
  cudaFree(ctx->ws_rho);
  cudaFree(ctx->ws_list);
  cudaFree(ctx->ws_ulist);
  cudaFree(ctx->ws_count);
  cudaFree(ctx->lab_out);
  cudaFree(ctx->lab_iters);
  cudaFree(ctx->lab_rho_map);
  cudaFree(ctx->lab_z);
  cudaFree(ctx->lab_best_it);
  cudaFree(ctx->lab_best_rho);
  cudaFree(ctx->lab_grid);
  cudaFree(ctx->lab_counts);
  cudaFree(ctx->ws_em);
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
    if (ctx->ev_done[i]) cudaEventDestroy(ctx->ev_done[i]);
  }
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  delete ctx;
  return NLEM_OK;
}

int em_solve_batch(nlem_ctx* ctx, const float* points, const float* weights, long long B, int n, int d,
                   nlem_box box, float rho, int iters, const float* x0, const nlem_options* opt,
                   float* x_out, int* iters_used, float* residual, double* obj64, double* kkt64,
                   void* stream) {
  NLEM_TRACE("em_solve_batch");
  int rc = check_common(ctx, box, rho, iters, opt);
  if (rc) return rc;
  if ((rc = no_irls(opt, "em_solve_batch"))) return rc;
  if (B < 0) return fail(NLEM_ERR_INVALID, "B must be >= 0");
  if (n < 1) return fail(NLEM_ERR_INVALID, "n must be >= 1 (got %d)", n);
  if (d < 1 || d > 148) return fail(NLEM_ERR_INVALID, "d must be in [1, 148] (got %d)", d);
  if (B == 0) return NLEM_OK;   // an empty batch may pass NULL buffers
  if (!points || !weights || !x_out) return fail(NLEM_ERR_INVALID, "points, weights and x_out must be non-NULL");
  if ((rc = fast_shape(opt, n, d))) return rc;
  if (n > nlemk::em_capacity(d))
    return fail(NLEM_ERR_UNSUPPORTED, "n = %d, d = %d exceeds the on-chip solver (max n %d for this d)", n,
                d, nlemk::em_capacity(d));
  if ((rc = set_device(ctx))) return rc;
  nlemk::EmLaunch L;
  L.pts = points;
  L.w = weights;
  L.B = B;
  L.n = n;
  L.d = d;
  L.prm = make_params(box, rho, iters, opt, d);
  L.x0 = x0;
  L.x_out = x_out;
  L.iters_used = iters_used;
  L.resid = residual;
  const bool chk = opt && opt->fp64_check;
  L.obj64 = chk ? obj64 : nullptr;
  L.kkt64 = chk ? kkt64 : nullptr;
  L.sm_count = ctx->sm_count;
  L.stream = (cudaStream_t)stream;
  L.penalty = opt ? opt->penalty : NLEM_PENALTY_UNIFORM;
  int e = nlemk::launch_em_batch(L);
  if (e == -1 && L.penalty != NLEM_PENALTY_UNIFORM)
    return fail(NLEM_ERR_UNSUPPORTED, "per-point penalties are compiled for d = 49 (got d = %d)", d);
  if (e == -1) return fail(NLEM_ERR_UNSUPPORTED, "no kernel shape for n = %d, d = %d", n, d);
  if (e != 0) return cuda_fail((cudaError_t)e, "em_solve_batch launch");
  return NLEM_OK;
}

int em_solve_batch_set(nlem_ctx* ctx, const float* points, const float* weights, long long B, int n, int d,
                       const nlem_set* set, float rho, int iters, const float* x0, const nlem_options* opt,
                       float* x_out, int* iters_used, float* residual, void* stream) {
  NLEM_TRACE("em_solve_batch_set");
  const nlem_box any = {0.f, 0.f};
  int rc = check_common(ctx, any, rho, iters, opt);
  if (rc) return rc;
  if ((rc = admm_only(opt, "em_solve_batch_set"))) return rc;
  if ((rc = uniform_penalty_only(opt, "em_solve_batch_set"))) return rc;
  if (!set) return fail(NLEM_ERR_INVALID, "set is NULL");
  if (set->kind == NLEM_SET_COORD_BOXES) {
    if (!set->lo || !set->hi) return fail(NLEM_ERR_INVALID, "coordinate boxes need lo and hi");
  } else if (set->kind == NLEM_SET_BALL) {
    if (!set->center) return fail(NLEM_ERR_INVALID, "the ball needs its centre");
    if (!(set->radius >= 0.f) || !finite(set->radius))
      return fail(NLEM_ERR_INVALID, "radius must be finite and >= 0 (got %g)", set->radius);
  } else {
    return fail(NLEM_ERR_INVALID, "unknown set kind %d", set->kind);
  }
  if (B < 0) return fail(NLEM_ERR_INVALID, "B must be >= 0");
  if (n < 1) return fail(NLEM_ERR_INVALID, "n must be >= 1 (got %d)", n);
  if (d < 1 || d > 148) return fail(NLEM_ERR_INVALID, "d must be in [1, 148] (got %d)", d);
  if (B == 0) return NLEM_OK;
  if (!points || !weights || !x_out) return fail(NLEM_ERR_INVALID, "points, weights and x_out must be non-NULL");
  if (n > nlemk::em_set_capacity(d))
    return fail(NLEM_ERR_UNSUPPORTED, "n = %d exceeds the %d points the set kernels hold for d = %d", n,
                nlemk::em_set_capacity(d), d);
  if (opt && opt->fp64_check)
    return fail(NLEM_ERR_UNSUPPORTED, "the FP64 check is the box's; not available for other sets");
  if ((rc = set_device(ctx))) return rc;
  nlemk::EmLaunch L;
  L.pts = points;
  L.w = weights;
  L.B = B;
  L.n = n;
  L.d = d;
  L.prm = make_params(any, rho, iters, opt, d);
  L.x0 = x0;
  L.x_out = x_out;
  L.iters_used = iters_used;
  L.resid = residual;
  L.obj64 = nullptr;
  L.kkt64 = nullptr;
  L.sm_count = ctx->sm_count;
  L.stream = (cudaStream_t)stream;
  const float* a = set->kind == NLEM_SET_BALL ? set->center : set->lo;
  const int e = nlemk::launch_em_set(L, set->kind, a, set->hi, set->radius);
  if (e == -1) return fail(NLEM_ERR_UNSUPPORTED, "no kernel shape for n = %d, d = %d", n, d);
  if (e != 0) return cuda_fail((cudaError_t)e, "em_solve_batch_set launch");
  return NLEM_OK;
}

int em_solve(nlem_ctx* ctx, const float* points, const float* weights, int n, int d, nlem_box box, float rho,
             int iters, float* x_out, void* stream) {
  NLEM_TRACE("em_solve");
  return em_solve_batch(ctx, points, weights, 1, n, d, box, rho, iters, nullptr, nullptr, x_out, nullptr, nullptr,
                        nullptr, nullptr, stream);
}

int em_solve_batch_host(nlem_ctx* ctx, const float* points_host, const float* weights_host, long long B, int n,
                        int d, nlem_box box, float rho, int iters, const float* x0_host, const nlem_options* opt,
                        long long chunk, float* x_out_host, int* iters_used_host, float* residual_host,
                        void* stream) {
  NLEM_TRACE("em_solve_batch_host");
  int rc = check_common(ctx, box, rho, iters, opt);
  if (rc) return rc;
  if ((rc = no_irls(opt, "em_solve_batch_host"))) return rc;
  if ((rc = fast_shape(opt, n, d))) return rc;
  if (B < 0) return fail(NLEM_ERR_INVALID, "B must be >= 0");
  if (n < 1) return fail(NLEM_ERR_INVALID, "n must be >= 1 (got %d)", n);
  if (d < 1 || d > 148) return fail(NLEM_ERR_INVALID, "d must be in [1, 148] (got %d)", d);
  if (chunk < 0) return fail(NLEM_ERR_INVALID, "chunk must be >= 0 (got %lld)", chunk);
  if (B == 0) return NLEM_OK;   // an empty batch may pass NULL buffers
  if (!points_host || !weights_host || !x_out_host)
    return fail(NLEM_ERR_INVALID, "points_host, weights_host and x_out_host must be non-NULL");
  if (n > nlemk::em_capacity(d))
    return fail(NLEM_ERR_UNSUPPORTED, "n = %d, d = %d exceeds the on-chip solver (max n %d for this d)", n,
                d, nlemk::em_capacity(d));
  if ((rc = set_device(ctx))) return rc;
  const size_t pb = (size_t)n * d * sizeof(float);   // one problem's points
  long long Bc = chunk > 0 ? chunk : (long long)std::max<size_t>(1, ((size_t)1 << 30) / pb);
  if (Bc > B) Bc = B;
  // one chunk buffer: points, weights, start points, results; regions 256-byte aligned
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_w = al((size_t)Bc * pb);
  const size_t o_x0 = o_w + al((size_t)Bc * n * 4);
  const size_t o_x = o_x0 + (x0_host ? al((size_t)Bc * d * 4) : 0);
  const size_t o_it = o_x + al((size_t)Bc * d * 4);
  const size_t o_res = o_it + al((size_t)Bc * 4);
  const size_t per = o_res + al((size_t)Bc * 4);
  if (2 * per > ctx->ws_em_bytes) {
    // every call waits for its streams before returning, so the old buffers are idle
    cudaFree(ctx->ws_em);
    ctx->ws_em = nullptr;
    ctx->ws_em_bytes = 0;
    if (cudaMalloc(&ctx->ws_em, 2 * per) != cudaSuccess) {
      cudaGetLastError();
      return fail(NLEM_ERR_OOM, "chunk workspace of %zu bytes could not be allocated", 2 * per);
    }
    ctx->ws_em_bytes = 2 * per;
  }
  if (!ctx->copy_stream) {
    cudaError_t ce = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && ce == cudaSuccess; ++i) {
      ce = cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming);
    }
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
    if (ce != cudaSuccess) return cuda_fail(ce, "copy stream and events of em_solve_batch_host");
  }
  cudaStream_t s = (cudaStream_t)stream, cs = ctx->copy_stream;
  // the copies start after the work already queued on the caller's stream
  cudaError_t e = cudaEventRecord(ctx->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->ev_start, 0);
  const long long nchunks = (B + Bc - 1) / Bc;
  for (long long k = 0; k < nchunks && e == cudaSuccess && rc == NLEM_OK; ++k) {
    const int b = (int)(k & 1);
    const long long off = k * Bc, cnt = std::min(Bc, B - off);
    char* base = ctx->ws_em + b * per;
    float* dp = reinterpret_cast<float*>(base);
    float* dw = reinterpret_cast<float*>(base + o_w);
    float* dx0 = x0_host ? reinterpret_cast<float*>(base + o_x0) : nullptr;
    float* dx = reinterpret_cast<float*>(base + o_x);
    int* dit = reinterpret_cast<int*>(base + o_it);
    float* dres = reinterpret_cast<float*>(base + o_res);
    // buffer b is free once chunk k-2's solve and read-back on the caller's stream are done
    if (k >= 2) e = cudaStreamWaitEvent(cs, ctx->ev_done[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, points_host + off * n * d, (size_t)cnt * pb, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dw, weights_host + off * n, (size_t)cnt * n * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && x0_host)
      e = cudaMemcpyAsync(dx0, x0_host + off * d, (size_t)cnt * d * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied[b], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_copied[b], 0);
    if (e != cudaSuccess) break;
    rc = em_solve_batch(ctx, dp, dw, cnt, n, d, box, rho, iters, dx0, opt, dx, iters_used_host ? dit : nullptr,
                        residual_host ? dres : nullptr, nullptr, nullptr, stream);
    if (rc != NLEM_OK) break;
    e = cudaMemcpyAsync(x_out_host + off * d, dx, (size_t)cnt * d * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && iters_used_host)
      e = cudaMemcpyAsync(iters_used_host + off, dit, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && residual_host)
      e = cudaMemcpyAsync(residual_host + off, dres, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_done[b], s);
  }
  // wait for both streams, on an error too, so that no copy into the workspace is left in flight
  const cudaError_t ec = cudaStreamSynchronize(cs);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (rc != NLEM_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "em_solve_batch_host copies");
  if (ec != cudaSuccess) return cuda_fail(ec, "em_solve_batch_host copy stream");
  if (es != cudaSuccess) return cuda_fail(es, "em_solve_batch_host");
  return NLEM_OK;
}

int nlem_denoise(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                 float rho, int iters, nlem_box box, const nlem_options* opt, float* out, int* iters_used,
                 float* residual, double* obj64, double* kkt64, void* stream) {
  NLEM_TRACE("nlem_denoise");
  int rc = check_common(ctx, box, rho, iters, opt);
  if (rc) return rc;
  if (H < 1 || W < 1) return fail(NLEM_ERR_INVALID, "image must be at least 1x1 (got %dx%d)", H, W);
  if (pitch < W) return fail(NLEM_ERR_INVALID, "pitch %d < W %d", pitch, W);
  if (patch < 1 || (patch % 2) == 0) return fail(NLEM_ERR_INVALID, "patch must be odd and >= 1 (got %d)", patch);
  if (window < 1 || (window % 2) == 0) return fail(NLEM_ERR_INVALID, "window must be odd and >= 1 (got %d)", window);
  int side = H < W ? H : W;
  if (patch > side) return fail(NLEM_ERR_INVALID, "patch %d exceeds the image side %d", patch, side);
  if (!(h > 0.f) || !finite(h)) return fail(NLEM_ERR_INVALID, "h must be finite and > 0 (got %g)", h);
  if (!image || !out) return fail(NLEM_ERR_INVALID, "image and out must be non-NULL");
  if (patch * patch > 128) return fail(NLEM_ERR_UNSUPPORTED, "patch^2 must be <= 128");
  int cap = nlemk::nlem_capacity(patch);
  if (cap == 0) return fail(NLEM_ERR_UNSUPPORTED, "patch %d not compiled (5, 7, 9 are)", patch);
  if (window * window > cap)
    return fail(NLEM_ERR_UNSUPPORTED, "window %d holds %d points; the patch-%d kernels hold %d", window,
                window * window, patch, cap);
  if ((rc = set_device(ctx))) return rc;
  nlemk::NlemLaunch L;
  L.img = image;
  L.H = H;
  L.W = W;
  L.pitch = pitch;
  L.patch = patch;
  L.S = window;
  L.inv_h2 = 1.f / (h * h);
  L.inv_h2_exact = 1.0 / ((double)h * (double)h);
  L.prm = make_params(box, rho, iters, opt, patch * patch);
  L.init_mode = opt ? opt->init : NLEM_INIT_WEIGHTED_MEAN;
  L.out = out;
  L.iters_used = iters_used;
  L.resid = residual;
  const bool chk = opt && opt->fp64_check;
  L.obj64 = chk ? obj64 : nullptr;
  L.kkt64 = chk ? kkt64 : nullptr;
  L.sm_count = ctx->sm_count;
  L.stream = (cudaStream_t)stream;
  L.wtab = nullptr;
  L.pix_list = nullptr;
  L.n_list = nullptr;
  L.max_items = 0;
  L.ex = nlemk::PixelExtra{};
  L.layout = opt ? opt->layout : NLEM_LAYOUT_AUTO;
  L.penalty = opt ? opt->penalty : NLEM_PENALTY_UNIFORM;
  if (L.penalty != NLEM_PENALTY_UNIFORM && (patch != 7 || L.layout == NLEM_LAYOUT_PAIR))
    return fail(NLEM_ERR_UNSUPPORTED, "per-point penalties are compiled for 7x7 patches on the one-pixel layout");
  if (L.prm.solver == NLEM_SOLVER_FAST &&
      (patch != 7 || window * window > nlemk::fast_capacity() || L.layout == NLEM_LAYOUT_PAIR))
    return fail(NLEM_ERR_UNSUPPORTED, "the accelerated solver is compiled for 7x7 patches, windows of at most %d "
                "points, on the one-pixel layout (got patch %d, window %d)", nlemk::fast_capacity(), patch, window);
  if (opt && opt->precision == NLEM_PREC_BF16) {
    // cross terms on the tensor cores into the weight table, then the solver reads it
    const size_t need = (size_t)H * W * (size_t)window * window;
    if (need > ctx->ws_wtab_floats) {
      cudaStreamSynchronize((cudaStream_t)stream);
      cudaFree(ctx->ws_wtab);
      ctx->ws_wtab = nullptr;
      ctx->ws_wtab_floats = 0;
      if (cudaMalloc(&ctx->ws_wtab, need * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NLEM_ERR_OOM, "weight table of %zu floats could not be allocated", need);
      }
      ctx->ws_wtab_floats = need;
    }
    if (!ctx->ws_err) {
      if (cudaMalloc(&ctx->ws_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NLEM_ERR_OOM, "status flag could not be allocated");
      }
      cudaMemset(ctx->ws_err, 0, sizeof(int));
    }
    int we = nlemk::launch_bf16_weights(image, H, W, pitch, patch, window, L.inv_h2, ctx->ws_wtab, ctx->ws_err,
                                        (cudaStream_t)stream);
    if (we == -1) return fail(NLEM_ERR_UNSUPPORTED, "BF16 weights are compiled for patch 5, 7 and 9 with window <= 31");
    if (we != 0) return cuda_fail((cudaError_t)we, "BF16 weight kernel launch");
    L.wtab = ctx->ws_wtab;
  }
  int e = nlemk::launch_nlem_fp32(L);
  if (e == -1 && L.layout == NLEM_LAYOUT_PAIR)
    return fail(NLEM_ERR_UNSUPPORTED, "the pair layout takes EM-ADMM in FP32, patch 7 and window <= 21 (got patch %d, window %d)",
                patch, window);
  if (e == -1) return fail(NLEM_ERR_UNSUPPORTED, "no kernel shape for patch %d, window %d", patch, window);
  if (e != 0) return cuda_fail((cudaError_t)e, "nlem_denoise launch");
  return NLEM_OK;
}

int nlem_denoise_color(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int channels, int patch,
                       int window, float h, float rho, int iters, nlem_box box, const nlem_options* opt, float* out,
                       int* iters_used, float* residual, double* obj64, double* kkt64, void* stream) {
  NLEM_TRACE("nlem_denoise_color");
  int rc = check_common(ctx, box, rho, iters, opt);
  if (rc) return rc;
  if ((rc = admm_only(opt, "nlem_denoise_color"))) return rc;
  if ((rc = uniform_penalty_only(opt, "nlem_denoise_color"))) return rc;
  if (H < 1 || W < 1) return fail(NLEM_ERR_INVALID, "image must be at least 1x1 (got %dx%d)", H, W);
  if (pitch < W) return fail(NLEM_ERR_INVALID, "pitch %d < W %d", pitch, W);
  if (channels < 1) return fail(NLEM_ERR_INVALID, "channels must be >= 1 (got %d)", channels);
  if (patch < 1 || (patch % 2) == 0) return fail(NLEM_ERR_INVALID, "patch must be odd and >= 1 (got %d)", patch);
  if (window < 1 || (window % 2) == 0) return fail(NLEM_ERR_INVALID, "window must be odd and >= 1 (got %d)", window);
  if (patch > (H < W ? H : W)) return fail(NLEM_ERR_INVALID, "patch %d exceeds the image side", patch);
  if (!(h > 0.f) || !finite(h)) return fail(NLEM_ERR_INVALID, "h must be finite and > 0 (got %g)", h);
  if (!image || !out) return fail(NLEM_ERR_INVALID, "image and out must be non-NULL");
  if (opt && opt->precision != NLEM_PREC_FP32)
    return fail(NLEM_ERR_UNSUPPORTED, "multichannel NLEM computes its weights in FP32 only");
  if (opt && opt->layout == NLEM_LAYOUT_PAIR)
    return fail(NLEM_ERR_UNSUPPORTED, "multichannel NLEM runs one pixel per CTA");
  const int cap = nlemk::nlem_color_capacity(channels, patch);
  if (cap == 0) return fail(NLEM_ERR_UNSUPPORTED, "%d channels with patch %d not compiled (3 channels, patch 5 or 7)",
                            channels, patch);
  if (window * window > cap)
    return fail(NLEM_ERR_UNSUPPORTED, "window %d holds %d points; the %d-channel patch-%d kernel holds %d", window,
                window * window, channels, patch, cap);
  if (opt && opt->fp64_check && window * window > nlemk::nlem_color_single_cta_capacity(channels, patch))
    return fail(NLEM_ERR_UNSUPPORTED, "the FP64 check needs the window in one CTA (at most %d points here)",
                nlemk::nlem_color_single_cta_capacity(channels, patch));
  if ((rc = set_device(ctx))) return rc;
  nlemk::NlemColorLaunch L;
  L.img = image;
  L.H = H;
  L.W = W;
  L.pitch = pitch;
  L.cstride = (long long)H * pitch;
  L.channels = channels;
  L.patch = patch;
  L.S = window;
  L.inv_h2 = 1.f / (h * h);
  L.inv_h2_exact = 1.0 / ((double)h * (double)h);
  L.prm = make_params(box, rho, iters, opt, channels * patch * patch);
  L.init_mode = opt ? opt->init : NLEM_INIT_WEIGHTED_MEAN;
  L.out = out;
  L.iters_used = iters_used;
  L.resid = residual;
  const bool chk = opt && opt->fp64_check;
  L.obj64 = chk ? obj64 : nullptr;
  L.kkt64 = chk ? kkt64 : nullptr;
  L.sm_count = ctx->sm_count;
  L.stream = (cudaStream_t)stream;
  const int e = nlemk::launch_nlem_color(L);
  if (e == -1) return fail(NLEM_ERR_UNSUPPORTED, "no kernel shape for %d channels, patch %d, window %d", channels,
                           patch, window);
  if (e != 0) return cuda_fail((cudaError_t)e, "nlem_denoise_color launch");
  return NLEM_OK;
}

int nlem_denoise_host(nlem_ctx* ctx, const float* image_host, int H, int W, int patch, int window, float h,
                      float rho, int iters, nlem_box box, const nlem_options* opt, float* out_host,
                      int* iters_used_host, void* stream) {
  NLEM_TRACE("nlem_denoise_host");
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  if (!image_host || !out_host) return fail(NLEM_ERR_INVALID, "image_host and out_host must be non-NULL");
  if (H < 1 || W < 1) return fail(NLEM_ERR_INVALID, "image must be at least 1x1");
  int rc = set_device(ctx);
  if (rc) return rc;
  size_t npix = (size_t)H * W;
  if (npix > ctx->ws_pixels) {
    cudaFree(ctx->ws_img);
    cudaFree(ctx->ws_out);
    cudaFree(ctx->ws_iters);
    ctx->ws_img = ctx->ws_out = nullptr;
    ctx->ws_iters = nullptr;
    ctx->ws_pixels = 0;
    if (cudaMalloc(&ctx->ws_img, npix * 4) != cudaSuccess || cudaMalloc(&ctx->ws_out, npix * 4) != cudaSuccess ||
        cudaMalloc(&ctx->ws_iters, npix * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(NLEM_ERR_OOM, "workspace of %zu pixels could not be allocated", npix);
    }
    ctx->ws_pixels = npix;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(ctx->ws_img, image_host, npix * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy image to device");
  rc = nlem_denoise(ctx, ctx->ws_img, H, W, W, patch, window, h, rho, iters, box, opt, ctx->ws_out,
                    iters_used_host ? ctx->ws_iters : nullptr, nullptr, nullptr, nullptr, stream);
  if (rc) return rc;
  e = cudaMemcpyAsync(out_host, ctx->ws_out, npix * 4, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy result to host");
  if (iters_used_host) {
    e = cudaMemcpyAsync(iters_used_host, ctx->ws_iters, npix * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy iteration counts to host");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "nlem_denoise_host");
  return NLEM_OK;
}

int nlem_bf16_weights(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                      float* wtab, void* stream) {
  NLEM_TRACE("nlem_bf16_weights");
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  if (!image || !wtab) return fail(NLEM_ERR_INVALID, "image and wtab must be non-NULL");
  if (H < 1 || W < 1 || pitch < W) return fail(NLEM_ERR_INVALID, "bad image size or pitch");
  if (patch < 1 || patch % 2 == 0 || window < 1 || window % 2 == 0)
    return fail(NLEM_ERR_INVALID, "patch and window must be odd and >= 1");
  if (patch > std::min(H, W)) return fail(NLEM_ERR_INVALID, "patch exceeds the image side");
  if (!(h > 0.f) || !std::isfinite(h)) return fail(NLEM_ERR_INVALID, "h must be finite and > 0");
  int rc = set_device(ctx);
  if (rc) return rc;
  if (!ctx->ws_err) {
    if (cudaMalloc(&ctx->ws_err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(NLEM_ERR_OOM, "status flag could not be allocated");
    }
    cudaMemset(ctx->ws_err, 0, sizeof(int));
  }
  int we = nlemk::launch_bf16_weights(image, H, W, pitch, patch, window, 1.f / (h * h), wtab, ctx->ws_err,
                                      (cudaStream_t)stream);
  if (we == -1) return fail(NLEM_ERR_UNSUPPORTED, "BF16 weights are compiled for patch 5, 7 and 9 with window <= 31");
  if (we != 0) return cuda_fail((cudaError_t)we, "BF16 weight kernel launch");
  return NLEM_OK;
}

int nlem_device_status(nlem_ctx* ctx) {
  NLEM_TRACE("nlem_device_status");
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  int rc = set_device(ctx);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
  if (!ctx->ws_err) return NLEM_OK;
  int flag = 0;
  e = cudaMemcpy(&flag, ctx->ws_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status flag");
  if (flag) {
    cudaMemset(ctx->ws_err, 0, sizeof(int));
    return fail(NLEM_ERR_TIMEOUT, "a bounded tensor-core wait ran out; affected weights were not written");
  }
  return NLEM_OK;
}

int nlem_selftest_timeout(nlem_ctx* ctx) {
  NLEM_TRACE("nlem_selftest_timeout");
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  int rc = set_device(ctx);
  if (rc) return rc;
  rc = nlem_device_status(ctx);   // start from a clean flag
  if (rc) return rc;
  if (!ctx->ws_err) {
    if (cudaMalloc(&ctx->ws_err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(NLEM_ERR_OOM, "status flag could not be allocated");
    }
    cudaMemset(ctx->ws_err, 0, sizeof(int));
  }
  // a 16 x 16 zero image, 5 x 5 patches, 5 x 5 window: two CTAs, each waiting 256 polls for a
  // tensor-core commit that is never issued
  const int n = 16;
  float* img = nullptr;
  float* tab = nullptr;
  if (cudaMalloc(&img, n * n * sizeof(float)) != cudaSuccess || cudaMalloc(&tab, n * n * 25 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(img);
    return fail(NLEM_ERR_OOM, "self-test buffers could not be allocated");
  }
  cudaMemset(img, 0, n * n * sizeof(float));
  int we = nlemk::launch_bf16_weights(img, n, n, n, 5, 5, 1.f, tab, ctx->ws_err, (cudaStream_t)0, 256u, 0);
  rc = we ? cuda_fail((cudaError_t)we, "self-test launch") : nlem_device_status(ctx);
  cudaFree(img);
  cudaFree(tab);
  return rc;
}

int nlem_fp32_peak(nlem_ctx* ctx, double* tflops, int* sm_count) {
  NLEM_TRACE("nlem_fp32_peak");
  if (!ctx || !tflops) return fail(NLEM_ERR_INVALID, "ctx and tflops must be non-NULL");
  int rc = set_device(ctx);
  if (rc) return rc;
  int e = nlemk::measure_fp32_peak(ctx->sm_count, tflops);
  if (e != 0) return cuda_fail((cudaError_t)e, "fp32 peak probe");
  if (sm_count) *sm_count = ctx->sm_count;
  return NLEM_OK;
}

}  // extern "C"

namespace {

// Autotuner: time every launch shape on a strided sample of the batch (items 0, s, 2s, ...,
// about 16k pixels) and keep the fastest.  Keyed by the workload class, not by the images.
int autotune_batch(nlem_ctx* ctx, nlemk::BatchLaunch L, const std::string& key, cudaStream_t stream,
                   nlemk::BatchConfig* best) {
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) {
    *best = it->second;
    return NLEM_OK;
  }
  const long long sample = 16384;
  L.stride = std::max<long long>(1, L.total / sample);
  static const int fetches[] = {1, 4, 16};
  static const int ctas[] = {2, 1};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  nlemk::BatchConfig winner{0, 1, 2};
  bool warmed = false;
  for (int v = 0; v < nlemk::kBatchVariants; ++v) {
    for (int f : fetches) {
      for (int c : ctas) {
        if (L.prm.solver == NLEM_SOLVER_FAST && c != 1) continue;   // the accelerated shapes fill an SM
        L.cfg = nlemk::BatchConfig{v, f, c};
        for (int rep = warmed ? 0 : -1; rep < 1; ++rep) {   // one untimed warm-up run at first
          cudaMemsetAsync(L.queue, 0, sizeof(unsigned long long), stream);
          cudaEventRecord(e0, stream);
          int rc = nlemk::launch_batch(L);
          cudaEventRecord(e1, stream);
          if (rc != 0) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail((cudaError_t)rc, "autotune launch");
          }
          cudaError_t e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "autotune run");
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep == 0 && ms < best_ms) {
            best_ms = ms;
            winner = L.cfg;
          }
          warmed = true;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune[key] = winner;
  *best = winner;
  return NLEM_OK;
}

}  // namespace

extern "C" {

int nlem_denoise_batch(nlem_ctx* ctx, const nlem_image_desc* images, int count, float rho, int iters, nlem_box box,
                       const nlem_options* opt, void* stream) {
  NLEM_TRACE("nlem_denoise_batch");
  int rc = check_common(ctx, box, rho, iters, opt);
  if (rc) return rc;
  if ((rc = no_irls(opt, "nlem_denoise_batch"))) return rc;
  if ((rc = uniform_penalty_only(opt, "nlem_denoise_batch"))) return rc;
  if (count < 0) return fail(NLEM_ERR_INVALID, "count must be >= 0");
  if (count == 0) return NLEM_OK;
  if (!images) return fail(NLEM_ERR_INVALID, "images is NULL");
  if (opt && opt->precision != NLEM_PREC_FP32)
    return fail(NLEM_ERR_UNSUPPORTED, "the batched kernel computes weights in FP32 only");
  std::vector<nlemk::BatchImage> imgs((size_t)count);
  long long total = 0;
  int maxS = 0, mask = 0;
  for (int i = 0; i < count; ++i) {
    const nlem_image_desc& d = images[i];
    if (!d.image || !d.out) return fail(NLEM_ERR_INVALID, "image %d: image and out must be non-NULL", i);
    if (d.H < 1 || d.W < 1 || d.pitch < d.W) return fail(NLEM_ERR_INVALID, "image %d: bad size %dx%d pitch %d", i, d.H, d.W, d.pitch);
    if (d.patch < 1 || d.patch % 2 == 0 || d.window < 1 || d.window % 2 == 0)
      return fail(NLEM_ERR_INVALID, "image %d: patch and window must be odd and >= 1", i);
    if (d.patch > std::min(d.H, d.W)) return fail(NLEM_ERR_INVALID, "image %d: patch exceeds the image side", i);
    if (!(d.h > 0.f) || !std::isfinite(d.h)) return fail(NLEM_ERR_INVALID, "image %d: h must be finite and > 0", i);
    if (d.patch != 5 && d.patch != 7)
      return fail(NLEM_ERR_UNSUPPORTED, "image %d: the batched kernel handles patch 5 and 7 (got %d)", i, d.patch);
    if (d.window * d.window > std::min(nlemk::batch_max_points(d.patch, 0), nlemk::batch_max_points(d.patch, 1)) ||
        !nlemk::batch_tile_fits(d.patch, d.window))
      return fail(NLEM_ERR_UNSUPPORTED, "image %d: window %d too large for the batched kernel", i, d.window);
    nlemk::BatchImage& b = imgs[(size_t)i];
    b.img = d.image;
    b.out = d.out;
    b.iters = d.iters_used;
    b.resid = d.residual;
    b.H = d.H;
    b.W = d.W;
    b.pitch = d.pitch;
    b.patch = d.patch;
    b.S = d.window;
    b.inv_h2 = 1.f / (d.h * d.h);
    b.ih2 = 1.0 / ((double)d.h * (double)d.h);
    b.pix_begin = total;
    total += (long long)d.H * d.W;
    maxS = std::max(maxS, d.window);
    mask |= d.patch == 5 ? 1 : 2;
  }
  if ((rc = set_device(ctx))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  nlemk::SolveParams prm = make_params(box, rho, iters, opt, 0);
  const int init_mode = opt ? opt->init : NLEM_INIT_WEIGHTED_MEAN;

  const bool same = ctx->have_plan && ctx->plan.imgs.size() == imgs.size() &&
                    std::memcmp(ctx->plan.imgs.data(), imgs.data(), imgs.size() * sizeof(nlemk::BatchImage)) == 0 &&
                    std::memcmp(&ctx->plan.prm, &prm, sizeof(prm)) == 0 && ctx->plan.init_mode == init_mode;
  if (!same) {
    // drop the old plan, grow the workspace, upload the descriptors
    if (ctx->have_plan && ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
    ctx->have_plan = false;
    if (count > ctx->ws_batch_cap) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->ws_batch);
      ctx->ws_batch = nullptr;
      ctx->ws_batch_cap = 0;
      if (cudaMalloc(&ctx->ws_batch, sizeof(nlemk::BatchImage) * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        return fail(NLEM_ERR_OOM, "batch workspace for %d images could not be allocated", count);
      }
      ctx->ws_batch_cap = count;
    }
    if (!ctx->ws_queue) {
      if (cudaMalloc(&ctx->ws_queue, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NLEM_ERR_OOM, "work-queue counter could not be allocated");
      }
    }
    if (!ctx->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    cudaError_t e = cudaMemcpyAsync(ctx->ws_batch, imgs.data(), sizeof(nlemk::BatchImage) * (size_t)count,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload batch descriptors");
    nlemk::BatchLaunch L{};
    L.imgs = ctx->ws_batch;
    L.count = count;
    L.total = total;
    L.stride = 1;
    L.queue = ctx->ws_queue;
    L.prm = prm;
    L.init_mode = init_mode;
    L.sm_count = ctx->sm_count;
    L.stream = s;
    char key[160];
    std::snprintf(key, sizeof(key), "sm%d/patches%d/S%d/tol%d/it%d/init%d/solver%d", ctx->sm_count, mask, maxS,
                  prm.tol > 0.f ? 1 : 0, iters, init_mode, prm.solver);
    nlemk::BatchConfig cfg{};
    if (ctx->forced.variant >= 0) {
      cfg = ctx->forced;
    } else {
      rc = autotune_batch(ctx, L, key, s, &cfg);
      if (rc) return rc;
    }
    // capture queue reset + launch once on the private stream, after the upload completes
    L.cfg = cfg;
    L.stride = 1;
    L.stream = ctx->cap_stream;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch set-up");
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin graph capture");
    cudaMemsetAsync(ctx->ws_queue, 0, sizeof(unsigned long long), ctx->cap_stream);
    int lrc = nlemk::launch_batch(L);
    e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (lrc != 0) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail((cudaError_t)lrc, "capture batch launch");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end graph capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate batch graph");
    ctx->plan.imgs = imgs;
    ctx->plan.prm = prm;
    ctx->plan.init_mode = init_mode;
    ctx->plan.cfg = cfg;
    ctx->plan.total = total;
    ctx->plan.exec = exec;
    ctx->have_plan = true;
    char desc[256];
    std::snprintf(desc, sizeof(desc), "%s; fetch=%d items; %d CTA/SM; %lld items; key %s",
                  nlemk::batch_variant_name(cfg.variant, prm.solver), cfg.fetch,
                  prm.solver == NLEM_SOLVER_FAST ? 1 : cfg.ctas_per_sm, total, key);
    ctx->last_cfg = desc;
  }
  cudaError_t e = cudaGraphLaunch(ctx->plan.exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch batch graph");
  return NLEM_OK;
}

int nlem_batch_force_config(nlem_ctx* ctx, int variant, int fetch, int ctas_per_sm) {
  if (!ctx) return fail(NLEM_ERR_INVALID, "ctx is NULL");
  if (variant < 0) {
    ctx->forced = nlemk::BatchConfig{-1, 0, 0};
  } else {
    if (variant >= nlemk::kBatchVariants) return fail(NLEM_ERR_INVALID, "variant must be < %d", nlemk::kBatchVariants);
    if (fetch < 1 || ctas_per_sm < 1 || ctas_per_sm > 2)
      return fail(NLEM_ERR_INVALID, "fetch >= 1 and 1 <= ctas_per_sm <= 2 are required");
    ctx->forced = nlemk::BatchConfig{variant, fetch, ctas_per_sm};
  }
  // the next call captures a new graph with this shape
  if (ctx->have_plan && ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
  ctx->have_plan = false;
  return NLEM_OK;
}

int nlem_batch_config(nlem_ctx* ctx, char* buf, int len) {
  if (!ctx || !buf || len < 1) return fail(NLEM_ERR_INVALID, "ctx and buf must be non-NULL, len >= 1");
  if (!ctx->have_plan) {
    buf[0] = 0;
    return fail(NLEM_ERR_INVALID, "no batch has run on this context");
  }
  std::snprintf(buf, (size_t)len, "%s", ctx->last_cfg.c_str());
  return NLEM_OK;
}

}  // extern "C"
