// C ABI of the learned warm start and of the extended NLEM entry point (pixel lists,
// per-pixel start points and penalties, full solution patches, features).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/nlem.h"
#include "ctx.h"
#include "kernels.h"
#include "trace.h"
#include "warmstart.h"

struct nlem_warmstart {
  nlem_ctx* ctx = nullptr;
  nlemk::WsModel m;
  nlemk::WsScratch sc;
  // minibatch workspace of nlem_ws_train: sample order, gathered rows, per-step losses
  int* perm = nullptr;
  float* fb = nullptr;
  float* tb = nullptr;
  float* losses = nullptr;
  size_t cap_perm = 0, cap_fb = 0, cap_tb = 0, cap_losses = 0;
};

namespace {

int wfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  nlemk::set_last_error(buf);
  return code;
}

int wcuda(cudaError_t e, const char* what) { return wfail(NLEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e)); }

template <class T>
int grow(T** p, size_t* cap_elems, size_t need, const char* what) {
  if (need <= *cap_elems && *p) return NLEM_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap_elems = 0;
  if (cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return wfail(NLEM_ERR_OOM, "%s: %zu elements could not be allocated", what, need);
  }
  *cap_elems = need;
  return NLEM_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014) for the seeded weight initialisation.
uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double normal(uint64_t& st) {
  const double u1 = ((double)(splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// shared validation of the NLEM geometry arguments
int check_nlem_args(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h) {
  if (!ctx) return wfail(NLEM_ERR_INVALID, "ctx is NULL");
  if (!image) return wfail(NLEM_ERR_INVALID, "image is NULL");
  if (H < 1 || W < 1 || pitch < W) return wfail(NLEM_ERR_INVALID, "bad image size %dx%d or pitch %d", H, W, pitch);
  if (patch < 1 || patch % 2 == 0 || window < 1 || window % 2 == 0)
    return wfail(NLEM_ERR_INVALID, "patch and window must be odd and >= 1");
  if (patch > (H < W ? H : W)) return wfail(NLEM_ERR_INVALID, "patch exceeds the image side");
  if (!(h > 0.f) || !std::isfinite(h)) return wfail(NLEM_ERR_INVALID, "h must be finite and > 0");
  if (nlemk::nlem_capacity(patch) == 0) return wfail(NLEM_ERR_UNSUPPORTED, "patch %d not compiled", patch);
  if (window * window > nlemk::nlem_capacity(patch)) return wfail(NLEM_ERR_UNSUPPORTED, "window %d too large", window);
  return NLEM_OK;
}

nlemk::NlemLaunch base_launch(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window,
                              float h, float rho, int iters, nlem_box box, const nlem_options* opt, cudaStream_t s) {
  nlemk::NlemLaunch L{};
  L.img = image;
  L.H = H;
  L.W = W;
  L.pitch = pitch;
  L.patch = patch;
  L.S = window;
  L.inv_h2 = 1.f / (h * h);
  L.inv_h2_exact = 1.0 / ((double)h * (double)h);
  L.prm.lo = box.lo;
  L.prm.hi = box.hi;
  L.prm.mu = rho;
  L.prm.inv_mu = 1.f / rho;
  L.prm.iters = iters;
  L.prm.tol = opt ? opt->tol : 0.f;
  L.prm.check_every = opt ? opt->check_every : 1;
  L.prm.d = patch * patch;
  L.prm.solver = opt ? opt->solver : NLEM_SOLVER_ADMM;
  L.prm.restart_every = opt ? opt->restart_every : 0;
  L.init_mode = opt ? opt->init : NLEM_INIT_WEIGHTED_MEAN;
  L.penalty = opt ? opt->penalty : NLEM_PENALTY_UNIFORM;
  L.sm_count = ctx->sm_count;
  L.stream = s;
  return L;
}

int run_launch(const nlemk::NlemLaunch& L, const char* what) {
  const int e = nlemk::launch_nlem_fp32(L);
  if (e == -1) return wfail(NLEM_ERR_UNSUPPORTED, "%s: no kernel shape (or shared memory) for patch %d, window %d", what,
                            L.patch, L.S);
  if (e != 0) return wcuda((cudaError_t)e, what);
  return NLEM_OK;
}

int ensure_counts(nlem_ctx* ctx) {
  if (ctx->ws_count) return NLEM_OK;
  if (cudaMalloc(&ctx->ws_count, 2 * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return wfail(NLEM_ERR_OOM, "count buffer could not be allocated");
  }
  return NLEM_OK;
}

}  // namespace

extern "C" {

long long nlem_ws_num_params(int d) { return d >= 1 ? nlemk::ws_num_params(d) : -1; }

int nlem_ws_create(nlem_ctx* ctx, int d, float nref, unsigned long long seed, nlem_warmstart** out) {
  if (!ctx || !out) return wfail(NLEM_ERR_INVALID, "ctx and out must be non-NULL");
  if (d < 1 || d > 81) return wfail(NLEM_ERR_INVALID, "d must be in [1, 81]");
  if (!(nref > 1.f)) return wfail(NLEM_ERR_INVALID, "nref must be > 1");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  nlem_warmstart* ws = new (std::nothrow) nlem_warmstart();
  if (!ws) return wfail(NLEM_ERR_OOM, "out of host memory");
  ws->ctx = ctx;
  ws->m.d = d;
  ws->m.nref = nref;
  const long long P = nlemk::ws_num_params(d);
  bool ok = cudaMalloc(&ws->m.p32, P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&ws->m.w16, P * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&ws->m.adam_m, P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&ws->m.adam_v, P * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    nlem_ws_destroy(ws);
    return wfail(NLEM_ERR_OOM, "warm-start parameters could not be allocated");
  }
  // He-normal weights, zero biases; the output layer starts small (x0 ~ weighted mean) and the
  // log-penalty output starts at log(0.01)
  const int F = 2 * d + 2, O = d + 1, Hd = nlemk::kWsHidden;
  std::vector<float> h((size_t)P, 0.f);
  uint64_t st = seed;
  size_t k = 0;
  for (int i = 0; i < Hd * F; ++i) h[k++] = (float)(normal(st) * std::sqrt(2.0 / F));
  k += Hd;
  for (int i = 0; i < Hd * Hd; ++i) h[k++] = (float)(normal(st) * std::sqrt(2.0 / Hd));
  k += Hd;
  for (int i = 0; i < O * Hd; ++i) h[k++] = (float)(normal(st) * 0.1 * std::sqrt(2.0 / Hd));
  h[k + d] = (float)std::log(0.01);
  int rc = nlem_ws_set_params(ws, h.data());
  if (rc) {
    nlem_ws_destroy(ws);
    return rc;
  }
  *out = ws;
  return NLEM_OK;
}

int nlem_ws_destroy(nlem_warmstart* ws) {
  if (!ws) return NLEM_OK;
  cudaFree(ws->m.p32);
  cudaFree(ws->m.w16);
  cudaFree(ws->m.adam_m);
  cudaFree(ws->m.adam_v);
  cudaFree(ws->sc.y);
  cudaFree(ws->sc.xs);
  cudaFree(ws->sc.a1);
  cudaFree(ws->sc.a2);
  cudaFree(ws->sc.dy);
  cudaFree(ws->sc.da1);
  cudaFree(ws->sc.da2);
  cudaFree(ws->sc.grad);
  cudaFree(ws->perm);
  cudaFree(ws->fb);
  cudaFree(ws->tb);
  cudaFree(ws->losses);
  delete ws;
  return NLEM_OK;
}

int nlem_ws_get_params(nlem_warmstart* ws, float* host_params) {
  if (!ws || !host_params) return wfail(NLEM_ERR_INVALID, "ws and host_params must be non-NULL");
  cudaError_t e = cudaMemcpy(host_params, ws->m.p32, nlemk::ws_num_params(ws->m.d) * sizeof(float),
                             cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? NLEM_OK : wcuda(e, "read parameters");
}

int nlem_ws_set_params(nlem_warmstart* ws, const float* host_params) {
  if (!ws || !host_params) return wfail(NLEM_ERR_INVALID, "ws and host_params must be non-NULL");
  const long long P = nlemk::ws_num_params(ws->m.d);
  cudaError_t e = cudaMemcpy(ws->m.p32, host_params, P * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return wcuda(e, "write parameters");
  cudaMemset(ws->m.adam_m, 0, P * sizeof(float));
  cudaMemset(ws->m.adam_v, 0, P * sizeof(float));
  ws->m.step = 0;
  int rc = nlemk::ws_sync_half(ws->m, ws->ctx->sm_count, nullptr);
  if (rc) return wcuda((cudaError_t)rc, "FP16 copy");
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? NLEM_OK : wcuda(e, "set parameters");
}

int nlem_ws_save(nlem_warmstart* ws, const char* path) {
  if (!ws || !path) return wfail(NLEM_ERR_INVALID, "ws and path must be non-NULL");
  const long long P = nlemk::ws_num_params(ws->m.d);
  std::vector<float> buf((size_t)(3 * P));
  cudaMemcpy(buf.data(), ws->m.p32, P * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(buf.data() + P, ws->m.adam_m, P * sizeof(float), cudaMemcpyDeviceToHost);
  cudaError_t e = cudaMemcpy(buf.data() + 2 * P, ws->m.adam_v, P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return wcuda(e, "read model");
  FILE* f = std::fopen(path, "wb");
  if (!f) return wfail(NLEM_ERR_INVALID, "cannot open %s for writing", path);
  const char magic[8] = {'N', 'L', 'E', 'M', 'W', 'S', '0', '1'};
  const int32_t hdr[2] = {ws->m.d, nlemk::kWsHidden};
  const int64_t step = ws->m.step;
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(&ws->m.nref, sizeof(float), 1, f) == 1 && std::fwrite(&step, sizeof(step), 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? NLEM_OK : wfail(NLEM_ERR_INVALID, "write to %s failed", path);
}

int nlem_ws_load(nlem_warmstart* ws, const char* path) {
  if (!ws || !path) return wfail(NLEM_ERR_INVALID, "ws and path must be non-NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return wfail(NLEM_ERR_INVALID, "cannot open %s", path);
  char magic[8];
  int32_t hdr[2];
  float nref;
  int64_t step;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "NLEMWS01", 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&nref, sizeof(float), 1, f) == 1 &&
            std::fread(&step, sizeof(step), 1, f) == 1;
  if (!ok || hdr[0] != ws->m.d || hdr[1] != nlemk::kWsHidden) {
    std::fclose(f);
    return wfail(NLEM_ERR_INVALID, "%s is not a warm-start model for d = %d", path, ws->m.d);
  }
  const long long P = nlemk::ws_num_params(ws->m.d);
  std::vector<float> buf((size_t)(3 * P));
  ok = std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return wfail(NLEM_ERR_INVALID, "%s is truncated", path);
  int rc = nlem_ws_set_params(ws, buf.data());
  if (rc) return rc;
  cudaMemcpy(ws->m.adam_m, buf.data() + P, P * sizeof(float), cudaMemcpyHostToDevice);
  cudaError_t e = cudaMemcpy(ws->m.adam_v, buf.data() + 2 * P, P * sizeof(float), cudaMemcpyHostToDevice);
  ws->m.step = step;
  ws->m.nref = nref;
  return e == cudaSuccess ? NLEM_OK : wcuda(e, "load model");
}

int nlem_ws_forward(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, long long B, float* y, void* stream) {
  NLEM_TRACE("nlem_ws_forward");
  if (!ctx || !ws || !feats || !y || B < 0) return wfail(NLEM_ERR_INVALID, "bad arguments");
  cudaSetDevice(ctx->device);
  const int rc = nlemk::ws_forward(ws->m, feats, B, y, nullptr, nullptr, nullptr, ctx->sm_count, (cudaStream_t)stream);
  return rc ? wcuda((cudaError_t)rc, "warm-start forward") : NLEM_OK;
}

int nlem_ws_loss_grad(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long B,
                      float* loss, float* grad, void* stream) {
  NLEM_TRACE("nlem_ws_loss_grad");
  if (!ctx || !ws || !feats || !targets || B < 1) return wfail(NLEM_ERR_INVALID, "bad arguments");
  cudaSetDevice(ctx->device);
  nlemk::WsScratch& sc = ws->sc;
  if (B > sc.cap) {
    cudaStreamSynchronize((cudaStream_t)stream);
    float** bufs[] = {&sc.y, &sc.xs, &sc.a1, &sc.a2, &sc.dy, &sc.da1, &sc.da2};
    for (float** b : bufs) {
      cudaFree(*b);
      *b = nullptr;
    }
    const int d = ws->m.d, F = 2 * d + 2, O = d + 1, Hd = nlemk::kWsHidden;
    const size_t sizes[] = {(size_t)O, (size_t)F, (size_t)Hd, (size_t)Hd, (size_t)O, (size_t)Hd, (size_t)Hd};
    for (int i = 0; i < 7; ++i) {
      if (cudaMalloc(bufs[i], (size_t)B * sizes[i] * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        sc.cap = 0;
        return wfail(NLEM_ERR_OOM, "training scratch for %lld samples could not be allocated", B);
      }
    }
    sc.cap = B;
  }
  if (!sc.grad) {
    if (cudaMalloc(&sc.grad, nlemk::ws_num_params(ws->m.d) * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return wfail(NLEM_ERR_OOM, "gradient buffer could not be allocated");
    }
  }
  const int rc = nlemk::ws_loss_grad(ws->m, sc, feats, targets, B, loss, grad ? grad : sc.grad, ctx->sm_count,
                                     (cudaStream_t)stream);
  return rc ? wcuda((cudaError_t)rc, "warm-start loss/gradient") : NLEM_OK;
}

int nlem_ws_train_step(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long B,
                       float lr, float* loss, void* stream) {
  NLEM_TRACE("nlem_ws_train_step");
  int rc = nlem_ws_loss_grad(ctx, ws, feats, targets, B, loss, nullptr, stream);
  if (rc) return rc;
  rc = nlemk::ws_adam(ws->m, ws->sc.grad, lr, ctx->sm_count, (cudaStream_t)stream);
  return rc ? wcuda((cudaError_t)rc, "Adam step") : NLEM_OK;
}

// SplitMix64 output function (Steele, Lea & Flood 2014), used in counter mode for the epoch
// orders of nlem_ws_train.
static unsigned long long ws_mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int nlem_ws_train(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long N,
                  int epochs, int batch, float lr, unsigned long long seed, float* epoch_loss, void* stream) {
  NLEM_TRACE("nlem_ws_train");
  if (!ctx || !ws || !feats || !targets || N < 1 || epochs < 0 || batch < 1 || !(lr > 0.f) || !std::isfinite(lr))
    return wfail(NLEM_ERR_INVALID, "bad arguments");
  if (N > 2147483647LL) return wfail(NLEM_ERR_UNSUPPORTED, "at most 2^31 - 1 samples");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ws->m.d, F = 2 * d + 2, O = d + 1;
  const long long B = batch < N ? batch : N;
  const long long steps = N / B;   // full minibatches; the remainder joins a later epoch's order
  int rc;
  if (N > (long long)ws->cap_perm || B * F > (long long)ws->cap_fb || B * O > (long long)ws->cap_tb ||
      steps > (long long)ws->cap_losses)
    cudaStreamSynchronize(s);
  if ((rc = grow(&ws->perm, &ws->cap_perm, (size_t)N, "sample order"))) return rc;
  if ((rc = grow(&ws->fb, &ws->cap_fb, (size_t)(B * F), "minibatch features"))) return rc;
  if ((rc = grow(&ws->tb, &ws->cap_tb, (size_t)(B * O), "minibatch targets"))) return rc;
  if ((rc = grow(&ws->losses, &ws->cap_losses, (size_t)steps, "losses"))) return rc;
  std::vector<int> order((size_t)N);
  std::vector<float> lh((size_t)steps);
  for (int ep = 0; ep < epochs; ++ep) {
    // Fisher-Yates shuffle; draw i of epoch ep is mix64(key_ep + (i + 1) * golden)
    for (long long i = 0; i < N; ++i) order[(size_t)i] = (int)i;
    const unsigned long long key = ws_mix64(seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(ep + 1)));
    for (long long i = N - 1; i > 0; --i) {
      const unsigned long long r = ws_mix64(key + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull);
      const long long j = (long long)(r % (unsigned long long)(i + 1));
      std::swap(order[(size_t)i], order[(size_t)j]);
    }
    cudaError_t e = cudaMemcpyAsync(ws->perm, order.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host order is rewritten next epoch
    if (e != cudaSuccess) return wcuda(e, "sample order upload");
    for (long long k = 0; k < steps; ++k) {
      int ge = nlemk::ws_gather_rows(feats, F, ws->perm + k * B, B, ws->fb, ctx->sm_count, s);
      if (!ge) ge = nlemk::ws_gather_rows(targets, O, ws->perm + k * B, B, ws->tb, ctx->sm_count, s);
      if (ge) return wcuda((cudaError_t)ge, "minibatch gather");
      if ((rc = nlem_ws_train_step(ctx, ws, ws->fb, ws->tb, B, lr, ws->losses + k, stream))) return rc;
    }
    if (epoch_loss) {
      e = cudaMemcpyAsync(lh.data(), ws->losses, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return wcuda(e, "read losses");
      double acc = 0.0;
      for (long long k = 0; k < steps; ++k) acc += lh[(size_t)k];
      epoch_loss[ep] = (float)(acc / (double)steps);
    }
  }
  return NLEM_OK;
}

int nlem_ws_predict(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, long long B, nlem_box box, float* y,
                    float* x0, float* rho, void* stream) {
  NLEM_TRACE("nlem_ws_predict");
  if (!ctx || !ws || !feats || !y || !x0 || !rho || B < 0) return wfail(NLEM_ERR_INVALID, "bad arguments");
  cudaSetDevice(ctx->device);
  int rc = nlemk::ws_forward(ws->m, feats, B, y, nullptr, nullptr, nullptr, ctx->sm_count, (cudaStream_t)stream);
  if (!rc) rc = nlemk::ws_apply(feats, y, B, ws->m.d, box.lo, box.hi, x0, rho, ctx->sm_count, (cudaStream_t)stream);
  return rc ? wcuda((cudaError_t)rc, "warm-start predict") : NLEM_OK;
}

int nlem_features(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                  const int* pixels, long long npix, float* feats, void* stream) {
  NLEM_TRACE("nlem_features");
  int rc = check_nlem_args(ctx, image, H, W, pitch, patch, window, h);
  if (rc) return rc;
  if (!feats) return wfail(NLEM_ERR_INVALID, "feats is NULL");
  if (pixels && npix < 0) return wfail(NLEM_ERR_INVALID, "npix must be >= 0");
  if ((window + patch - 1) * (window + patch - 1) > 1024)
    return wfail(NLEM_ERR_UNSUPPORTED, "features need (window + patch - 1)^2 <= 1024");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = ensure_counts(ctx))) return rc;
  const long long* n_list = nullptr;
  if (pixels) {
    long long n = npix;
    cudaMemcpyAsync(ctx->ws_count + 1, &n, sizeof(long long), cudaMemcpyHostToDevice, s);
    n_list = ctx->ws_count + 1;
  }
  const int e = nlemk::launch_features(image, H, W, pitch, patch, window, 1.f / (h * h), pixels, n_list, npix, feats,
                                       ctx->sm_count, s);
  if (e == -1) return wfail(NLEM_ERR_UNSUPPORTED, "features: patch %d not compiled (5, 7, 9 are)", patch);
  if (e != 0) return wfail(NLEM_ERR_CUDA, "features launch: %s", cudaGetErrorString((cudaError_t)e));
  return NLEM_OK;
}

int nlem_denoise_ex(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                    float rho, int iters, nlem_box box, const nlem_options* opt, const int* pixels, long long npix,
                    const float* x0, const float* rho_pix, float* out, int* iters_used, float* residual,
                    float* z_out, void* stream) {
  NLEM_TRACE("nlem_denoise_ex");
  int rc = check_nlem_args(ctx, image, H, W, pitch, patch, window, h);
  if (rc) return rc;
  if (!out) return wfail(NLEM_ERR_INVALID, "out is NULL");
  if (!(rho > 0.f) || !std::isfinite(rho) || iters < 0 || !(box.lo <= box.hi))
    return wfail(NLEM_ERR_INVALID, "rho > 0, iters >= 0 and lo <= hi are required");
  if (opt && (opt->check_every < 1 || opt->precision != NLEM_PREC_FP32 ||
              (opt->solver != NLEM_SOLVER_ADMM && opt->solver != NLEM_SOLVER_FAST) || opt->restart_every < 0))
    return wfail(NLEM_ERR_INVALID, "options: check_every >= 1, FP32 precision, the EM-ADMM solver (plain or "
                 "accelerated) and restart_every >= 0");
  if (pixels && npix < 0) return wfail(NLEM_ERR_INVALID, "npix must be >= 0");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  nlemk::NlemLaunch L = base_launch(ctx, image, H, W, pitch, patch, window, h, rho, iters, box, opt, s);
  L.out = out;
  L.iters_used = iters_used;
  L.resid = residual;
  if ((rc = ensure_counts(ctx))) return rc;
  if (pixels) {
    if (npix == 0) return NLEM_OK;
    // the solver reads a copy of the list without the entries outside the image (their count on
    // the device), so its item loop needs no bounds test
    if ((rc = grow(&ctx->ws_ulist, &ctx->ws_ulist_cap, (size_t)npix, "pixel list"))) return rc;
    const int ce = nlemk::ws_compact_list(pixels, npix, (long long)H * W, ctx->ws_ulist, ctx->ws_count + 1,
                                          ctx->sm_count, s);
    if (ce) return wfail(NLEM_ERR_CUDA, "pixel list: %s", cudaGetErrorString((cudaError_t)ce));
    L.pix_list = ctx->ws_ulist;
    L.n_list = ctx->ws_count + 1;
    L.max_items = npix;
  }
  L.ex.x0 = x0;
  L.ex.rho = rho_pix;
  L.ex.z_out = z_out;
  return run_launch(L, "nlem_denoise_ex");
}

int nlem_ws_labels(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                   nlem_box box, const int* pixels, long long n, const float* rho_grid, int n_rho, float tol,
                   int check_every, int cap, float tight_tol, int tight_cap, const float* feats, float* targets,
                   long long* rho_counts, void* stream) {
  NLEM_TRACE("nlem_ws_labels");
  int rc = check_nlem_args(ctx, image, H, W, pitch, patch, window, h);
  if (rc) return rc;
  if (n < 0) return wfail(NLEM_ERR_INVALID, "n must be >= 0");
  if (n > 0 && (!pixels || !feats || !targets)) return wfail(NLEM_ERR_INVALID, "pixels, feats and targets must be non-NULL");
  if (!rho_grid || n_rho < 1 || n_rho > 64) return wfail(NLEM_ERR_INVALID, "rho_grid must hold 1 to 64 penalties");
  for (int j = 0; j < n_rho; ++j)
    if (!(rho_grid[j] > 0.f) || !std::isfinite(rho_grid[j])) return wfail(NLEM_ERR_INVALID, "penalties must be finite and > 0");
  if (!(tol > 0.f) || !(tight_tol > 0.f) || !std::isfinite(tol) || !std::isfinite(tight_tol))
    return wfail(NLEM_ERR_INVALID, "tol and tight_tol must be finite and > 0");
  if (check_every < 1 || cap < 1 || tight_cap < 1) return wfail(NLEM_ERR_INVALID, "check_every, cap and tight_cap must be >= 1");
  if (!std::isfinite(box.lo) || !std::isfinite(box.hi) || box.lo > box.hi) return wfail(NLEM_ERR_INVALID, "bad box");
  if (rho_counts)
    for (int j = 0; j < n_rho; ++j) rho_counts[j] = 0;
  if (n == 0) return NLEM_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int d = patch * patch;
  const size_t npix = (size_t)H * W;
  if ((rc = grow(&ctx->lab_out, &ctx->lab_out_cap, npix, "label outputs"))) return rc;
  if ((rc = grow(&ctx->lab_iters, &ctx->lab_iters_cap, npix, "label iterations"))) return rc;
  if ((rc = grow(&ctx->lab_rho_map, &ctx->lab_rho_map_cap, npix, "label penalty map"))) return rc;
  if ((rc = grow(&ctx->lab_z, &ctx->lab_z_cap, npix * d, "label patches"))) return rc;
  if ((rc = grow(&ctx->lab_best_it, &ctx->lab_best_it_cap, (size_t)n, "label iteration counts"))) return rc;
  if ((rc = grow(&ctx->lab_best_rho, &ctx->lab_best_rho_cap, (size_t)n, "label penalties"))) return rc;
  if ((rc = grow(&ctx->lab_grid, &ctx->lab_grid_cap, (size_t)n_rho, "penalty grid"))) return rc;
  if ((rc = grow(&ctx->lab_counts, &ctx->lab_counts_cap, (size_t)n_rho, "penalty counts"))) return rc;
  cudaError_t e = cudaMemcpyAsync(ctx->lab_grid, rho_grid, sizeof(float) * n_rho, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->lab_counts, 0, sizeof(unsigned long long) * n_rho, s);
  if (e != cudaSuccess) return wcuda(e, "label set-up");
  const long long total = (long long)npix;
  int ke = nlemk::ws_label_init(n, ctx->lab_best_it, ctx->lab_best_rho, ctx->sm_count, s);
  if (ke) return wcuda((cudaError_t)ke, "label init");
  nlem_options o;
  nlem_options_default(&o);
  o.tol = tol;
  o.check_every = check_every;
  // 1. every pixel solved with each penalty of the grid; the first to reach the tolerance wins
  for (int j = 0; j < n_rho; ++j) {
    rc = nlem_denoise_ex(ctx, image, H, W, pitch, patch, window, h, rho_grid[j], cap, box, &o, pixels, n, nullptr,
                         nullptr, ctx->lab_out, ctx->lab_iters, nullptr, nullptr, stream);
    if (rc) return rc;
    ke = nlemk::ws_label_select(ctx->lab_iters, total, pixels, n, rho_grid[j], ctx->lab_best_it, ctx->lab_best_rho,
                                ctx->sm_count, s);
    if (ke) return wcuda((cudaError_t)ke, "label selection");
  }
  // 2. the label penalties as a per-pixel map, and how often each grid value won
  ke = nlemk::ws_fill(ctx->lab_rho_map, total, 1.f, ctx->sm_count, s);
  if (!ke)
    ke = nlemk::ws_label_scatter(pixels, n, total, ctx->lab_best_rho, ctx->lab_rho_map, ctx->lab_grid, n_rho,
                                 ctx->lab_counts, ctx->sm_count, s);
  if (ke) return wcuda((cudaError_t)ke, "label penalty map");
  // 3. the tight solve at each pixel's label penalty gives the label start point
  o.tol = tight_tol;
  rc = nlem_denoise_ex(ctx, image, H, W, pitch, patch, window, h, 1.f, tight_cap, box, &o, pixels, n, nullptr,
                       ctx->lab_rho_map, ctx->lab_out, ctx->lab_iters, nullptr, ctx->lab_z, stream);
  if (rc) return rc;
  // 4. the targets of the network output
  ke = nlemk::ws_label_targets(ctx->lab_z, total, pixels, n, d, feats, ctx->lab_best_rho, targets, ctx->sm_count, s);
  if (ke) return wcuda((cudaError_t)ke, "label targets");
  if (rho_counts) {
    std::vector<unsigned long long> c((size_t)n_rho);
    e = cudaMemcpyAsync(c.data(), ctx->lab_counts, sizeof(unsigned long long) * n_rho, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return wcuda(e, "read penalty counts");
    for (int j = 0; j < n_rho; ++j) rho_counts[j] = (long long)c[(size_t)j];
  }
  return NLEM_OK;
}

int nlem_denoise_warm(nlem_ctx* ctx, nlem_warmstart* ws, const float* image, int H, int W, int pitch, int patch,
                      int window, float h, float rho_fallback, int iters, nlem_box box, const nlem_options* opt,
                      float* out, int* iters_used, long long* fallback_count, void* stream) {
  NLEM_TRACE("nlem_denoise_warm");
  int rc = check_nlem_args(ctx, image, H, W, pitch, patch, window, h);
  if (rc) return rc;
  if (!ws || !out || !iters_used) return wfail(NLEM_ERR_INVALID, "ws, out and iters_used must be non-NULL");
  if (ws->m.d != patch * patch) return wfail(NLEM_ERR_INVALID, "model is for d = %d, patch gives %d", ws->m.d, patch * patch);
  if (!opt || !(opt->tol > 0.f)) return wfail(NLEM_ERR_INVALID, "the warm start needs a tolerance (opt->tol > 0)");
  if (opt->solver != NLEM_SOLVER_ADMM) return wfail(NLEM_ERR_INVALID, "the warm start runs EM-ADMM only");
  if (!(rho_fallback > 0.f) || iters < 1 || !(box.lo <= box.hi)) return wfail(NLEM_ERR_INVALID, "bad rho, iters or box");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int d = patch * patch;
  const size_t npix = (size_t)H * W;
  if (npix > ctx->ws_warm_pixels || d != ctx->ws_warm_d) {
    cudaStreamSynchronize(s);
    size_t cf = 0, cy = 0, cx = 0, cr = 0, cl = 0;
    ctx->ws_warm_pixels = 0;
    if ((rc = grow(&ctx->ws_feats, &cf, npix * (2 * d + 2), "features"))) return rc;
    if ((rc = grow(&ctx->ws_y, &cy, npix * (d + 1), "network outputs"))) return rc;
    if ((rc = grow(&ctx->ws_x0, &cx, npix * d, "start points"))) return rc;
    if ((rc = grow(&ctx->ws_rho, &cr, npix, "penalties"))) return rc;
    if ((rc = grow(&ctx->ws_list, &cl, npix, "fallback list"))) return rc;
    ctx->ws_warm_pixels = npix;
    ctx->ws_warm_d = d;
  }
  if ((rc = ensure_counts(ctx))) return rc;
  // 1. features of every pixel's problem
  rc = nlem_features(ctx, image, H, W, pitch, patch, window, h, nullptr, 0, ctx->ws_feats, stream);
  if (rc) return rc;
  // 2. network -> (x0, rho)
  rc = nlem_ws_predict(ctx, ws, ctx->ws_feats, (long long)npix, box, ctx->ws_y, ctx->ws_x0, ctx->ws_rho, stream);
  if (rc) return rc;
  // 3. EM-ADMM from the learned start and penalty
  nlemk::NlemLaunch L = base_launch(ctx, image, H, W, pitch, patch, window, h, rho_fallback, iters, box, opt, s);
  L.out = out;
  L.iters_used = iters_used;
  L.ex.x0 = ctx->ws_x0;
  L.ex.rho = ctx->ws_rho;
  if ((rc = run_launch(L, "warm-started solve"))) return rc;
  // 4. plain EM-ADMM (weighted-mean start, rho_fallback) where the cap was reached first
  rc = nlemk::ws_fallback_list(iters_used, (long long)npix, iters, ctx->ws_list, ctx->ws_count, ctx->sm_count, s);
  if (rc) return wcuda((cudaError_t)rc, "fallback list");
  nlemk::NlemLaunch F = base_launch(ctx, image, H, W, pitch, patch, window, h, rho_fallback, iters, box, opt, s);
  F.out = out;
  F.iters_used = iters_used;
  F.pix_list = ctx->ws_list;
  F.n_list = ctx->ws_count;
  F.max_items = (long long)npix;
  if ((rc = run_launch(F, "fallback solve"))) return rc;
  if (fallback_count) {
    cudaError_t e = cudaMemcpyAsync(fallback_count, ctx->ws_count, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return wcuda(e, "read fallback count");
  }
  return NLEM_OK;
}

}  // extern "C"
