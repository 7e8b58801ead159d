// nlem_denoise_batch_noalloc: the batched NLEM launch for callers that must not allocate
// device memory, e.g. code running inside another framework's memory pool or allocator
// hooks, or under a strict memory budget where every device allocation belongs to the host
// application.  The work-queue counter and the image descriptors, which nlem_denoise_batch
// keeps in a context workspace obtained with cudaMalloc, live here in one file-scope device
// array instead.  The kernel is the same persistent batch kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/nlem.h"
#include "batch.h"
#include "kernels.h"
#include "trace.h"

namespace {

constexpr size_t kQueueBytes = 256;   // the counter, padded so the descriptors stay aligned
constexpr size_t kScratchBytes = kQueueBytes + sizeof(nlemk::BatchImage) * NLEM_NOALLOC_MAX_IMAGES;

// Every GPU that loads the library holds this array until the process exits.  All calls on a
// device share it; each call rewrites the descriptors and clears the counter.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

int nerr(int code, const char* msg, int image = -1) {
  char buf[256];
  if (image >= 0)
    std::snprintf(buf, sizeof(buf), "image %d: %s", image, msg);
  else
    std::snprintf(buf, sizeof(buf), "%s", msg);
  nlemk::set_last_error(buf);   // reported by nlem_last_error()
  return code;
}

}  // namespace

extern "C" int nlem_denoise_batch_noalloc(const nlem_image_desc* images, int count, float rho, int iters,
                                          nlem_box box, const nlem_options* opt, void* stream) {
  NLEM_TRACE("nlem_denoise_batch_noalloc");
  if (count < 0 || count > NLEM_NOALLOC_MAX_IMAGES)
    return nerr(NLEM_ERR_INVALID, "count must be in [0, NLEM_NOALLOC_MAX_IMAGES]");
  if (count == 0) return NLEM_OK;
  if (!images) return nerr(NLEM_ERR_INVALID, "images is NULL");
  if (!(rho > 0.f) || !std::isfinite(rho)) return nerr(NLEM_ERR_INVALID, "rho must be finite and > 0");
  if (iters < 0) return nerr(NLEM_ERR_INVALID, "iters must be >= 0");
  if (!std::isfinite(box.lo) || !std::isfinite(box.hi) || box.lo > box.hi)
    return nerr(NLEM_ERR_INVALID, "box must satisfy lo <= hi, both finite");
  // the option checks of nlem_denoise_batch, with its error codes
  if (opt) {
    if (opt->check_every < 1) return nerr(NLEM_ERR_INVALID, "check_every must be >= 1");
    if (!std::isfinite(opt->tol)) return nerr(NLEM_ERR_INVALID, "tol must be finite");
    if (opt->precision != NLEM_PREC_FP32 && opt->precision != NLEM_PREC_BF16)
      return nerr(NLEM_ERR_INVALID, "unknown precision");
    if (opt->init != NLEM_INIT_WEIGHTED_MEAN && opt->init != NLEM_INIT_NOISY_PATCH)
      return nerr(NLEM_ERR_INVALID, "unknown init");
    if (opt->layout < NLEM_LAYOUT_AUTO || opt->layout > NLEM_LAYOUT_PAIR)
      return nerr(NLEM_ERR_INVALID, "unknown layout");
    if (opt->penalty != NLEM_PENALTY_UNIFORM && opt->penalty != NLEM_PENALTY_WEIGHTED)
      return nerr(NLEM_ERR_INVALID, "unknown penalty");
    if (opt->solver != NLEM_SOLVER_ADMM && opt->solver != NLEM_SOLVER_IRLS && opt->solver != NLEM_SOLVER_FAST)
      return nerr(NLEM_ERR_INVALID, "unknown solver");
    if (opt->restart_every < 0) return nerr(NLEM_ERR_INVALID, "restart_every must be >= 0");
    if (opt->solver == NLEM_SOLVER_IRLS)
      return nerr(NLEM_ERR_INVALID, "the batched kernel runs EM-ADMM only (plain or accelerated), not IRLS");
    if (opt->penalty != NLEM_PENALTY_UNIFORM)
      return nerr(NLEM_ERR_UNSUPPORTED, "the batched kernel takes one penalty for every point only");
    if (opt->precision != NLEM_PREC_FP32)
      return nerr(NLEM_ERR_UNSUPPORTED, "the batched kernel computes weights in FP32 only");
  }

  // descriptors on the stack: this entry point makes no heap or device allocation of its own
  nlemk::BatchImage host[NLEM_NOALLOC_MAX_IMAGES];
  long long total = 0;
  for (int i = 0; i < count; ++i) {
    const nlem_image_desc& d = images[i];
    if (!d.image || !d.out) return nerr(NLEM_ERR_INVALID, "image and out must be non-NULL", i);
    if (d.H < 1 || d.W < 1 || d.pitch < d.W) return nerr(NLEM_ERR_INVALID, "bad size or pitch", i);
    if (d.patch < 1 || d.patch % 2 == 0 || d.window < 1 || d.window % 2 == 0)
      return nerr(NLEM_ERR_INVALID, "patch and window must be odd and >= 1", i);
    if (d.patch > (d.H < d.W ? d.H : d.W)) return nerr(NLEM_ERR_INVALID, "patch exceeds the image side", i);
    if (!(d.h > 0.f) || !std::isfinite(d.h)) return nerr(NLEM_ERR_INVALID, "h must be finite and > 0", i);
    if (d.patch != 5 && d.patch != 7) return nerr(NLEM_ERR_UNSUPPORTED, "patch must be 5 or 7", i);
    if (d.window * d.window > nlemk::batch_max_points(d.patch, 0) || !nlemk::batch_tile_fits(d.patch, d.window))
      return nerr(NLEM_ERR_UNSUPPORTED, "window too large for the batched kernel", i);
    nlemk::BatchImage& b = host[i];
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
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nerr(NLEM_ERR_CUDA, cudaGetErrorString(e));
  // The host-side name of the array is not a device address: ask the runtime for the address
  // in the CURRENT context, on every call.  The address belongs to a context, not to a device:
  // after cudaDeviceReset, or under a caller's own driver-API context on the same device, an
  // address kept from an earlier call would be stale.  The lookup allocates nothing; the first
  // call in a context also loads the library's device code there.
  void* scratch_p = nullptr;
  e = cudaGetSymbolAddress(&scratch_p, g_noalloc_scratch);
  if (e != cudaSuccess) return nerr(NLEM_ERR_CUDA, cudaGetErrorString(e));
  unsigned char* scratch = static_cast<unsigned char*>(scratch_p);
  auto* queue = reinterpret_cast<unsigned long long*>(scratch);
  auto* d_imgs = reinterpret_cast<nlemk::BatchImage*>(scratch + kQueueBytes);
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemcpyAsync(d_imgs, host, sizeof(nlemk::BatchImage) * (size_t)count, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return nerr(NLEM_ERR_CUDA, cudaGetErrorString(e));
  e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);   // the counter starts at zero
  if (e != cudaSuccess) return nerr(NLEM_ERR_CUDA, cudaGetErrorString(e));
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return nerr(NLEM_ERR_CUDA, cudaGetErrorString(e));

  nlemk::BatchLaunch L{};
  L.imgs = d_imgs;
  L.count = count;
  L.total = total;
  L.stride = 1;
  L.queue = queue;
  L.cfg = nlemk::BatchConfig{0, 4, 2};   // fixed launch shape: no tuning trials
  L.prm.lo = box.lo;
  L.prm.hi = box.hi;
  L.prm.mu = rho;
  L.prm.inv_mu = 1.f / rho;
  L.prm.iters = iters;
  L.prm.tol = opt ? opt->tol : 0.f;
  L.prm.check_every = opt ? opt->check_every : 1;
  L.prm.solver = opt ? opt->solver : NLEM_SOLVER_ADMM;   // Algorithm 1 or the accelerated solver
  L.prm.restart_every = opt ? opt->restart_every : 0;
  L.prm.d = 0;
  L.init_mode = opt ? opt->init : NLEM_INIT_WEIGHTED_MEAN;
  L.sm_count = sms;
  L.stream = s;
  int rc = nlemk::launch_batch(L);
  if (rc != 0) return nerr(NLEM_ERR_CUDA, cudaGetErrorString((cudaError_t)rc));
  return NLEM_OK;
}
