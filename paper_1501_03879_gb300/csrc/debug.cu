// nlem_debug_status: the fault record of the debug build's bounds checks (debug.h).
#include <cuda_runtime.h>

#include "../../include/nlem.h"
#include "debug.h"
#include "kernels.h"

namespace nlemk {
#ifdef NLEM_DEBUG
__device__ DebugRecord g_nlem_debug;
#endif
}  // namespace nlemk

extern "C" int nlem_debug_status(int reset, int* site, long long* index, long long* limit, long long* count) {
#ifdef NLEM_DEBUG
  nlemk::DebugRecord r{};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&r, nlemk::g_nlem_debug, sizeof(r));
  if (e == cudaSuccess && reset) {
    const nlemk::DebugRecord z{};
    e = cudaMemcpyToSymbol(nlemk::g_nlem_debug, &z, sizeof(z));
  }
  if (e != cudaSuccess) {
    nlemk::set_last_error(cudaGetErrorString(e));
    return NLEM_ERR_CUDA;
  }
  if (site) *site = r.site;
  if (index) *index = r.index;
  if (limit) *limit = r.limit;
  if (count) *count = (long long)r.count;
  return NLEM_OK;
#else
  (void)reset;
  if (site) *site = 0;
  if (index) *index = 0;
  if (limit) *limit = 0;
  if (count) *count = 0;
  nlemk::set_last_error("not a debug build (libnlem_debug.so has the bounds checks)");
  return NLEM_ERR_UNSUPPORTED;
#endif
}
