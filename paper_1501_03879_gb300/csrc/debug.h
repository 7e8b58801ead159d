// Bounds checks of the debug build (-DNLEM_DEBUG, built as libnlem_debug.so).  The shared-memory
// tile, point-row and image indices that depend on the image size, the window clipping, the
// reflect padding and the work-item lookup are checked against the size of what they index: an
// index outside it is recorded in one device record (the first fault: its site, index and limit,
// plus a count of all faults) and the access is skipped (a load reads 0), so that the kernel runs
// on and the host reads the record with nlem_debug_status.  In the release build every check
// is the constant true and the access compiles as written.
#pragma once
#include <cuda_runtime.h>

namespace nlemk {

// sites of the checked accesses
enum DebugSite : int {
  kDbgTileWrite = 1,      // one-pixel NLEM: tile store
  kDbgImageRead = 2,      // NLEM kernels: image load (reflect-padded row and column)
  kDbgTileRead = 3,       // one-pixel NLEM: tile load while filling the point rows or the centre patch
  kDbgPointRow = 4,       // point-row store (NLEM set-up or standalone batch)
  kDbgPairTile = 5,       // pixel pairs: tile store or load
  kDbgPairRow = 6,        // pixel pairs: point-row store
  kDbgBatchItem = 7,      // batched launch: item -> image lookup
  kDbgFastVec = 8,        // accelerated solver: a finalize lane's pair of d-vector slots
  kDbgFastPartial = 9,    // accelerated solver: a per-warp partial column sum
};

struct DebugRecord {
  unsigned long long count;   // faults seen since the last reset
  int site;                   // the first fault's site
  int pad;
  long long index, limit;     // its index and the size it was checked against
};

#ifdef NLEM_DEBUG
extern __device__ DebugRecord g_nlem_debug;
__device__ __forceinline__ bool dbg_ok(long long index, long long limit, int site) {
  if (index >= 0 && index < limit) return true;
  if (atomicAdd(&g_nlem_debug.count, 1ull) == 0ull) {
    g_nlem_debug.site = site;
    g_nlem_debug.index = index;
    g_nlem_debug.limit = limit;
  }
  return false;
}
#define NLEM_DBG_OK(index, limit, site) ::nlemk::dbg_ok((long long)(index), (long long)(limit), (site))
#else
#define NLEM_DBG_OK(index, limit, site) ((void)(index), (void)(limit), true)
#endif

}  // namespace nlemk
