// Host-side trace ranges: each C-ABI call opens an NVTX range named after itself, so that a
// profiler's timeline (Nsight Systems, or ncu with --nvtx) shows which library call issued which
// kernels.  NVTX v3 is header-only and loads its implementation only when a tool is attached;
// without one a range costs two calls that return at once.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace nlemk {
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace nlemk

#define NLEM_TRACE(name) ::nlemk::TraceRange nlem_trace_range_(name)
