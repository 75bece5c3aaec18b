// swe_trace.h -- NVTX ranges around the host ABI calls, so that a profiler's
// timeline (Nsight Systems, ncu's NVTX filters) shows which call issued
// which work.  NVTX 3 is header-only and costs a null check per range when
// no tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace swe {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace swe
