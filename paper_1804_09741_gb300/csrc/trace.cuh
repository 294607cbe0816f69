// NVTX ranges over the library's host entry points: a profiler attached to
// the process (Nsight Systems, Nsight Compute's range filters) shows where a
// table build, a graph load, a batch step or a serving round starts and ends;
// without one, a push/pop costs a few nanoseconds (NVTX v3, header only).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mt {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace mt
