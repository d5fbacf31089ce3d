// xy_trace.h -- named NVTX ranges around the library's host entry points, so
// a timeline tool shows each call (sweeps, measures, batch rounds, HMC
// trajectories) over the kernels it launched.  NVTX v3 is header-only and does
// nothing unless a tool is attached; a toolkit without it compiles the ranges
// to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define XY_HAVE_NVTX 1
#endif
#endif

namespace xyk {

// One range for the lifetime of the object (the enclosing entry point).
struct TraceRange {
  explicit TraceRange(const char* name) {
#ifdef XY_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifdef XY_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace xyk
