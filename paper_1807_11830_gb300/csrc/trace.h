// Host-side NVTX ranges around the library's entry points, so a timeline
// tool (Nsight Systems, or ncu --nvtx --nvtx-include "<name>/") can attribute
// every kernel to the call that enqueued it.  Ranges cover the host call
// (validation, launches, graph replay), not device execution.  NVTX is
// header-only and costs a few nanoseconds per range when no tool is
// attached; without its headers the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define SENSE_HAVE_NVTX 1
#endif
#endif

namespace sense {

class TraceRange {
 public:
  explicit TraceRange(const char* name) {
#ifdef SENSE_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifdef SENSE_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace sense
