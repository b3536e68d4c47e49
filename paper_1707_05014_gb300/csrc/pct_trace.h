// Named host-side ranges around the library's entry points (NVTX v3, header
// only). They cost one indirect call when no tool is attached; under a
// profiler (ncu --nvtx) they mark which call queued the work, e.g. the load,
// the first sweep after it, or a batch autotune.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace pct {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pct
