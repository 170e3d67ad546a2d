// NVTX ranges around the library's stages (set-up, low-rank build, solve,
// batched set-up and solve), so that ncu and nsys show them on the timeline.
// NVTX v3 is header-only; with no tool attached a range costs a few branches.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pslr {

class TraceRange {
  public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace pslr
