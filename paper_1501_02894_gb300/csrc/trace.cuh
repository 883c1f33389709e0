// trace.cuh -- named host ranges for profilers (NVTX, header-only: a no-op
// unless a profiling tool is attached to the process).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace fic {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace fic
