// Host-side trace ranges: every entry point that enqueues device work opens an
// NVTX range named after itself for the length of the call, so that a profiler
// can attribute and select the kernels each call launches (ncu --nvtx
// --nvtx-include "rx_batch_run/").  With no tool attached a range costs one
// branch.  Host code only.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace rxh {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace rxh
