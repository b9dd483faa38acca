// trace.h — NVTX ranges around the library's host entry points (a sweep launch, a batch run, a
// serving tick), so that a profiler can attribute the kernels to the calls that issued them.
// Without a tool attached a range costs two calls that return at once.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace isf {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace isf
