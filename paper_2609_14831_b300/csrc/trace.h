// trace.h -- named ranges around the library's phases, for profilers.
//
// The paper reports compile, reload, set-up and execution separately; the
// library marks the same phases as NVTX ranges ("cut_build/count",
// "cut_graph_load/upload", "cut_flow", ...), so that a profiler attached to
// the caller's program shows where each call spends its time.  With no
// profiler attached a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace cut {

// A range from construction to end() or destruction, whichever is first
// (an exception still closes it).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    void end() {
        if (open_) nvtxRangePop();
        open_ = false;
    }
    ~TraceRange() { end(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

  private:
    bool open_ = true;
};

}  // namespace cut
