// trace.h -- named ranges around the library's phases, for profilers and logs.
//
// The paper reports compile, reload, set-up and execution separately; the
// library marks the same phases as NVTX ranges ("cut_build/count",
// "cut_graph_load/upload", "cut_flow", ...), so that a profiler attached to
// the caller's program shows where each call spends its time.  With the
// environment variable CUT_LOG set to 1 or more, every range also writes one
// line "[cut] <name> <milliseconds> ms" to stderr when it closes (host wall
// time: for calls that only queue GPU work, the time to queue it).  With no
// profiler attached and CUT_LOG unset a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace cut {

inline int trace_log_level() {
    static const int level = [] {
        const char *v = std::getenv("CUT_LOG");
        return v ? std::atoi(v) : 0;
    }();
    return level;
}

// A range from construction to end() or destruction, whichever is first
// (an exception still closes it).
struct TraceRange {
    explicit TraceRange(const char *name) : name_(name) {
        nvtxRangePushA(name);
        if (trace_log_level() > 0) t0_ = std::chrono::steady_clock::now();
    }
    void end() {
        if (!open_) return;
        nvtxRangePop();
        open_ = false;
        if (trace_log_level() > 0) {
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
            std::fprintf(stderr, "[cut] %s %.3f ms\n", name_, ms);
        }
    }
    ~TraceRange() { end(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

  private:
    const char *name_;
    bool open_ = true;
    std::chrono::steady_clock::time_point t0_;
};

}  // namespace cut
