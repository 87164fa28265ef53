// alloc.h -- device scratch of the library's calls.
#pragma once
#include <cuda_runtime.h>

namespace cut {
// Stream-ordered allocation from the library's own memory pool of the
// current device and context (free with cudaFreeAsync).  The pool keeps up
// to kScratchKeepBytes of freed scratch reserved across calls, so a call
// that follows another of the same size maps no new memory; the default
// pool (release threshold 0) returns it to the driver at every
// synchronisation.
constexpr unsigned long long kScratchKeepBytes = 1ull << 30;
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t scratch_alloc(T **p, size_t bytes, cudaStream_t s) {
    return scratch_alloc(reinterpret_cast<void **>(p), bytes, s);
}
}  // namespace cut
