// pdl.cuh -- programmatic dependent launch.
//
// The library launches its kernels with programmatic stream serialization,
// so a kernel's blocks may become resident while the kernel before it on the
// stream is still running.  Every such kernel waits on the device
// (pdl_wait) before it touches memory its predecessor writes or reads, and
// then lets the next grid on the stream be scheduled (pdl_trigger); that
// grid waits the same way, so only launch latency and set-up (barriers,
// tensor-memory allocation) overlap the previous kernel, never its work.
// For a kernel launched without the attribute both instructions return at
// once.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <utility>

namespace cut {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

// Kernel launch with programmatic stream serialization.
template <typename... P, typename... A>
static inline cudaError_t pdl_launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     A &&...args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at;
    memset(&at, 0, sizeof(at));
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace cut
