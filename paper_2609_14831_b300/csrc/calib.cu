// calib.cu -- measured arithmetic roofs of this GPU (the FP64 rate binds the
// FP64 graph traversal on B300, so the benchmark reports against a measured
// number, not a datasheet figure).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "cut.h"
#include "status.h"

namespace cut {
namespace calib {

// Independent FMA chains per thread (enough in flight to fill the pipe);
// the result is stored only when it equals an impossible value, so the
// compiler keeps every FMA and nothing is written.
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) fma_chains(int iters, T b, T c, T *sink) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; k++) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < CHAINS; k++) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; k++) s += a[k];
    if (s == T(-1.2345e30)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t rate(int device, double seconds, double *tflops) {
    constexpr int CHAINS = 8;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const int blocks = nsm * 8, threads = 256;
    cudaStream_t s;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    // b, c keep |a| bounded (a -> a b + c converges to c / (1 - b))
    const T b = T(0.999999), c = T(1e-7);
    int iters = 1024;
    float ms = 0.0f;
    for (int pass = 0; pass < 8; pass++) {   // grow the loop until one launch takes ~seconds / 4
        cudaEventRecord(t0, s);
        fma_chains<T, CHAINS><<<blocks, threads, 0, s>>>(iters, b, c, nullptr);
        cudaEventRecord(t1, s);
        if ((e = cudaEventSynchronize(t1)) != cudaSuccess) break;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms >= 250.0 * seconds || iters >= (1 << 28) / 4) break;
        iters = (int)std::min<double>((double)iters * std::max(2.0, 250.0 * seconds / std::max(ms, 0.01f)),
                                      (double)(1 << 28));
    }
    if (e == cudaSuccess) {
        // timed: best of three launches of the final size
        float best = 1e30f;
        for (int r = 0; r < 3 && e == cudaSuccess; r++) {
            cudaEventRecord(t0, s);
            fma_chains<T, CHAINS><<<blocks, threads, 0, s>>>(iters, b, c, nullptr);
            cudaEventRecord(t1, s);
            e = cudaEventSynchronize(t1);
            cudaEventElapsedTime(&ms, t0, t1);
            best = std::min(best, ms);
        }
        const double flop = 2.0 * CHAINS * (double)iters * blocks * threads;
        *tflops = flop / (best * 1e-3) / 1e12;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamDestroy(s);
    return e;
}

}  // namespace calib
}  // namespace cut

extern "C" cut_status cut_measure_fma_rate(int device, int fp64, double seconds, double *tflops) {
    using namespace cut;
    if (!tflops || device < 0 || !(seconds > 0.0) || seconds > 60.0)
        return set_error(CUT_ERR_INVALID_ARG, "cut_measure_fma_rate: bad argument");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    cudaError_t e = fp64 ? calib::rate<double>(device, seconds, tflops) : calib::rate<float>(device, seconds, tflops);
    cudaSetDevice(cur);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_measure_fma_rate: ") + cudaGetErrorString(e));
    return CUT_OK;
}
