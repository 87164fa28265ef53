// kernels.cuh -- sm_103a kernels of the graph traversals (paper Eq.
// graph-actions and Sec. 2.4).
//
// Records of one output form a contiguous CSR segment (Sec. 2.2: "records
// that contribute to the same output are stored together").  One warp owns a
// segment: its lanes stream the packed 8-byte records with coalesced loads,
// multiply the exact factor by the gathered coefficients, and the partial
// sums meet in a warp-shuffle reduction.  Nothing is scattered and nothing
// uses atomics, so every result is bitwise reproducible.
#pragma once
#include <cstdint>

namespace cut {
namespace k {

constexpr uint32_t kIdx = (1u << 24) - 1;
constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = 32 * kWarpsPerBlock;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool skip(const int *done) { return done != nullptr && *done != 0; }

// Load the exact factor table (<= 256 values) into shared memory.
__device__ __forceinline__ void load_table(double *ws, const double *wtab, int n_codes) {
    for (int c = threadIdx.x; c < n_codes; c += blockDim.x) ws[c] = wtab[c];
    __syncthreads();
}

// Generator stage: xi[a] = sum_e alpha_e h[i_e] h[j_e]   (Eq. graph-actions, line 1)
__global__ void __launch_bounds__(kBlock) gen_stage(const uint64_t *__restrict__ rp,
                                                    const uint2 *__restrict__ rec,
                                                    const double *__restrict__ wtab, int n_codes,
                                                    const double *__restrict__ h,
                                                    double *__restrict__ xi, int64_t rows,
                                                    const int *done) {
    __shared__ double ws[256];
    if (skip(done)) return;
    load_table(ws, wtab, n_codes);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        const uint64_t b = rp[r], e = rp[r + 1];
        double acc = 0.0;
        uint64_t p = b + lane;
        for (; p + 96 < e; p += 128) {
            uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + 32), q2 = __ldcs(rec + p + 64),
                  q3 = __ldcs(rec + p + 96);
            acc += ws[q0.x >> 24] * h[q0.x & kIdx] * h[q0.y];
            acc += ws[q1.x >> 24] * h[q1.x & kIdx] * h[q1.y];
            acc += ws[q2.x >> 24] * h[q2.x & kIdx] * h[q2.y];
            acc += ws[q3.x >> 24] * h[q3.x & kIdx] * h[q3.y];
        }
        for (; p < e; p += 32) {
            uint2 q = __ldcs(rec + p);
            acc += ws[q.x >> 24] * h[q.x & kIdx] * h[q.y];
        }
        acc = warp_sum(acc);
        if (lane == 0) xi[r] = acc;
    }
}

template <int NOPS>
struct Ops {
    const double *x[NOPS];
    double *dx[NOPS];
};

// Commutator stage: dx_o[k] = sum_e beta_e xi[a_e] x_o[j_e]  (Eq. graph-actions,
// line 2) for NOPS operands at once: one record read serves every operand.
template <int NOPS>
__global__ void __launch_bounds__(kBlock) comm_stage(const uint64_t *__restrict__ rp,
                                                     const uint2 *__restrict__ rec,
                                                     const double *__restrict__ wtab, int n_codes,
                                                     const double *__restrict__ xi, Ops<NOPS> ops,
                                                     int64_t rows, const int *done) {
    __shared__ double ws[256];
    if (skip(done)) return;
    load_table(ws, wtab, n_codes);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        const uint64_t b = rp[r], e = rp[r + 1];
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        uint64_t p = b + lane;
        for (; p + 32 < e; p += 64) {
            uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + 32);
            double c0 = ws[q0.x >> 24] * xi[q0.x & kIdx];
            double c1 = ws[q1.x >> 24] * xi[q1.x & kIdx];
#pragma unroll
            for (int o = 0; o < NOPS; o++) {
                acc[o] += c0 * ops.x[o][q0.y];
                acc[o] += c1 * ops.x[o][q1.y];
            }
        }
        for (; p < e; p += 32) {
            uint2 q = __ldcs(rec + p);
            double c = ws[q.x >> 24] * xi[q.x & kIdx];
#pragma unroll
            for (int o = 0; o < NOPS; o++) acc[o] += c * ops.x[o][q.y];
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            double v = warp_sum(acc[o]);
            if (lane == 0) ops.dx[o][r] = v;
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Transposed commutator pass over operands: rows j, entries (code|a, k):
//   x_bar_o[j] = sum beta xi[a] w_o[k]
template <int NOPS>
__global__ void __launch_bounds__(kBlock) commT_x(const uint64_t *__restrict__ rp,
                                                  const uint2 *__restrict__ rec,
                                                  const double *__restrict__ wtab, int n_codes,
                                                  const double *__restrict__ xi, Ops<NOPS> ops,
                                                  int64_t rows) {
    __shared__ double ws[256];
    load_table(ws, wtab, n_codes);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        for (uint64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            uint2 q = __ldcs(rec + p);
            double c = ws[q.x >> 24] * xi[q.x & kIdx];
#pragma unroll
            for (int o = 0; o < NOPS; o++) acc[o] += c * ops.x[o][q.y];  // x holds w_o
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            double v = warp_sum(acc[o]);
            if (lane == 0) ops.dx[o][r] = v;
        }
    }
}

// Transposed commutator pass over the generator: rows a, entries (code|k, j):
//   xi_bar[a] = sum beta sum_o x_o[j] w_o[k]
template <int NOPS>
struct Pairs {
    const double *x[NOPS];
    const double *w[NOPS];
};

template <int NOPS>
__global__ void __launch_bounds__(kBlock) commT_xi(const uint64_t *__restrict__ rp,
                                                   const uint2 *__restrict__ rec,
                                                   const double *__restrict__ wtab, int n_codes,
                                                   Pairs<NOPS> pr, double *__restrict__ xi_bar,
                                                   int64_t rows, int accumulate) {
    __shared__ double ws[256];
    load_table(ws, wtab, n_codes);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        double acc = 0.0;
        for (uint64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            uint2 q = __ldcs(rec + p);
            const uint32_t kk = q.x & kIdx;
            double s = 0.0;
#pragma unroll
            for (int o = 0; o < NOPS; o++) s += pr.x[o][q.y] * pr.w[o][kk];
            acc += ws[q.x >> 24] * s;
        }
        acc = warp_sum(acc);
        if (lane == 0) xi_bar[r] = accumulate ? xi_bar[r] + acc : acc;
    }
}

// Transposed generator pass: rows = registry coordinates r, entries
// (code|a, other) where `other` is the partner input of the record:
//   h_bar[r] = x0_bar[r] + sum alpha xi_bar[a] h[other]
__global__ void __launch_bounds__(kBlock) genT(const uint64_t *__restrict__ rp,
                                               const uint2 *__restrict__ rec,
                                               const double *__restrict__ wtab, int n_codes,
                                               const double *__restrict__ xi_bar,
                                               const double *__restrict__ h,
                                               const double *__restrict__ x0_bar,
                                               double *__restrict__ h_bar, int64_t rows) {
    __shared__ double ws[256];
    load_table(ws, wtab, n_codes);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        double acc = 0.0;
        for (uint64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            uint2 q = __ldcs(rec + p);
            acc += ws[q.x >> 24] * xi_bar[q.x & kIdx] * h[q.y];
        }
        acc = warp_sum(acc);
        if (lane == 0) h_bar[r] = (x0_bar ? x0_bar[r] : 0.0) + acc;
    }
}

// ---------------------------------------------------------------- RK algebra
// out = base + sum_s coef_s * ds * K_s   (coefficients scaled by *ds_ptr
// when ds_ptr is given, else by ds_const); vectors of length len.
struct Combine {
    const double *base;
    const double *K[7];
    double c[7];
    int nk;
};

__global__ void rk_combine(Combine cb, double *__restrict__ out, int64_t len, const double *ds_ptr,
                           double ds_const, const int *done) {
    if (skip(done)) return;
    const double ds = ds_ptr ? *ds_ptr : ds_const;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = cb.base[i];
        for (int s = 0; s < cb.nk; s++) v += (cb.c[s] * ds) * cb.K[s][i];
        out[i] = v;
    }
}

}  // namespace k
}  // namespace cut
