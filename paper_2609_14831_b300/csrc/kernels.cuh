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

// Exact factors of one graph.  When every factor has the same magnitude
// (+-1 for fermion monomials, +-2 for Pauli strings) the record's factor is
// a sign, applied by flipping the sign bit of one operand, and the magnitude
// multiplies the finished row sum once: one FP64 FMA per record and operand,
// which is what bounds these kernels on B300 (the FP64 pipe, not HBM).
struct Weights {
    const double *val;                 // value of each code
    const unsigned long long *sign;    // sign bit of each code (uniform case)
    double mag;                        // common magnitude (uniform case)
    int n_codes, uniform;
};

__device__ __forceinline__ void load_weights(double *ws, unsigned long long *sg, const Weights &w) {
    for (int c = threadIdx.x; c < w.n_codes; c += blockDim.x) {
        ws[c] = w.val[c];
        sg[c] = w.sign[c];
    }
    __syncthreads();
}

// +-v by the code's sign bit (an integer XOR, no FP64 instruction)
__device__ __forceinline__ double signed_by(double v, unsigned long long sbit) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)sbit);
}

// Generator stage: xi[a] = sum_e alpha_e h[i_e] h[j_e]   (Eq. graph-actions, line 1)
template <bool UNIFORM>
__global__ void __launch_bounds__(kBlock) gen_stage(const uint64_t *__restrict__ rp,
                                                    const uint2 *__restrict__ rec, Weights wt,
                                                    const double *__restrict__ h,
                                                    double *__restrict__ xi, int64_t rows,
                                                    const int *done) {
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        const uint64_t b = rp[r], e = rp[r + 1];
        double acc = 0.0;
        uint64_t p = b + lane;
#define TERM(q)                                                                   \
    (UNIFORM ? signed_by(h[(q).x & kIdx], sg[(q).x >> 24]) * h[(q).y]             \
             : ws[(q).x >> 24] * h[(q).x & kIdx] * h[(q).y])
        for (; p + 96 < e; p += 128) {
            uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + 32), q2 = __ldcs(rec + p + 64),
                  q3 = __ldcs(rec + p + 96);
            acc += TERM(q0);
            acc += TERM(q1);
            acc += TERM(q2);
            acc += TERM(q3);
        }
        for (; p < e; p += 32) {
            uint2 q = __ldcs(rec + p);
            acc += TERM(q);
        }
#undef TERM
        acc = warp_sum(acc);
        if (lane == 0) xi[r] = UNIFORM ? acc * wt.mag : acc;
    }
}

template <int NOPS>
struct Ops {
    const double *x[NOPS];
    double *dx[NOPS];
};

// Commutator stage: dx_o[k] = sum_e beta_e xi[a_e] x_o[j_e]  (Eq. graph-actions,
// line 2) for NOPS operands at once: one record read serves every operand.
template <int NOPS, bool UNIFORM>
__global__ void __launch_bounds__(kBlock) comm_stage(const uint64_t *__restrict__ rp,
                                                     const uint2 *__restrict__ rec, Weights wt,
                                                     const double *__restrict__ xi, Ops<NOPS> ops,
                                                     int64_t rows, const int *done) {
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        const uint64_t b = rp[r], e = rp[r + 1];
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        uint64_t p = b + lane;
#define COEF(q) (UNIFORM ? signed_by(xi[(q).x & kIdx], sg[(q).x >> 24]) : ws[(q).x >> 24] * xi[(q).x & kIdx])
        for (; p + 32 < e; p += 64) {
            uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + 32);
            const double c0 = COEF(q0), c1 = COEF(q1);
#pragma unroll
            for (int o = 0; o < NOPS; o++) {
                acc[o] += c0 * ops.x[o][q0.y];
                acc[o] += c1 * ops.x[o][q1.y];
            }
        }
        for (; p < e; p += 32) {
            uint2 q = __ldcs(rec + p);
            const double c = COEF(q);
#pragma unroll
            for (int o = 0; o < NOPS; o++) acc[o] += c * ops.x[o][q.y];
        }
#undef COEF
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            double v = warp_sum(acc[o]);
            if (lane == 0) ops.dx[o][r] = UNIFORM ? v * wt.mag : v;
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
