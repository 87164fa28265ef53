// kernels.cuh -- sm_103a kernels of the graph traversals (paper Eq.
// graph-actions and Sec. 2.4).
//
// Records of one output form a contiguous CSR segment (Sec. 2.2, records
// grouped by output).  One warp (or a fixed group of its lanes) owns a
// segment: its lanes stream the packed 8-byte records with coalesced loads,
// multiply the exact factor by the gathered coefficients, and the partial
// sums meet in a warp-shuffle reduction.  Nothing is scattered and nothing
// uses atomics, so every result is bitwise reproducible.
#pragma once
#include <cstdint>

#include "pdl.cuh"

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

// Sub-warp rows: LANES lanes share one CSR segment (32 / LANES segments per
// warp).  Short segments waste fewer lanes and the closing shuffle reduction
// costs log2(LANES) FP64 adds per operand instead of 5.
template <int LANES>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Generator stage: xi[a] = sum_e alpha_e h[i_e] h[j_e]   (Eq. graph-actions, line 1)
// over the rows of the calling grid (ws/sg: the factor tables in shared memory)
template <bool UNIFORM, int LANES>
__device__ __forceinline__ void gen_rows(const uint64_t *__restrict__ rp, const uint2 *__restrict__ rec,
                                         const Weights &wt, const double *__restrict__ h,
                                         double *__restrict__ xi, int64_t rows, const double *ws,
                                         const unsigned long long *sg) {
    constexpr int RPW = 32 / LANES;
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
#define TERM(q)                                                                   \
    (UNIFORM ? signed_by(h[(q).x & kIdx], sg[(q).x >> 24]) * h[(q).y]             \
             : ws[(q).x >> 24] * h[(q).x & kIdx] * h[(q).y])
            uint64_t p = rp[r] + sl;
            for (; p + LANES < e; p += 2 * LANES) {
                const uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + LANES);
                acc += TERM(q0);
                acc += TERM(q1);
            }
            if (p < e) {
                const uint2 q = __ldcs(rec + p);
                acc += TERM(q);
            }
#undef TERM
        }
        acc = group_sum<LANES>(acc);
        if (sl == 0 && r < rows) xi[r] = UNIFORM ? acc * wt.mag : acc;
    }
}

template <bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) gen_stage(const uint64_t *__restrict__ rp,
                                                    const uint2 *__restrict__ rec, Weights wt,
                                                    const double *__restrict__ h,
                                                    double *__restrict__ xi, int64_t rows,
                                                    const int *done) {
    pdl_enter();
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    gen_rows<UNIFORM, LANES>(rp, rec, wt, h, xi, rows, ws, sg);
}

template <int NOPS>
struct Ops {
    const double *x[NOPS];
    double *dx[NOPS];
};

// Commutator stage: dx_o[k] = sum_e beta_e xi[a_e] x_o[j_e]  (Eq. graph-actions,
// line 2) for NOPS operands at once: one record read serves every operand.
template <int NOPS, bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) comm_stage(const uint64_t *__restrict__ rp,
                                                     const uint2 *__restrict__ rec, Weights wt,
                                                     const double *__restrict__ xi, Ops<NOPS> ops,
                                                     int64_t rows, const int *done) {
    pdl_enter();
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
#define COEF(q) (UNIFORM ? signed_by(xi[(q).x & kIdx], sg[(q).x >> 24]) : ws[(q).x >> 24] * xi[(q).x & kIdx])
            uint64_t p = rp[r] + sl;
            // several records per lane per step, every load issued before the
            // arithmetic: the gathers are L2 round trips, the FMAs are not
            constexpr int U = NOPS <= 4 ? 4 : 2;
            for (; p + (U - 1) * LANES < e; p += U * LANES) {
                uint2 q[U];
#pragma unroll
                for (int u = 0; u < U; u++) q[u] = __ldcs(rec + p + u * LANES);
                double c[U], xv[U][NOPS];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    c[u] = COEF(q[u]);
#pragma unroll
                    for (int o = 0; o < NOPS; o++) xv[u][o] = ops.x[o][q[u].y];
                }
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int o = 0; o < NOPS; o++) acc[o] += c[u] * xv[u][o];
            }
            for (; p < e; p += LANES) {
                const uint2 q = __ldcs(rec + p);
                const double c = COEF(q);
#pragma unroll
                for (int o = 0; o < NOPS; o++) acc[o] += c * ops.x[o][q.y];
            }
#undef COEF
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            const double v = group_sum<LANES>(acc[o]);
            if (sl == 0 && r < rows) ops.dx[o][r] = UNIFORM ? v * wt.mag : v;
        }
    }
}

// The same stage with the (up to eight) operands of one input index stored
// together in NB = ceil(NOPS / 4) blocks of 32 bytes, X4[j][4 NB] (one
// 256-bit load per block and record instead of one load per operand).  Per
// lane and operand the records are summed in the same order with the same
// FMAs as comm_stage, so both give the same bits.
__device__ __forceinline__ void ld_quad64(const double *p, double &a, double &b, double &c, double &d) {
    asm volatile("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}

template <int NOPS, bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) comm_stage_x4(const uint64_t *__restrict__ rp,
                                                        const uint2 *__restrict__ rec, Weights wt,
                                                        const double *__restrict__ xi,
                                                        const double *__restrict__ X4, Ops<NOPS> ops,
                                                        int64_t rows, const int *done) {
    pdl_enter();
    static_assert(NOPS <= 8, "at most two packed blocks");
    constexpr int NB = (NOPS + 3) / 4;
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
#define COEF(q) (UNIFORM ? signed_by(xi[(q).x & kIdx], sg[(q).x >> 24]) : ws[(q).x >> 24] * xi[(q).x & kIdx])
            uint64_t p = rp[r] + sl;
            constexpr int U = NOPS <= 4 ? 4 : 2;   // as comm_stage
            for (; p + (U - 1) * LANES < e; p += U * LANES) {
                uint2 q[U];
#pragma unroll
                for (int u = 0; u < U; u++) q[u] = __ldcs(rec + p + u * LANES);
                double c[U], xv[U][4 * NB];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    c[u] = COEF(q[u]);
#pragma unroll
                    for (int b = 0; b < NB; b++)
                        ld_quad64(X4 + 4 * NB * (int64_t)q[u].y + 4 * b, xv[u][4 * b], xv[u][4 * b + 1],
                                  xv[u][4 * b + 2], xv[u][4 * b + 3]);
                }
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int o = 0; o < NOPS; o++) acc[o] += c[u] * xv[u][o];
            }
            // the lane's last records (fewer than U).  Rows of a 32-lane
            // stage are short (a graph of fewer than 16,384 rows; often
            // every record of a lane is here): their loads are issued
            // together, then summed in record order as one at a time would
            // be.  Long rows keep the one-at-a-time tail, which needs fewer
            // registers (6 CTAs per SM for the 8-lane FP64 stage).
            if constexpr (LANES == 32) {
                if (p < e) {
                    uint2 q[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        ok[u] = p + u * LANES < e;
                        q[u] = ok[u] ? __ldcs(rec + p + u * LANES) : make_uint2(0u, 0u);
                    }
                    double c[U], xv[U][4 * NB];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        if (!ok[u]) continue;
                        c[u] = COEF(q[u]);
#pragma unroll
                        for (int b = 0; b < NB; b++)
                            ld_quad64(X4 + 4 * NB * (int64_t)q[u].y + 4 * b, xv[u][4 * b], xv[u][4 * b + 1],
                                      xv[u][4 * b + 2], xv[u][4 * b + 3]);
                    }
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (ok[u]) {
#pragma unroll
                            for (int o = 0; o < NOPS; o++) acc[o] += c[u] * xv[u][o];
                        }
                }
            } else {
                for (; p < e; p += LANES) {
                    const uint2 q = __ldcs(rec + p);
                    const double c = COEF(q);
                    double xv[4 * NB];
#pragma unroll
                    for (int b = 0; b < NB; b++)
                        ld_quad64(X4 + 4 * NB * (int64_t)q.y + 4 * b, xv[4 * b], xv[4 * b + 1], xv[4 * b + 2],
                                  xv[4 * b + 3]);
#pragma unroll
                    for (int o = 0; o < NOPS; o++) acc[o] += c * xv[o];
                }
            }
#undef COEF
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            const double v = group_sum<LANES>(acc[o]);
            if (sl == 0 && r < rows) ops.dx[o][r] = UNIFORM ? v * wt.mag : v;
        }
    }
}

// X4[j][o] = x_o[j] for o < NOPS, blocks of 4 NB doubles per index (the
// remaining slots are never used)
template <int NOPS>
__global__ void pack_x4(Ops<NOPS> ops, int64_t n, double *__restrict__ X4, const int *done) {
    pdl_enter();
    constexpr int NB = (NOPS + 3) / 4;
    if (skip(done)) return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int o = 0; o < NOPS; o++) X4[4 * NB * j + o] = ops.x[o][j];
    }
}

// pack_x4 and gen_stage in one launch (they are independent: the generator
// reads h itself, not the packed blocks); the same values as the two.
template <int NOPS, bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) gen_pack(const uint64_t *__restrict__ rp, const uint2 *__restrict__ rec,
                                                   Weights wt, double *__restrict__ xi, int64_t rows,
                                                   Ops<NOPS> ops, int64_t n, double *__restrict__ X4,
                                                   const int *done) {
    pdl_enter();
    constexpr int NB = (NOPS + 3) / 4;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int o = 0; o < NOPS; o++) X4[4 * NB * j + o] = ops.x[o][j];
    }
    load_weights(ws, sg, wt);
    gen_rows<UNIFORM, LANES>(rp, rec, wt, ops.x[0], xi, rows, ws, sg);
}

// ---------------------------------------------------------------- double-float
// The same commutator stage with the products and sums carried as unevaluated
// pairs of FP32 numbers (hi + lo, about 48 significant bits), on the FP32
// pipes instead of the FP64 pipe.  Each product is formed with an exact
// two-product (FMA residual) plus the two cross terms; each sum with an
// exact two-sum whose error is accumulated separately.  Partial sums are
// converted to FP64 for the closing reduction.  Inputs: xi and the operands
// split into FP32 pairs, the operands interleaved as X2[j][4] (32 bytes).
__device__ __forceinline__ void df_madd(float ch, float cl, float xh, float xl, float &s, float &c) {
    const float p = __fmul_rn(ch, xh);
    const float pe = __fmaf_rn(ch, xh, -p);
    const float pl = __fmaf_rn(ch, xl, __fmaf_rn(cl, xh, pe));
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    c = __fadd_rn(c, __fadd_rn(e, pl));
    s = t;
}

// The 32-byte operand pair block of one input index in one 256-bit load
// (sm_100 and later): one L1 request per gathered record instead of two.
// The operand blocks are spread over the whole registry and rarely reused
// from L1, so they bypass L1 allocation (no_allocate), which leaves L1 to
// the generator pairs; those are reused by neighbouring records (rows are
// sorted by generator index) and kept with evict_last.  Measured on the
// 3.4e8-record stress graph: 1.77 -> 1.64 ms per launch.
__device__ __forceinline__ void ld_pairs32(const float4 *p, float4 &a, float4 &b) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ float2 ld_xi_pair(const float2 *p) {
    float2 v;
    asm volatile("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

template <int NOPS, int LANES>
__global__ void __launch_bounds__(kBlock) comm_stage_df(const uint64_t *__restrict__ rp,
                                                        const uint2 *__restrict__ rec, Weights wt,
                                                        const float2 *__restrict__ xi2,
                                                        const float4 *__restrict__ X2, Ops<NOPS> ops,
                                                        int64_t rows, const int *done) {
    pdl_enter();
    static_assert(NOPS <= 3, "three operands per interleaved pair block");
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        float s[NOPS], c[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) { s[o] = 0.0f; c[o] = 0.0f; }
        if (r < rows) {
            const uint64_t e = rp[r + 1];
            uint64_t p = rp[r] + sl;
            // four records per lane per step, all loads ahead of the
            // arithmetic (measured best with 256-bit operand loads on the
            // 3.4e8-record graph)
            constexpr int U = 4;
            for (; p + (U - 1) * LANES < e; p += U * LANES) {
                uint2 q[U];
#pragma unroll
                for (int u = 0; u < U; u++) q[u] = __ldcs(rec + p + u * LANES);
                float2 cf[U];
                float4 a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    cf[u] = ld_xi_pair(xi2 + (q[u].x & kIdx));
                    ld_pairs32(X2 + 2 * (int64_t)q[u].y, a[u], b[u]);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const unsigned int sb = (unsigned int)(sg[q[u].x >> 24] >> 32);
                    const float ch = __uint_as_float(__float_as_uint(cf[u].x) ^ sb);
                    const float cl = __uint_as_float(__float_as_uint(cf[u].y) ^ sb);
                    df_madd(ch, cl, a[u].x, a[u].y, s[0], c[0]);
                    if (NOPS > 1) df_madd(ch, cl, a[u].z, a[u].w, s[1], c[1]);
                    if (NOPS > 2) df_madd(ch, cl, b[u].x, b[u].y, s[2], c[2]);
                }
            }
            for (; p < e; p += LANES) {
                const uint2 q = __ldcs(rec + p);
                float2 cf = ld_xi_pair(xi2 + (q.x & kIdx));
                const unsigned int sb = (unsigned int)(sg[q.x >> 24] >> 32);
                cf.x = __uint_as_float(__float_as_uint(cf.x) ^ sb);
                cf.y = __uint_as_float(__float_as_uint(cf.y) ^ sb);
                float4 a, b;
                ld_pairs32(X2 + 2 * (int64_t)q.y, a, b);
                df_madd(cf.x, cf.y, a.x, a.y, s[0], c[0]);
                if (NOPS > 1) df_madd(cf.x, cf.y, a.z, a.w, s[1], c[1]);
                if (NOPS > 2) df_madd(cf.x, cf.y, b.x, b.y, s[2], c[2]);
            }
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            const double v = group_sum<LANES>((double)s[o] + (double)c[o]);
            if (sl == 0 && r < rows) ops.dx[o][r] = v * wt.mag;
        }
    }
}

// Split doubles into FP32 pairs: out[i * stride + slot] = (hi, lo)
__global__ void split_pairs(const double *__restrict__ in, int64_t len, float2 *__restrict__ out, int stride,
                            int slot, const int *done) {
    pdl_enter();
    if (skip(done)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i];
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);
        out[i * stride + slot] = make_float2(hi, lo);
    }
}

// ---------------------------------------------------------------- assembly
// Multi-operator assembly (Sec. 2.4, last paragraph): output operator m is
// the combination sum_i C[m][i] X_i(s) of transformed source operators.
// One thread per (m, k) output coefficient sums the sources in index order
// (a fixed FMA chain), so every run gives the same bits.  The sources for a
// tile of 32 coefficients are staged in shared memory once per CTA.
__global__ void __launch_bounds__(256) assemble(const double *__restrict__ X, int n_src, int64_t n,
                                                const double *__restrict__ C, int n_out,
                                                double *__restrict__ out) {
    pdl_enter();
    extern __shared__ double xs[];                     // [n_src][32]
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int kc = threadIdx.x & 31;
    for (int e = threadIdx.x; e < n_src * 32; e += blockDim.x) {
        const int i = e / 32, c = e % 32;
        xs[e] = (k0 + c < n) ? X[(int64_t)i * n + k0 + c] : 0.0;
    }
    __syncthreads();
    if (k0 + kc >= n) return;
    for (int m = threadIdx.x >> 5; m < n_out; m += blockDim.x >> 5) {
        const double *cm = C + (int64_t)m * n_src;
        double acc = 0.0;
        for (int i = 0; i < n_src; i++) acc = fma(cm[i], xs[i * 32 + kc], acc);
        out[(int64_t)m * n + k0 + kc] = acc;
    }
}

// ---------------------------------------------------------------- tangent
// Directional derivative (Sec. 2.4, Eq. directional-derivative): the product
// rule applied record by record.
//   d xi[a]   = sum alpha (dh[i] h[j] + h[i] dh[j])
//   d F_o[k]  = sum beta (d xi[a] x_o[j] + xi[a] dx_o[j])
__global__ void __launch_bounds__(kBlock) gen_jvp(const uint64_t *__restrict__ rp, const uint2 *__restrict__ rec,
                                                  Weights wt, const double *__restrict__ h,
                                                  const double *__restrict__ dh, double *__restrict__ dxi,
                                                  int64_t rows) {
    pdl_enter();
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        double acc = 0.0;
        for (uint64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            const uint2 q = __ldcs(rec + p);
            const uint32_t i = q.x & kIdx, j = q.y;
            acc += ws[q.x >> 24] * (dh[i] * h[j] + h[i] * dh[j]);
        }
        acc = warp_sum(acc);
        if (lane == 0) dxi[r] = acc;
    }
}

template <int NOPS>
struct TanOps {
    const double *x[NOPS], *dx[NOPS];
    double *out[NOPS];
};

template <int NOPS>
__global__ void __launch_bounds__(kBlock) comm_jvp(const uint64_t *__restrict__ rp, const uint2 *__restrict__ rec,
                                                   Weights wt, const double *__restrict__ xi,
                                                   const double *__restrict__ dxi, TanOps<NOPS> t, int64_t rows) {
    pdl_enter();
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); r < rows; r += nw) {
        double acc[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; o++) acc[o] = 0.0;
        for (uint64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            const uint2 q = __ldcs(rec + p);
            const double w = ws[q.x >> 24];
            const uint32_t a = q.x & kIdx, j = q.y;
            const double c = w * xi[a], dc = w * dxi[a];
#pragma unroll
            for (int o = 0; o < NOPS; o++) acc[o] += dc * t.x[o][j] + c * t.dx[o][j];
        }
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            const double v = warp_sum(acc[o]);
            if (lane == 0) t.out[o][r] = v;
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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
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

// ---------------------------------------------------------------- adjoint, packed
// The transposed passes of the reverse traversal (Sec. 2.4) in the layout of
// the forward stages: LANES lanes per row, records streamed with coalesced
// loads, uniform factors applied as sign flips, operands gathered as packed
// 32-byte blocks.  (The operand transpose x_bar_o[j] = sum beta xi[a] w_o[k]
// has the forward commutator's form and runs in comm_stage_x4 itself.)
//
// Generator adjoint from the commutator stage, rows a, records (code|k, j):
//   xi_bar[a] = sum_e beta_e sum_o W4[k][o] X4[j][o]
template <int NOPS, bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) commT_xi_x4(const uint64_t *__restrict__ rp,
                                                      const uint2 *__restrict__ rec, Weights wt,
                                                      const double *__restrict__ W4,
                                                      const double *__restrict__ X4,
                                                      double *__restrict__ xi_bar, int64_t rows) {
    pdl_enter();
    static_assert(NOPS <= 8, "at most two packed blocks");
    constexpr int NB = (NOPS + 3) / 4;
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
            for (uint64_t p = rp[r] + sl; p < e; p += LANES) {
                const uint2 q = __ldcs(rec + p);
                double wv[4 * NB], xv[4 * NB];
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    ld_quad64(W4 + 4 * NB * (int64_t)(q.x & kIdx) + 4 * b, wv[4 * b], wv[4 * b + 1], wv[4 * b + 2],
                              wv[4 * b + 3]);
                    ld_quad64(X4 + 4 * NB * (int64_t)q.y + 4 * b, xv[4 * b], xv[4 * b + 1], xv[4 * b + 2],
                              xv[4 * b + 3]);
                }
                if (UNIFORM) {
                    // the factor's sign flips the w values (integer XOR); the
                    // products then go straight into the row sum: NOPS FP64
                    // FMAs per record, the forward stage's count
                    const unsigned long long sb = sg[q.x >> 24];
#pragma unroll
                    for (int o = 0; o < NOPS; o++) acc = fma(signed_by(wv[o], sb), xv[o], acc);
                } else {
                    double d = wv[0] * xv[0];
#pragma unroll
                    for (int o = 1; o < NOPS; o++) d = fma(wv[o], xv[o], d);
                    acc = fma(ws[q.x >> 24], d, acc);
                }
            }
        }
        acc = group_sum<LANES>(acc);
        if (sl == 0 && r < rows) xi_bar[r] = UNIFORM ? acc * wt.mag : acc;
    }
}

// Input adjoint of the generator stage, rows = registry coordinates r,
// records (code|a, partner) (both inputs of every generator record):
//   h_bar[r] = x0_bar[r] + sum_e alpha_e xi_bar[a] h[partner]
template <bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) genT_lanes(const uint64_t *__restrict__ rp,
                                                     const uint2 *__restrict__ rec, Weights wt,
                                                     const double *__restrict__ xi_bar,
                                                     const double *__restrict__ h,
                                                     const double *__restrict__ x0_bar,
                                                     double *__restrict__ h_bar, int64_t rows) {
    pdl_enter();
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    load_weights(ws, sg, wt);
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
            for (uint64_t p = rp[r] + sl; p < e; p += LANES) {
                const uint2 q = __ldcs(rec + p);
                const double c = xi_bar[q.x & kIdx];
                acc += UNIFORM ? signed_by(c, sg[q.x >> 24]) * h[q.y] : ws[q.x >> 24] * c * h[q.y];
            }
        }
        acc = group_sum<LANES>(acc);
        if (sl == 0 && r < rows) h_bar[r] = (x0_bar ? x0_bar[r] : 0.0) + (UNIFORM ? acc * wt.mag : acc);
    }
}

// Rows split into pieces: out_o[r] = add[r] (operand 0, if given) + the
// piece sums in_o[v] for v = vr[r] .. vr[r+1]-1, added in piece order.  One
// thread per (operand, row); neighbouring threads take neighbouring rows of
// one operand, so their pieces and outputs are neighbours in memory.
__global__ void piece_reduce(const uint64_t *__restrict__ vr, int64_t rows, Ops<8> io, int nops,
                             const double *__restrict__ add) {
    pdl_enter();
    const int64_t total = rows * nops;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t / rows);
        const int64_t r = t - (int64_t)o * rows;
        const uint64_t v0 = vr[r], v1 = vr[r + 1];
        const double *__restrict__ in = io.x[o];
        double acc = in[v0];
#pragma unroll 4
        for (uint64_t v = v0 + 1; v < v1; v++) acc += in[v];
        io.dx[o][r] = (add && o == 0) ? add[r] + acc : acc;
    }
}

// ---------------------------------------------------------------- fused stage
// One Runge-Kutta stage's input and generator in one launch (flows):
//   U = base + sum_s (c_s ds) K_s   (the rk_combine arithmetic), written in
//        the packed operand blocks X4[k][4 NB] the commutator stage reads
//        (and in full to U_full when the caller keeps it);
//   xi[a] = sum alpha U_0[i] U_0[j]   (gen_stage), the U values it needs
//        formed on the fly with the same arithmetic, so no block waits for
//        another's writes.
// The values are those of rk_combine + pack_x4 + gen_stage bit for bit.
struct StageIn {
    const double *base;
    const double *K[7];
    double c[7];
    int nk;
    const double *ds_ptr;   // ds from the control block, or
    double ds_const;
};

__device__ __forceinline__ double stage_u(const StageIn &si, double ds, int64_t e) {
    double v = si.base[e];
    for (int s = 0; s < si.nk; s++) v += (si.c[s] * ds) * si.K[s][e];
    return v;
}

template <int NOPS, bool UNIFORM, int LANES>
__global__ void __launch_bounds__(kBlock) stage_gen(StageIn si, int64_t n, double *__restrict__ X4,
                                                    double *__restrict__ U_full, const uint64_t *__restrict__ rp,
                                                    const uint2 *__restrict__ rec, Weights wt,
                                                    double *__restrict__ xi, int64_t rows, const int *done) {
    pdl_enter();
    constexpr int NB = (NOPS + 3) / 4;
    constexpr int RPW = 32 / LANES;
    __shared__ double ws[256];
    __shared__ unsigned long long sg[256];
    if (skip(done)) return;
    load_weights(ws, sg, wt);
    const double ds = si.ds_ptr ? *si.ds_ptr : si.ds_const;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int o = 0; o < NOPS; o++) {
            const double u = stage_u(si, ds, o * n + k);
            X4[4 * NB * k + o] = u;
            if (U_full) U_full[o * n + k] = u;
        }
    }
    const int lane = threadIdx.x & 31, sub = lane / LANES, sl = lane % LANES;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t rg = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); rg * RPW < rows; rg += nw) {
        const int64_t r = rg * RPW + sub;
        double acc = 0.0;
        if (r < rows) {
            const uint64_t e = rp[r + 1];
#define UAT(idx) stage_u(si, ds, (int64_t)(idx))
#define TERM(q)                                                                   \
    (UNIFORM ? signed_by(UAT((q).x & kIdx), sg[(q).x >> 24]) * UAT((q).y)         \
             : ws[(q).x >> 24] * UAT((q).x & kIdx) * UAT((q).y))
            uint64_t p = rp[r] + sl;
            for (; p + LANES < e; p += 2 * LANES) {
                const uint2 q0 = __ldcs(rec + p), q1 = __ldcs(rec + p + LANES);
                acc += TERM(q0);
                acc += TERM(q1);
            }
            if (p < e) {
                const uint2 q = __ldcs(rec + p);
                acc += TERM(q);
            }
#undef TERM
#undef UAT
        }
        acc = group_sum<LANES>(acc);
        if (sl == 0 && r < rows) xi[r] = UNIFORM ? acc * wt.mag : acc;
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
    pdl_enter();
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
