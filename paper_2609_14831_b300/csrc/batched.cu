// batched.cu -- many coefficient sets through one graph (paper Sec. 1 and 4:
// parameter ensembles reuse one compiled algebra; Eq. graph-actions applied
// to a batch of Hamiltonians).
//
// One persistent kernel integrates the whole batch.  Each CTA owns TILE
// instance slots.  A record is read once per CTA and applied to all TILE
// instances: lane = (record group g, instance b), 32/TILE records in flight
// per warp.  The stage input U and the generator xi live in shared memory
// with the instance index fastest ([row][TILE]), so the gathers of one record
// are one contiguous shared-memory access per group.  The RK state Y, Y5 and
// the error control are FP64 (per instance, in the CTA's global workspace);
// records, products and sums run in the compute type T (float or double).
// A slot whose instance finishes is refilled from a global queue (active-set
// compaction): no host round trip and no grid-wide barrier anywhere.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "alloc.h"
#include "cut.h"
#include "status.h"

namespace cut {
namespace kb {

constexpr uint32_t kIdx = (1u << 24) - 1;
constexpr int kThreads = 512;   // 16 warps share one CTA's shared-memory tile
constexpr int kWarps = kThreads / 32;

struct Tableau {
    int stages;       // RHS evaluations per step (RK4: 4; DP45: 7 incl. FSAL stage)
    double a[7][7];
    double b[7];      // solution weights
    double e[7];      // error weights (b - b*)
    int adaptive;
};

struct Args {
    const uint64_t *rp0, *rp1;
    const uint2 *rec0, *rec1;
    const double *wtab;
    int n_codes;
    int signs;                  // factors are +-mag with codes < 32: signs from negmask, no table
    uint32_t negmask;
    double mag;
    int64_t n, n_g;
    int nops, B;
    int slots;                  // instance slots used per CTA (<= TILE)
    double *H, *X;              // user state, instance-major, in/out
    int *steps_out, *status_out;
    int *queue;                 // next instance to start
    double *ws;                 // per-CTA workspace
    int64_t ws_stride;          // bytes per CTA
    double s0, s1, ds0, rtol, atol;
    long long max_steps;        // attempts per instance
    long long probe_attempts;   // > 0: stop every CTA after that many attempts (autotuning)
    double *record;             // [B][record_cap] accepted step sizes of each instance, or null
    long long record_cap;
    Tableau tb;
};

// v with its sign flipped when neg is 1 (an integer XOR, no multiply)
__device__ __forceinline__ float flip_if(float v, uint32_t neg) { return __uint_as_float(__float_as_uint(v) ^ (neg << 31)); }
__device__ __forceinline__ double flip_if(double v, uint32_t neg) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

// Operand values of one (index, slot) pair are stored together,
// [index][slot][P] with P >= NOPS: FP32 with three operands is padded to
// four so that one 16-byte shared-memory load fetches them (one wavefront
// per lane group, no bank conflicts inside a group).
template <typename T, int NOPS>
struct OpPad {
    static constexpr int P = (sizeof(T) == 4 && NOPS == 3) ? 4 : NOPS;
};

template <int NOPS, int P>
__device__ __forceinline__ void load_ops(const float *p, float (&v)[NOPS]) {
    if constexpr (P == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x;
        if constexpr (NOPS > 1) v[1] = t.y;
        if constexpr (NOPS > 2) v[2] = t.z;
        if constexpr (NOPS > 3) v[3] = t.w;
    } else if constexpr (P == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x;
        if constexpr (NOPS > 1) v[1] = t.y;
    } else {
#pragma unroll
        for (int o = 0; o < NOPS; o++) v[o] = p[o];
    }
}
template <int NOPS, int P>
__device__ __forceinline__ void load_ops(const double *p, double (&v)[NOPS]) {
#pragma unroll
    for (int o = 0; o < NOPS; o++) v[o] = p[o];
}

// first row index in [0, rows] whose offset is >= target (rps[rows] >= target)
__device__ __forceinline__ int64_t lower_row(const uint32_t *rps, int64_t rows, uint32_t target) {
    int64_t lo = 0, hi = rows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rps[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Row sums of one CSR stage (Eq. graph-actions) for the TILE slots of a CTA.
// The 32/TILE lane groups of all warps (NG groups) each own a contiguous
// range of rows holding about 1/NG of the records, rounded to whole rows, so
// a group's records form one contiguous stream.  The TILE lanes of a group
// (one instance each) load TILE consecutive records per instruction, M
// instructions per chunk, the next chunk in flight while the current one is
// applied; records reach the group's lanes by width-TILE shuffles.  Every
// lane sums whole rows itself in record order: no cross-lane reduction.
//   GEN:  out[r][b] = sum alpha U0[i][b] U0[j][b]            (xi, shared memory)
//   else: out[o][r][b] = sum beta xi[a][b] U_o[j][b]         (slopes, global)
// v with its sign bit flipped by the sign bit of mask (bit 31)
__device__ __forceinline__ float flip_by(float v, uint32_t mask) { return __uint_as_float(__float_as_uint(v) ^ mask); }
__device__ __forceinline__ double flip_by(double v, uint32_t mask) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)mask << 32));
}

// SIGNS: every factor is +-mag (codes < 32).  Then the lane that loads a
// record decodes it once for the TILE lanes that use it: x = offset of its
// first input in the gathered array (slot 0) with the factor's sign in bit
// 31, y = offset of its second input; the using lanes add their slot.
template <typename T, int TILE, int NOPS, bool GEN, bool SIGNS>
__device__ __forceinline__ void stage_stream(const uint32_t *__restrict__ rps, int64_t rows,
                                             const uint2 *__restrict__ rec, const T *__restrict__ U,
                                             const T *__restrict__ xis, const T *__restrict__ ws, int64_t n,
                                             T *__restrict__ out, int signs, uint32_t negmask, T mag) {
    constexpr int G = 32 / TILE, NG = kWarps * G;
    constexpr int M = TILE >= 8 ? 4 : 8;          // records per lane per chunk
    constexpr int CH = M * TILE;                  // records per group per chunk
    constexpr int SB = TILE < 8 ? TILE : 8;       // records gathered before they are summed
    constexpr int NA = GEN ? 1 : NOPS;
    constexpr int P = OpPad<T, NOPS>::P;
    const int lane = threadIdx.x & 31, b = lane % TILE, g = lane / TILE;
    const int gi = (threadIdx.x >> 5) * G + g;
    const unsigned gmask = TILE == 32 ? 0xffffffffu : (((1u << TILE) - 1u) << (g * TILE));
    const uint32_t R = rps[rows];
    const int64_t ra = lower_row(rps, rows, (uint32_t)((uint64_t)R * gi / NG));
    const int64_t rb = gi + 1 == NG ? rows : lower_row(rps, rows, (uint32_t)((uint64_t)R * (gi + 1) / NG));
    const uint32_t pe = rps[rb];
    uint32_t c = rps[ra];
    int64_t cur = ra;
    uint32_t nb = ra < rb ? rps[ra + 1] : pe;     // end of the current row
    T acc[NA];
#pragma unroll
    for (int o = 0; o < NA; o++) acc[o] = T(0);
    auto flush = [&]() {
#pragma unroll
        for (int o = 0; o < NA; o++) {
            // GEN: xi[row][slot]; else slopes [row][slot][P]
            out[GEN ? cur * TILE + b : (cur * TILE + b) * P + o] = signs ? acc[o] * mag : acc[o];
            acc[o] = T(0);
        }
        cur++;
    };
    constexpr uint32_t SX = GEN ? P : 1;          // stride of the first gathered array
    auto decode = [&](uint2 q) -> uint2 {
        if constexpr (SIGNS) {
            const uint32_t neg = (negmask >> ((q.x >> 24) & 31)) & 1u;
            return make_uint2(((q.x & kIdx) * (uint32_t)TILE * SX) | (neg << 31), q.y * (uint32_t)TILE * P);
        } else {
            return q;
        }
    };
    uint2 v[M];
#pragma unroll
    for (int m = 0; m < M; m++) {
        const uint32_t idx = c + m * TILE + b;
        v[m] = decode(idx < pe ? __ldg(rec + idx) : make_uint2(0u, 0u));
    }
    for (; c < pe; c += CH) {
        uint2 nv[M];
#pragma unroll
        for (int m = 0; m < M; m++) {
            const uint32_t idx = c + CH + m * TILE + b;
            nv[m] = decode(idx < pe ? __ldg(rec + idx) : make_uint2(0u, 0u));
        }
        // one TILE-record slice at a time from v[0]; the slices rotate down
#pragma unroll 1
        for (int m = 0; m < M; m++) {
#pragma unroll
            for (int s0 = 0; s0 < TILE; s0 += SB) {
                // gather SB records (padding records read index 0: in bounds, never summed)
                T cf[SB], uv[SB][NA];
#pragma unroll
                for (int s = 0; s < SB; s++) {
                    uint2 q;
                    q.x = __shfl_sync(gmask, v[0].x, s0 + s, TILE);
                    q.y = __shfl_sync(gmask, v[0].y, s0 + s, TILE);
                    if constexpr (SIGNS) {
                        const uint32_t ix = (q.x & 0x7fffffffu) + (uint32_t)b * SX, iy = q.y + (uint32_t)b * P;
                        const T src = GEN ? U[ix] : xis[ix];
                        cf[s] = flip_by(src, q.x & 0x80000000u);
                        if constexpr (GEN) {
                            uv[s][0] = U[iy];
                        } else {
                            load_ops<NOPS, P>(U + iy, uv[s]);
                        }
                    } else {
                        const int64_t i = (int64_t)(q.x & kIdx) * TILE + b, j = (int64_t)q.y * TILE + b;
                        const uint32_t code = q.x >> 24;
                        const T src = GEN ? U[i * P] : xis[i];
                        cf[s] = signs ? flip_if(src, (negmask >> (code & 31)) & 1u) : ws[code] * src;
                        if constexpr (GEN) {
                            uv[s][0] = U[j * P];
                        } else {
                            load_ops<NOPS, P>(U + j * P, uv[s]);
                        }
                    }
                }
                // sum them in record order, closing rows at their ends; most
                // slices lie inside one row and take the branch-free path
                const uint32_t t0 = c + m * TILE + s0;
                if (t0 + SB - 1 < nb && t0 + SB - 1 < pe) {
#pragma unroll
                    for (int s = 0; s < SB; s++)
#pragma unroll
                        for (int o = 0; o < NA; o++) acc[o] += cf[s] * uv[s][o];
                } else {
#pragma unroll
                    for (int s = 0; s < SB; s++) {
                        const uint32_t t = t0 + s;
                        if (t < pe) {
                            while (t >= nb) {
                                flush();
                                nb = rps[cur + 1];
                            }
#pragma unroll
                            for (int o = 0; o < NA; o++) acc[o] += cf[s] * uv[s][o];
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k + 1 < M; k++) v[k] = v[k + 1];
        }
#pragma unroll
        for (int m = 0; m < M; m++) v[m] = nv[m];
    }
    while (cur < rb) flush();   // the last row and any empty rows after it
}

// RHS of all TILE slots: U (smem, [n][TILE][P]) -> K (global, [n][TILE][P])
template <typename T, int TILE, int NOPS>
__device__ void rhs_tile(const Args &a, const uint32_t *__restrict__ rps0, const uint32_t *__restrict__ rps1,
                         const T *__restrict__ U, T *__restrict__ xis, const T *__restrict__ ws,
                         T *__restrict__ K) {
    if (a.signs) {
        stage_stream<T, TILE, NOPS, true, true>(rps0, a.n_g, a.rec0, U, nullptr, ws, a.n, xis, 1, a.negmask, T(a.mag));
        __syncthreads();
        stage_stream<T, TILE, NOPS, false, true>(rps1, a.n, a.rec1, U, xis, ws, a.n, K, 1, a.negmask, T(a.mag));
    } else {
        stage_stream<T, TILE, NOPS, true, false>(rps0, a.n_g, a.rec0, U, nullptr, ws, a.n, xis, 0, a.negmask, T(a.mag));
        __syncthreads();
        stage_stream<T, TILE, NOPS, false, false>(rps1, a.n, a.rec1, U, xis, ws, a.n, K, 0, a.negmask, T(a.mag));
    }
}

// Every (row, slot, operand) element of the RK arrays once: a thread keeps
// one slot (kThreads is a multiple of TILE) and walks its operands; the
// padding entries (o >= NOPS) are never touched.
#define FOR_ELEMENTS(e)                                                          \
    for (int64_t kb_ = threadIdx.x; kb_ < n * TILE; kb_ += kThreads)             \
        _Pragma("unroll") for (int o_ = 0; o_ < NOPS; o_++)                      \
            if (const int64_t e = kb_ * P + o_; true)

template <typename T, int TILE, int NOPS>
__global__ void __launch_bounds__(kThreads, 1) flow_batched_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = OpPad<T, NOPS>::P;
    const int64_t n = a.n, LP = (int64_t)P * n * TILE;   // elements of one RK array
    double *red = reinterpret_cast<double *>(smem);     // [kThreads]
    T *U = reinterpret_cast<T *>(red + kThreads);       // [n][TILE][P]
    T *xis = U + LP;                                    // [n_g][TILE]
    T *ws = xis + a.n_g * TILE;                         // [256]
    uint32_t *rps0 = reinterpret_cast<uint32_t *>(ws + 256);   // [n_g + 1] record offsets
    uint32_t *rps1 = rps0 + a.n_g + 1;                         // [n + 1]
    __shared__ int inst[TILE], status[TILE], need_k1[TILE], acc_flag[TILE];
    __shared__ double s_[TILE], ds_[TILE];
    __shared__ long long steps_[TILE], attempts_[TILE];
    __shared__ int any_active, any_new;
    __shared__ long long cta_attempts;

    for (int c = threadIdx.x; c < 256; c += kThreads) ws[c] = c < a.n_codes ? T(a.wtab[c]) : T(0);
    for (int64_t r = threadIdx.x; r <= a.n_g; r += kThreads) rps0[r] = (uint32_t)a.rp0[r];
    for (int64_t r = threadIdx.x; r <= a.n; r += kThreads) rps1[r] = (uint32_t)a.rp1[r];
    // workspace of this CTA: Y, Y5 (double) then K[7] (T), all [NOPS][n][TILE]
    double *Y = reinterpret_cast<double *>(reinterpret_cast<char *>(a.ws) + (int64_t)blockIdx.x * a.ws_stride);
    double *Y5 = Y + LP;
    T *Kb = reinterpret_cast<T *>(Y5 + LP);
    auto Kst = [&](int s) { return Kb + (int64_t)s * LP; };
    T *Yf = Kst(8);   // FP32 path: the state rounded to FP32 (stage inputs are formed in FP32)
    if (threadIdx.x < TILE) { inst[threadIdx.x] = -1; status[threadIdx.x] = 0; }
    if (threadIdx.x == 0) cta_attempts = 0;
    __syncthreads();
    const Tableau &tb = a.tb;
    const int S = tb.stages;
    const int mb = threadIdx.x % TILE;   // every element this thread touches belongs to slot mb

    for (;;) {
        // ---- refill idle slots from the queue
        if (threadIdx.x < TILE) {
            const int t = threadIdx.x;
            need_k1[t] = 0;
            if (inst[t] == -1 && t >= a.slots) {
                inst[t] = -2;   // slot not used at this CTA count
            } else if (inst[t] == -1) {
                int b = atomicAdd(a.queue, 1);
                if (b < a.B) {
                    inst[t] = b;
                    s_[t] = a.s0;
                    ds_[t] = tb.adaptive ? fmin(a.ds0, a.s1 - a.s0) : a.ds0;
                    steps_[t] = 0;
                    attempts_[t] = 0;
                    status[t] = 0;
                    need_k1[t] = 1;
                } else {
                    inst[t] = -2;   // queue exhausted
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int act = 0, nw = 0;
            for (int t = 0; t < TILE; t++) { act |= inst[t] >= 0; nw |= need_k1[t]; }
            any_active = act && !(a.probe_attempts > 0 && cta_attempts >= a.probe_attempts);
            any_new = nw;
        }
        // load the initial state of new instances
        FOR_ELEMENTS(e) {
            const int b = (int)(kb_ % TILE);
            if (!need_k1[b]) continue;
            const int64_t o = o_, k = kb_ / TILE;
            const int64_t i = inst[b];
            const double y0 = o == 0 ? a.H[i * n + k] : a.X[(i * (NOPS - 1) + (o - 1)) * n + k];
            Y[e] = y0;
            if (sizeof(T) == 4) Yf[e] = T(y0);
        }
        __syncthreads();
        if (!any_active) break;
        if (threadIdx.x == 0) cta_attempts++;

        // ---- stages
        for (int st = 0; st < S; st++) {
            const bool fsal_first = tb.adaptive && st == 0;
            if (fsal_first && !any_new) continue;       // K1 = f(Y) carried over (FSAL)
            // U = Y + ds sum_j a[st][j] K_j, rounded to T into shared memory.
            // FP32 slopes: the stage inputs are formed in FP32 from the FP32
            // copy of the state (they are rounded to FP32 anyway); only the
            // candidate state Y5 (last DP45 stage) is formed in FP64, with one
            // FP64 FMA.  FP64 slopes: all in FP64.
            const double ds = ds_[mb];
            const float dsf = (float)ds;
            float af[7];
#pragma unroll
            for (int j = 0; j < 7; j++) af[j] = (float)tb.a[st][j];
            const bool y5_stage = tb.adaptive && st == S - 1;
            FOR_ELEMENTS(e) {
                double u;
                if (sizeof(T) == 4) {
                    float inc = 0.0f;
#pragma unroll
                    for (int j = 0; j < 7; j++)
                        if (j < st && af[j] != 0.0f) inc = fmaf(af[j], (float)Kst(j)[e], inc);
                    if (!y5_stage) {
                        U[e] = T(fmaf(dsf, inc, (float)Yf[e]));
                        continue;
                    }
                    u = fma(ds, (double)inc, Y[e]);
                } else {
                    u = Y[e];
#pragma unroll
                    for (int j = 0; j < 7; j++)
                        if (j < st && tb.a[st][j] != 0.0) u += (tb.a[st][j] * ds) * (double)Kst(j)[e];
                }
                if (y5_stage) Y5[e] = u;
                U[e] = T(u);
            }
            __syncthreads();
            rhs_tile<T, TILE, NOPS>(a, rps0, rps1, U, xis, ws, fsal_first ? Kst(S) : Kst(st));
            __syncthreads();
            if (fsal_first) {   // only the new slots take the fresh K1
                FOR_ELEMENTS(e) {
                    if (need_k1[mb]) Kst(0)[e] = Kst(S)[e];
                }
                __syncthreads();
            }
        }
        // ---- error ratio per slot (adaptive) or the fixed-step update
        {
            double m = 0.0;
            bool bad = false;
            FOR_ELEMENTS(e) {
                const double ds = ds_[mb];
                if (tb.adaptive) {
                    double r;
                    if (sizeof(T) == 4) {   // error ratio in FP32 from FP32 slopes
                        float err = 0.0f;
#pragma unroll
                        for (int j = 0; j < 7; j++)
                            if (j < S && tb.e[j] != 0.0) err = fmaf((float)tb.e[j], (float)Kst(j)[e], err);
                        // U holds the last stage input, FP32(Y5)
                        const float sc = (float)a.atol + (float)a.rtol * fmaxf(fabsf((float)Yf[e]), fabsf((float)U[e]));
                        r = (double)(fabsf((float)ds * err) / sc);
                    } else {
                        double err = 0.0;
#pragma unroll
                        for (int j = 0; j < 7; j++)
                            if (j < S && tb.e[j] != 0.0) err += (ds * tb.e[j]) * (double)Kst(j)[e];
                        const double sc = a.atol + a.rtol * fmax(fabs(Y[e]), fabs(Y5[e]));
                        r = fabs(err) / sc;
                    }
                    if (!(r == r) || !isfinite(sizeof(T) == 4 ? (double)U[e] : Y5[e])) bad = true;
                    else m = fmax(m, r);
                } else {
                    double y;
                    if (sizeof(T) == 4) {
                        float inc = 0.0f;
#pragma unroll
                        for (int j = 0; j < 7; j++)
                            if (j < S && tb.b[j] != 0.0) inc = fmaf((float)tb.b[j], (float)Kst(j)[e], inc);
                        y = fma(ds, (double)inc, Y[e]);
                    } else {
                        y = Y[e];
#pragma unroll
                        for (int j = 0; j < 7; j++)
                            if (j < S && tb.b[j] != 0.0) y += (tb.b[j] * ds) * (double)Kst(j)[e];
                    }
                    Y5[e] = y;
                    if (!isfinite(y)) bad = true;
                }
            }
            red[threadIdx.x] = bad ? NAN : m;
        }
        __syncthreads();
        // ---- per-slot control (one thread per slot)
        if (threadIdx.x < TILE) {
            const int t = threadIdx.x;
            acc_flag[t] = 0;
            if (inst[t] >= 0) {
                double r = 0.0;
                bool bad = false;
                for (int q = t; q < kThreads; q += TILE) {
                    double v = red[q];
                    if (!(v == v)) bad = true;
                    else r = fmax(r, v);
                }
                attempts_[t]++;
                int done = 0;
                if (bad) {
                    status[t] = CUT_ERR_NONFINITE;
                    done = 1;
                } else if (!tb.adaptive) {
                    if (a.record && steps_[t] < a.record_cap) a.record[inst[t] * a.record_cap + steps_[t]] = ds_[t];
                    acc_flag[t] = 1;
                    steps_[t]++;
                    s_[t] = a.s0 + (double)steps_[t] * ds_[t];
                    if (steps_[t] >= a.max_steps) done = 1;
                } else {
                    const int accept = r <= 1.0;
                    double fac;
                    if (accept) fac = r == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(r, -0.2)));
                    else fac = fmin(1.0, fmax(0.2, 0.9 * pow(r, -0.2)));
                    if (accept) {
                        if (a.record && steps_[t] < a.record_cap) a.record[inst[t] * a.record_cap + steps_[t]] = ds_[t];
                        s_[t] += ds_[t];
                        steps_[t]++;
                        acc_flag[t] = 1;
                    }
                    double ds = ds_[t] * fac;
                    if (!(s_[t] < a.s1)) done = 1;
                    else {
                        ds = fmin(ds, a.s1 - s_[t]);
                        if (ds < 1e-14 * fmax(1.0, fabs(s_[t]))) { status[t] = CUT_ERR_STEP_UNDERFLOW; done = 1; }
                        else if (attempts_[t] >= a.max_steps) { status[t] = CUT_ERR_MAX_STEPS; done = 1; }
                        ds_[t] = ds;
                    }
                }
                if (done) {
                    a.steps_out[inst[t]] = (int)steps_[t];
                    a.status_out[inst[t]] = status[t];
                    acc_flag[t] |= 2;   // write back after the accept copy
                }
            }
        }
        __syncthreads();
        // ---- accept: Y <- Y5 (and K1 <- K7 under FSAL); write back finished slots
        FOR_ELEMENTS(e) {
            const int b = (int)(kb_ % TILE);
            if (acc_flag[b] & 1) {
                Y[e] = Y5[e];
                if (sizeof(T) == 4) Yf[e] = tb.adaptive ? U[e] : T(Y5[e]);
                if (tb.adaptive) Kst(0)[e] = Kst(S - 1)[e];
            }
            if (acc_flag[b] & 2) {
                const int64_t o = o_, k = kb_ / TILE;
                const int64_t i = inst[b];
                if (o == 0) a.H[i * n + k] = Y[e];
                else a.X[(i * (NOPS - 1) + (o - 1)) * n + k] = Y[e];
            }
        }
        __syncthreads();
        if (threadIdx.x < TILE && (acc_flag[threadIdx.x] & 2)) inst[threadIdx.x] = -1;
        __syncthreads();
    }
}

#undef FOR_ELEMENTS

}  // namespace kb

// ------------------------------------------------------------------ host side
struct BatchedGraphView {
    const uint64_t *rp0, *rp1;
    const uint2 *rec0, *rec1;
    const double *wtab;
    int n_codes;
    int64_t n, n_g;
    const unsigned char *sha;
    int64_t R0, R1;   // records of the two stages
    int uniform;      // every factor is +-mag
    double mag;
    uint32_t negmask; // sign of each code (codes < 32)
};

template <typename T, int TILE, int NOPS>
static size_t smem_bytes(const BatchedGraphView &v) {
    return sizeof(T) * TILE * ((size_t)kb::OpPad<T, NOPS>::P * v.n + v.n_g) + 256 * sizeof(T) +
           kb::kThreads * sizeof(double) + 4 * ((size_t)v.n + v.n_g + 2);
}

template <typename T, int TILE, int NOPS>
static size_t ws_bytes(const BatchedGraphView &v) {
    size_t L = (size_t)kb::OpPad<T, NOPS>::P * v.n * TILE;
    size_t b = L * (2 * sizeof(double) + 9 * sizeof(T));   // Y, Y5, K[8], FP32 state copy
    return (b + 255) & ~size_t(255);
}

template <typename T, int TILE, int NOPS>
static cudaError_t launch_tile(const BatchedGraphView &v, kb::Args args, int max_ctas, cudaStream_t s,
                               void **ws_base, size_t *ws_cap, int *ctas_out) {
    size_t sm = smem_bytes<T, TILE, NOPS>(v);
    auto kern = kb::flow_batched_kernel<T, TILE, NOPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kb::kThreads, sm);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    // slots per CTA: the fewest that still put the whole batch in flight on
    // every resident CTA (1024 instances, 148 SMs, TILE 8 -> 7 slots x 147 CTAs)
    const int64_t resident = (int64_t)nsm * per;
    int slots = (int)std::min<int64_t>(TILE, (args.B + resident - 1) / resident);
    if (slots < 1) slots = 1;
    args.slots = slots;
    int ctas = (int)std::min<int64_t>((args.B + slots - 1) / slots, resident);
    if (max_ctas > 0) ctas = std::min(ctas, max_ctas);
    size_t need = ws_bytes<T, TILE, NOPS>(v) * ctas;
    if (need > *ws_cap) {
        if (*ws_base) cudaFreeAsync(*ws_base, s);
        e = cut::scratch_alloc(ws_base, need, s);
        if (e != cudaSuccess) return e;
        *ws_cap = need;
    }
    args.ws = (double *)*ws_base;
    args.ws_stride = (int64_t)ws_bytes<T, TILE, NOPS>(v);
    if (ctas_out) *ctas_out = (int)std::min<int64_t>(args.B, (int64_t)ctas * slots);   // instances in flight
    kern<<<ctas, kb::kThreads, sm, s>>>(args);
    return cudaGetLastError();
}

typedef cudaError_t (*LaunchFn)(const BatchedGraphView &, kb::Args, int, cudaStream_t, void **, size_t *, int *);

template <typename T, int NOPS>
static LaunchFn pick(int tile) {
    switch (tile) {
        case 2: return launch_tile<T, 2, NOPS>;
        case 4: return launch_tile<T, 4, NOPS>;
        case 8: return launch_tile<T, 8, NOPS>;
        case 16: return launch_tile<T, 16, NOPS>;
        case 32: return launch_tile<T, 32, NOPS>;
    }
    return nullptr;
}

static LaunchFn pick_any(bool fp32, int nops, int tile) {
    if (fp32) {
        switch (nops) {
            case 1: return pick<float, 1>(tile);
            case 2: return pick<float, 2>(tile);
            case 3: return pick<float, 3>(tile);
            case 4: return pick<float, 4>(tile);
        }
    } else {
        switch (nops) {
            case 1: return pick<double, 1>(tile);
            case 2: return pick<double, 2>(tile);
            case 3: return pick<double, 3>(tile);
            case 4: return pick<double, 4>(tile);
        }
    }
    return nullptr;
}

static size_t smem_for(bool fp32, int nops, int tile, const BatchedGraphView &v) {
    size_t e = fp32 ? 4 : 8;
    const size_t P = (fp32 && nops == 3) ? 4 : (size_t)nops;   // kb::OpPad
    return e * tile * (P * v.n + v.n_g) + 256 * e + kb::kThreads * 8 + 4 * ((size_t)v.n + v.n_g + 2);  // matches smem_bytes
}

static kb::Tableau make_tableau(int method) {
    kb::Tableau t;
    memset(&t, 0, sizeof(t));
    if (method == CUT_RK4) {
        t.stages = 4;
        t.adaptive = 0;
        t.a[1][0] = 0.5;
        t.a[2][1] = 0.5;
        t.a[3][2] = 1.0;
        t.b[0] = 1.0 / 6; t.b[1] = 1.0 / 3; t.b[2] = 1.0 / 3; t.b[3] = 1.0 / 6;
        return t;
    }
    // Dormand & Prince (1980) 5(4); stage 7 is evaluated at Y5 (FSAL)
    static const double A[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {1.0 / 5, 0, 0, 0, 0, 0},
        {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
        {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
        {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
        {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
        {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
    static const double Bv[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
    static const double Bs[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                                 187.0 / 2100, 1.0 / 40};
    t.stages = 7;
    t.adaptive = 1;
    for (int i = 0; i < 7; i++) {
        for (int j = 0; j < 6; j++) t.a[i][j] = A[i][j];
        t.b[i] = Bv[i];
        t.e[i] = Bv[i] - Bs[i];
    }
    return t;
}

// Tile width chosen per (graph, batch, operands, precision, method, GPU) by
// timing a two-attempt probe of every width that fits in shared memory.
// With CUT_TUNE_CACHE=<file> in the environment the choices persist: the
// file is read once per process (lines "<graph SHA-256, hex> <batch>
// <operands> <fp32 0|1> <method> <tile> <GPU name>"; lines that do not parse
// are skipped) and every new choice is appended, so a later process skips
// the probes.
using TuneKey = std::tuple<std::string, int, int, int, int, std::string>;
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;
static std::set<std::string> g_tune_read;   // cache files already read

static std::string hex_of(const std::string &raw) {
    static const char *d = "0123456789abcdef";
    std::string h;
    for (unsigned char c : raw) { h += d[c >> 4]; h += d[c & 15]; }
    return h;
}

static std::string gpu_name(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) { (void)cudaGetLastError(); return "unknown"; }
    return p.name;
}

// caller holds g_tune_mu
static void read_tune_file(const std::string &path) {
    if (path.empty() || !g_tune_read.insert(path).second) return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char sha[80];
        int batch, nops, fp32, method, tile, used = 0;
        if (sscanf(line, "%70s %d %d %d %d %d %n", sha, &batch, &nops, &fp32, &method, &tile, &used) != 6) continue;
        if (strlen(sha) != 64 || batch < 1 || nops < 1 || (fp32 != 0 && fp32 != 1)) continue;
        if (tile != 2 && tile != 4 && tile != 8 && tile != 16 && tile != 32) continue;
        std::string raw;
        bool ok = true;
        for (int i = 0; i < 64 && ok; i += 2) {
            unsigned v;
            ok = sscanf(sha + i, "%2x", &v) == 1;
            raw += (char)v;
        }
        std::string name(line + used);
        while (!name.empty() && (name.back() == '\n' || name.back() == '\r')) name.pop_back();
        if (ok && !name.empty()) g_tune[TuneKey(raw, batch, nops, fp32, method, name)] = tile;
    }
    fclose(f);
}

static void append_tune_file(const std::string &path, const TuneKey &k, int tile) {
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %s\n", hex_of(std::get<0>(k)).c_str(), std::get<1>(k), std::get<2>(k),
            std::get<3>(k), std::get<4>(k), tile, std::get<5>(k).c_str());
    fclose(f);
}

cut_status flow_batched_impl(const BatchedGraphView &v, int device, int batch, double *h, int n_obs, double *x,
                             int precision, const cut_flow_opts *o, int tile, int *steps_out, int *status_out,
                             cudaStream_t user, int *chosen_tile) {
    const int nops = n_obs + 1;
    const bool fp32 = precision == CUT_FP32REC_FP64STATE;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    std::vector<int> cands;
    for (int t : {2, 4, 8, 16, 32})
        if (smem_for(fp32, nops, t, v) <= (size_t)dev_smem - 1024) cands.push_back(t);
    if (cands.empty()) return set_error(CUT_ERR_UNSUPPORTED, "cut_flow_batched: registry too large for the shared-memory tile");
    if (v.R0 >= (int64_t)1 << 32 || v.R1 >= (int64_t)1 << 32)
        return set_error(CUT_ERR_UNSUPPORTED, "cut_flow_batched: more than 2^32 - 1 records in a stage");
    if (tile != 0 && std::find(cands.begin(), cands.end(), tile) == cands.end())
        return set_error(CUT_ERR_INVALID_ARG, "cut_flow_batched: tile must be one of 2,4,8,16,32 and fit in shared memory");

    kb::Args a;
    memset(&a, 0, sizeof(a));
    a.rp0 = v.rp0; a.rp1 = v.rp1; a.rec0 = v.rec0; a.rec1 = v.rec1;
    a.wtab = v.wtab; a.n_codes = v.n_codes; a.n = v.n; a.n_g = v.n_g;
    a.signs = v.uniform && v.n_codes <= 32;
    a.negmask = v.negmask;
    a.mag = v.mag;
    a.nops = nops; a.B = batch;
    a.s0 = o->s0; a.s1 = o->s1; a.rtol = o->rtol; a.atol = o->atol;
    a.tb = make_tableau(o->method);
    if (o->batch_record_steps && o->record_cap > 0) {
        a.record = o->batch_record_steps;
        a.record_cap = o->record_cap;
    }
    if (o->method == CUT_RK4) {
        int64_t N = (int64_t)llround((o->s1 - o->s0) / o->ds);
        if (N < 1) N = 1;
        a.ds0 = (o->s1 - o->s0) / (double)N;
        a.max_steps = N;
    } else {
        a.ds0 = o->ds;
        a.max_steps = o->max_steps > 0 ? o->max_steps : 1000000;
    }
    cudaStream_t s;
    cudaEvent_t ev;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
    void *ws = nullptr;
    size_t ws_cap = 0;
    int *queue = nullptr;
    cudaError_t e = cut::scratch_alloc(&queue, 256, s);
    auto finish = [&](cut_status st) {
        if (ws) cudaFreeAsync(ws, s);
        if (queue) cudaFreeAsync(queue, s);
        cudaEventRecord(ev, s);
        cudaStreamWaitEvent(user, ev, 0);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        cudaEventDestroy(ev);
        return st;
    };
    if (e != cudaSuccess) return finish(set_error(CUT_ERR_OUT_OF_MEMORY, "cut_flow_batched: queue"));
    a.queue = queue;
    a.steps_out = steps_out;
    a.status_out = status_out;

    if (tile == 0) {
        const char *cache_env = getenv("CUT_TUNE_CACHE");
        const std::string cache = cache_env ? cache_env : "";
        const TuneKey key(std::string((const char *)v.sha, 32), batch, nops, (int)fp32, o->method, gpu_name(device));
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            read_tune_file(cache);
            auto it = g_tune.find(key);
            // a remembered width that no longer fits is probed again
            if (it != g_tune.end() && std::find(cands.begin(), cands.end(), it->second) != cands.end())
                tile = it->second;
        }
        if (tile == 0) {
            // probe on scratch copies so the caller's state is untouched
            double *hc = nullptr, *xc = nullptr;
            int *so = nullptr;
            size_t hb = (size_t)batch * v.n * 8, xb = (size_t)batch * n_obs * v.n * 8;
            e = cut::scratch_alloc(&hc, hb + xb + 2 * (size_t)batch * 4 + 64, s);
            if (e != cudaSuccess) return finish(set_error(CUT_ERR_OUT_OF_MEMORY, "cut_flow_batched: autotune scratch"));
            xc = hc + (size_t)batch * v.n;
            so = (int *)(xc + (size_t)batch * n_obs * v.n);
            cudaEvent_t t0, t1;
            cudaEventCreate(&t0);
            cudaEventCreate(&t1);
            float best = 1e30f;
            for (int t : cands) {
                cudaMemcpyAsync(hc, h, hb, cudaMemcpyDeviceToDevice, s);
                if (n_obs) cudaMemcpyAsync(xc, x, xb, cudaMemcpyDeviceToDevice, s);
                cudaMemsetAsync(queue, 0, 4, s);
                kb::Args p = a;
                p.H = hc; p.X = xc; p.steps_out = so; p.status_out = so + batch;
                p.probe_attempts = 2;
                int ctas = 0;
                cudaEventRecord(t0, s);
                e = pick_any(fp32, nops, t)(v, p, 0, s, &ws, &ws_cap, &ctas);
                cudaEventRecord(t1, s);
                cudaEventSynchronize(t1);
                if (e != cudaSuccess) { cudaGetLastError(); continue; }
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                // time per instance-attempt: every resident slot ran two attempts
                const double inflight = (double)ctas;
                const float norm = (float)(ms / inflight);
                if (norm < best) { best = norm; tile = t; }
            }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            cudaFreeAsync(hc, s);
            if (tile == 0) return finish(set_error(CUT_ERR_CUDA, "cut_flow_batched: no tile width ran"));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = tile;
            append_tune_file(cache, key, tile);
        }
    }
    if (chosen_tile) *chosen_tile = tile;
    a.H = h;
    a.X = x;
    cudaMemsetAsync(queue, 0, 4, s);
    e = pick_any(fp32, nops, tile)(v, a, 0, s, &ws, &ws_cap, nullptr);
    if (e != cudaSuccess) return finish(set_error(CUT_ERR_CUDA, std::string("cut_flow_batched: ") + cudaGetErrorString(e)));
    cut_status st = finish(CUT_OK);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_flow_batched: ") + cudaGetErrorString(e));
    return st;
}

}  // namespace cut
