// mlp.cu -- the learned surrogate: an MLP n_in -> H -> H -> n_out with GELU,
// BF16 operands and FP32 accumulation on the tcgen05 tensor cores, trained by
// the library's own forward, backward and AdamW kernels.  It maps a
// Hamiltonian parameter vector to the flowed coefficients (a warm start and a
// screen; the graph flow stays the fallback and the judge of its error).
//
// Layouts (rows padded to 128, feature dimensions padded to 64 / 128):
//   W_l  bf16 [out_l][in_l]   forward B operand (C = X W^T)
//   W_l^T bf16 [in_l][out_l]  backward B operand (dX = dZ W)
//   activations bf16 [M][f] and their transposes [f][M] (dW = dZ^T X),
//   written by the GEMM epilogues directly.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "alloc.h"
#include "cut.h"
#include "status.h"
#include "trace.h"
#include "tc_gemm.cuh"

using bf16 = __nv_bfloat16;

namespace cut {
namespace mlpk {

__global__ void pack_input(const float *__restrict__ x, int batch, int n_in, int in_p, int Mp, bf16 *__restrict__ xb,
                           bf16 *__restrict__ xt) {
    pdl_enter();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Mp * in_p;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / in_p), c = (int)(e % in_p);
        const float v = (m < batch && c < n_in) ? x[(int64_t)m * n_in + c] : 0.0f;
        const bf16 b = __float2bfloat16(v);
        xb[e] = b;
        xt[(int64_t)c * Mp + m] = b;
    }
}

// dZ = 2 (Y - t_hat) / (batch n_out) on valid entries, t_hat = (T - shift -
// J x) / scale (J, x optional: the linear skip term); loss sum.  One 32 x 32
// tile of (rows, columns) per block of 32 x 8 threads: J and x slices are
// staged in shared memory, and the transposed copy of dZ is written through
// a shared tile so that every global access is coalesced.
__global__ void __launch_bounds__(256) mse_grad(const float *__restrict__ Y, int ldy, const float *__restrict__ T,
                                                int batch, int n_out, const float *__restrict__ scale,
                                                const float *__restrict__ shift, int Mp, int Np,
                                                bf16 *__restrict__ dz, bf16 *__restrict__ dzt,
                                                float *__restrict__ dz32, float *__restrict__ loss,
                                                const float *__restrict__ J, const float *__restrict__ x, int K) {
    pdl_enter();
    __shared__ float Js[32][65], Xs[32][65], Gs[32][33], red[256];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int c0 = blockIdx.x * 32, m0 = blockIdx.y * 32, c = c0 + tx;
    const float inv = 1.0f / ((float)batch * (float)n_out);
    float lin[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (J) {
        for (int k0 = 0; k0 < K; k0 += 64) {
            const int kc = min(64, K - k0);
            for (int i = tid; i < 32 * 64; i += 256) {
                const int r = i / 64, k = i % 64;
                Js[r][k] = (k < kc && c0 + r < n_out) ? J[(int64_t)(c0 + r) * K + k0 + k] : 0.0f;
                Xs[r][k] = (k < kc && m0 + r < batch) ? x[(int64_t)(m0 + r) * K + k0 + k] : 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 4; i++)
                for (int k = 0; k < kc; k++) lin[i] = fmaf(Js[tx][k], Xs[ty + 8 * i][k], lin[i]);
            __syncthreads();
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int rr = ty + 8 * i, m = m0 + rr;
        float g = 0.0f;
        if (m < batch && c < n_out) {
            const float t = (T[(int64_t)m * n_out + c] - shift[c] - lin[i]) / scale[c];
            const float r = Y[(int64_t)m * ldy + c] - t;
            acc += r * r;
            g = 2.0f * r * inv;
        }
        const int64_t e = (int64_t)m * Np + c;
        dz[e] = __float2bfloat16(g);
        dz32[e] = g;
        Gs[rr][tx] = g;
    }
    red[tid] = acc;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int cc = ty + 8 * i;   // column within the tile; lanes run along rows
        dzt[(int64_t)(c0 + cc) * Mp + m0 + tx] = __float2bfloat16(Gs[tx][cc]);
    }
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0 && loss) atomicAdd(loss, red[0] * inv);
}

// db[c] = sum_m dz[m][c] (valid rows): 32 columns per block, 32 row groups
// (a thread adds every 32nd row, its loads independent of one another)
// summed in a fixed order (coalesced rows, deterministic result)
constexpr int kColSumGroups = 32;
__global__ void __launch_bounds__(32 * kColSumGroups) col_sum(const float *__restrict__ dz, int ld, int rows, int cols,
                                                             float *__restrict__ db) {
    pdl_enter();
    __shared__ float part[kColSumGroups][33];
    const int tx = threadIdx.x, ty = threadIdx.y, c = blockIdx.x * 32 + tx;
    float s = 0.0f;
    if (c < cols) {
#pragma unroll 8
        for (int m = ty; m < rows; m += kColSumGroups) s += dz[(int64_t)m * ld + c];
    }
    part[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && c < cols) {
        float t = 0.0f;
        for (int g = 0; g < kColSumGroups; g++) t += part[g][tx];
        db[c] = t;
    }
}

// Split-K partial products: out[e] = sum_z part[z][e] in z order.
__global__ void sum_splits(const float *__restrict__ part, int splits, int64_t count, float *__restrict__ out) {
    pdl_enter();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        float t = 0.0f;
        for (int z = 0; z < splits; z++) t += part[(int64_t)z * count + e];
        out[e] = t;
    }
}

// AdamW (Loshchilov & Hutter): decoupled weight decay.  Parameters are
// [out][in] (bias: in = 1).  adamw_all updates a list of segments element by
// element (the biases); adamw_tiles the weight matrices, refreshing their
// BF16 copies W and W^T.
struct AdamSeg {
    float *w, *g, *m, *v;
    bf16 *wb, *wt;      // BF16 copies, row-major and transposed (weights only)
    int64_t count, start;
    int in_p, out_p;
    float wd;
};
struct AdamSegs {
    AdamSeg s[6];
    int n;
    int64_t total;
};

// The three weight matrices W [out_p][in_p], walked in 32 x 32 tiles.
struct AdamTiles {
    AdamSeg s[3];
    int tiles_x[3];             // tiles per row of tiles (in_p / 32)
    int64_t tile_start[4];      // first tile of each matrix; tile_start[3] = all tiles
};

// The AdamW update of a weight tile (adamw_all's arithmetic), its BF16 copy
// row-major and, through shared memory, transposed W^T [in_p][out_p]: reads
// and writes of both copies coalesced.
__global__ void __launch_bounds__(256) adamw_tiles(AdamTiles a, float lr, float b1, float b2, float eps, float bc1,
                                                   float bc2) {
    pdl_enter();
    __shared__ bf16 tile[32][34];
    for (int64_t t = blockIdx.x; t < a.tile_start[3]; t += gridDim.x) {
        const int k = t >= a.tile_start[2] ? 2 : (t >= a.tile_start[1] ? 1 : 0);
        const AdamSeg &S = a.s[k];
        const int64_t lt = t - a.tile_start[k];
        const int c0 = (int)(lt % a.tiles_x[k]) * 32, r0 = (int)(lt / a.tiles_x[k]) * 32;
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int r = r0 + j, c = c0 + threadIdx.x;
            if (r >= S.out_p || c >= S.in_p) continue;
            const int64_t e = (int64_t)r * S.in_p + c;
            const float gr = S.g[e];
            const float mm = b1 * S.m[e] + (1.0f - b1) * gr;
            const float vv = b2 * S.v[e] + (1.0f - b2) * gr * gr;
            S.m[e] = mm;
            S.v[e] = vv;
            float x = S.w[e];
            x -= lr * ((mm / bc1) / (sqrtf(vv / bc2) + eps) + S.wd * x);
            S.w[e] = x;
            const bf16 bv = __float2bfloat16(x);
            S.wb[e] = bv;
            tile[j][threadIdx.x] = bv;
        }
        __syncthreads();
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int c = c0 + j, r = r0 + threadIdx.x;
            if (r < S.out_p && c < S.in_p) S.wt[(int64_t)c * S.out_p + r] = tile[threadIdx.x][j];
        }
        __syncthreads();
    }
}

__global__ void adamw_all(AdamSegs segs, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    pdl_enter();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < segs.total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < segs.n && t >= segs.s[k + 1].start) k++;
        const AdamSeg &S = segs.s[k];
        const int64_t e = t - S.start;
        const float gr = S.g[e];
        const float mm = b1 * S.m[e] + (1.0f - b1) * gr;
        const float vv = b2 * S.v[e] + (1.0f - b2) * gr * gr;
        S.m[e] = mm;
        S.v[e] = vv;
        float x = S.w[e];
        x -= lr * ((mm / bc1) / (sqrtf(vv / bc2) + eps) + S.wd * x);
        S.w[e] = x;
    }
}

__global__ void to_bf16(const float *__restrict__ w, int64_t count, int in_p, int out_p, bf16 *__restrict__ wb,
                        bf16 *__restrict__ wt) {
    pdl_enter();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const bf16 b = __float2bfloat16(w[e]);
        wb[e] = b;
        wt[(e % in_p) * (int64_t)out_p + e / in_p] = b;
    }
}

// ---- least-squares linear part of the surrogate (FP64, on the device)
// Design matrix A[b] = (1, x[b][0..n_in)), P = n_in + 1 columns; the
// "value" columns are A's own (for the Gram matrix A^T A) followed by the
// targets (for A^T T).  partial[ch][p][c] = sum over the chunk's rows of
// A[b][p] V[b][c]; chunks are summed in order afterwards (fixed sum order).
constexpr int kFitP = 64;        // at most 63 inputs
constexpr int kFitRows = 64;     // rows staged per shared-memory tile

__device__ __forceinline__ double fit_a(const float *x, int n_in, int64_t b, int p) {
    return p == 0 ? 1.0 : (double)x[b * n_in + (p - 1)];
}

__global__ void __launch_bounds__(128) fit_gram_partials(const float *__restrict__ x, const double *__restrict__ t,
                                                         int64_t batch, int n_in, int n_out, int64_t rows_per_chunk,
                                                         double *__restrict__ partial) {
    pdl_enter();
    const int P = n_in + 1, ncol = P + n_out;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * rows_per_chunk, b1 = min(batch, b0 + rows_per_chunk);
    __shared__ double As[kFitRows][kFitP];
    double acc[kFitP];
#pragma unroll
    for (int p = 0; p < kFitP; p++) acc[p] = 0.0;
    for (int64_t r0 = b0; r0 < b1; r0 += kFitRows) {
        const int nr = (int)(b1 - r0 < kFitRows ? b1 - r0 : kFitRows);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * P; e += blockDim.x) As[e / P][e % P] = fit_a(x, n_in, r0 + e / P, e % P);
        __syncthreads();
        if (c < ncol) {
            for (int r = 0; r < nr; r++) {
                const double v = c < P ? As[r][c] : t[(r0 + r) * n_out + (c - P)];
#pragma unroll
                for (int p = 0; p < kFitP; p++)
                    if (p < P) acc[p] = fma(As[r][p], v, acc[p]);
            }
        }
    }
    if (c < ncol)
        for (int p = 0; p < P; p++) partial[((int64_t)blockIdx.y * P + p) * ncol + c] = acc[p];
}

// M[p][c] = sum_ch partial[ch][p][c] (chunk order)
__global__ void fit_reduce(const double *__restrict__ partial, int chunks, int64_t len, double *__restrict__ M) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int ch = 0; ch < chunks; ch++) s += partial[ch * len + i];
        M[i] = s;
    }
}

// Cholesky of G = M[:, 0:P] + ridge I (thread 0), then each thread solves
// G coef[:, o] = M[:, P + o] for its outputs; coef[P][n_out].
__global__ void __launch_bounds__(256) fit_solve(const double *__restrict__ M, int n_in, int n_out, double ridge,
                                                 double *__restrict__ coef, int *__restrict__ bad) {
    pdl_enter();
    const int P = n_in + 1, ncol = P + n_out;
    __shared__ double Lm[kFitP][kFitP];
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        for (int i = 0; i < P; i++)
            for (int j = 0; j <= i; j++) {
                double v = M[i * ncol + j] + (i == j ? ridge : 0.0);
                for (int k2 = 0; k2 < j; k2++) v -= Lm[i][k2] * Lm[j][k2];
                if (i == j) {
                    if (!(v > 0.0)) { ok = 0; v = 1.0; }
                    Lm[i][i] = sqrt(v);
                } else {
                    Lm[i][j] = v / Lm[j][j];
                }
            }
        if (!ok && bad) *bad = 1;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        double y[kFitP];
        for (int i = 0; i < P; i++) {           // L y = rhs
            double v = M[i * ncol + P + o];
            for (int k2 = 0; k2 < i; k2++) v -= Lm[i][k2] * y[k2];
            y[i] = v / Lm[i][i];
        }
        for (int i = P - 1; i >= 0; i--) {      // L^T z = y
            double v = y[i];
            for (int k2 = i + 1; k2 < P; k2++) v -= Lm[k2][i] * y[k2];
            y[i] = v / Lm[i][i];
        }
        for (int i = 0; i < P; i++) coef[(int64_t)i * n_out + o] = y[i];
    }
}

// partial[ch][o] = sum over the chunk of (t[b][o] - A[b] . coef[:, o])^2
__global__ void __launch_bounds__(128) fit_resid_partials(const float *__restrict__ x, const double *__restrict__ t,
                                                          const double *__restrict__ coef, int64_t batch, int n_in,
                                                          int n_out, int64_t rows_per_chunk,
                                                          double *__restrict__ partial) {
    pdl_enter();
    const int P = n_in + 1;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * rows_per_chunk, b1 = min(batch, b0 + rows_per_chunk);
    if (o >= n_out) return;
    double cf[kFitP];
    for (int p = 0; p < P; p++) cf[p] = coef[(int64_t)p * n_out + o];
    double acc = 0.0;
    for (int64_t b = b0; b < b1; b++) {
        double r = t[b * n_out + o] - cf[0];
        for (int p = 1; p < P; p++) r -= cf[p] * (double)x[b * n_in + (p - 1)];
        acc = fma(r, r, acc);
    }
    partial[(int64_t)blockIdx.y * n_out + o] = acc;
}

// shift = intercept, J[o][i] = slope, scale = residual RMS / sqrt(weight)
__global__ void fit_write(const double *__restrict__ coef, const double *__restrict__ ss, const float *__restrict__ w,
                          int64_t batch, int n_in, int n_out, float *__restrict__ scale, float *__restrict__ shift,
                          float *__restrict__ J) {
    pdl_enter();
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
        shift[o] = (float)coef[o];
        for (int i = 0; i < n_in; i++) J[(int64_t)o * n_in + i] = (float)coef[(int64_t)(1 + i) * n_out + o];
        const double rms = sqrt(ss[o] / (double)(batch > 1 ? batch : 1));
        scale[o] = (float)(fmax(rms, 1e-9) / sqrt((double)(w ? w[o] : 1.0f)));
    }
}

// ---- ensemble statistics of K surrogate networks (the gate's error signal)
struct Members {
    const float *p[16];
};

// One CTA per query row: mean[b][o] = (1/K) sum_k p_k[b][o] (members in
// order) and spread[b] = max over the masked outputs of max_k - min_k.
__global__ void __launch_bounds__(256) ensemble_stats(Members m, int K, int n_out, const uint8_t *__restrict__ mask,
                                                      float *__restrict__ mean, float *__restrict__ spread) {
    pdl_enter();
    __shared__ float red[256];
    const int64_t b = blockIdx.x;
    float sp = 0.0f;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        float sum = 0.0f, lo = 3.0e38f, hi = -3.0e38f;
        for (int k = 0; k < K; k++) {
            const float v = m.p[k][b * n_out + o];
            sum += v;
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        if (mean) mean[b * n_out + o] = sum / (float)K;
        if (mask[o]) sp = fmaxf(sp, hi - lo);
    }
    red[threadIdx.x] = sp;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) spread[b] = red[0];
}

}  // namespace mlpk

static int pad_to(int v, int q) { return (v + q - 1) / q * q; }

// The tensor-map encoder is a driver entry point; it is fetched through the
// runtime so that the library loads on machines without a driver.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static cut_status make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(CUT_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(CUT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return CUT_OK;
}

// SMs of the current device (148 on B300), read once per device.
static int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 148;
    }
    return cache[dev];
}

// C[M][N] = A[M][K] B[N][K]^T, M % 128 == 0, N % 64 == 0, K % (64 splits) == 0.
// splits > 1: split k, partial products to ep.out_f32 + z ep.split_stride.
static cut_status gemm(const bf16 *A, const bf16 *B, int M, int N, int K, tc::Epi ep, cudaStream_t s,
                       int splits = 1, bool gelu = false) {
    if (M % 128 || N % 64 || splits < 1 || K % (64 * splits)) return set_error(CUT_ERR_INVALID_ARG, "gemm: shape not padded");
    if (M / 128 > 65535) return set_error(CUT_ERR_INVALID_ARG, "gemm: more than 65535 row tiles (batch above 8,388,480)");
    CUtensorMap ma, mb;
    const int bn = (N % 128 == 0) ? 128 : 64;
    cut_status st = make_map(&ma, A, M, K, 128);
    if (st != CUT_OK) return st;
    st = make_map(&mb, B, N, K, bn);
    if (st != CUT_OK) return st;
    dim3 grid(N / bn, M / 128, splits);
    const int act = ep.dgelu_z ? tc::kGeluGrad : (gelu ? tc::kGelu : tc::kLinear);
    auto launch = [&](auto kern, size_t sm) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        pdl_launch(kern, grid, tc::kThreads, sm, s, ma, mb, K / splits, ep);
    };
    // at most one CTA per SM: the deep ring (one CTA per SM, more copies in flight)
    const bool deep = (int64_t)grid.x * grid.y * grid.z <= num_sms();
    constexpr int D = tc::STAGES_DEEP;
    const size_t sm128 = tc::gemm_smem_bytes<128>(), sm64 = tc::gemm_smem_bytes<64>();
    const size_t sm128d = tc::gemm_smem_bytes<128, D>(), sm64d = tc::gemm_smem_bytes<64, D>();
    if (bn == 128 && deep) {
        if (act == tc::kGelu) launch(tc::gemm_bf16_tn<128, tc::kGelu, D>, sm128d);
        else if (act == tc::kGeluGrad) launch(tc::gemm_bf16_tn<128, tc::kGeluGrad, D>, sm128d);
        else launch(tc::gemm_bf16_tn<128, tc::kLinear, D>, sm128d);
    } else if (bn == 128) {
        if (act == tc::kGelu) launch(tc::gemm_bf16_tn<128, tc::kGelu>, sm128);
        else if (act == tc::kGeluGrad) launch(tc::gemm_bf16_tn<128, tc::kGeluGrad>, sm128);
        else launch(tc::gemm_bf16_tn<128, tc::kLinear>, sm128);
    } else if (deep) {
        if (act == tc::kGelu) launch(tc::gemm_bf16_tn<64, tc::kGelu, D>, sm64d);
        else if (act == tc::kGeluGrad) launch(tc::gemm_bf16_tn<64, tc::kGeluGrad, D>, sm64d);
        else launch(tc::gemm_bf16_tn<64, tc::kLinear, D>, sm64d);
    } else {
        if (act == tc::kGelu) launch(tc::gemm_bf16_tn<64, tc::kGelu>, sm64);
        else if (act == tc::kGeluGrad) launch(tc::gemm_bf16_tn<64, tc::kGeluGrad>, sm64);
        else launch(tc::gemm_bf16_tn<64, tc::kLinear>, sm64);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return CUT_OK;
}

constexpr int kMaxSplits = 16;   // split-k factor bound of the weight-gradient GEMMs

static tc::Epi epi0(int M, int N, int *err) {
    tc::Epi e;
    memset(&e, 0, sizeof(e));
    e.alpha = 1.0f;
    e.M = M;
    e.N = N;
    e.err = err;
    e.stall = err + 1;   // err[1]: the injection flag of cut_mlp_inject_stall
    return e;
}

}  // namespace cut

using namespace cut;

struct Layer {
    int in, out, in_p, out_p;
    float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;   // fp32 master and grads
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;  // Adam moments
    bf16 *wb = nullptr, *wt = nullptr;                                 // bf16 W, W^T
};

struct cut_mlp {
    int device = 0, n_in = 0, n_hid = 0, n_out = 0;
    Layer L[3];
    float *scale = nullptr, *shift = nullptr;   // output affine (targets standardised)
    float *J = nullptr;                         // linear skip [n_out][n_in] (FP32), or null
    float *splitbuf = nullptr;                  // split-k partial weight gradients
    int *err = nullptr;
    long long t = 0;                            // Adam step
    // activations for the largest padded batch seen
    int Mcap = 0;
    bf16 *xb = nullptr, *xt = nullptr;
    float *z[3] = {nullptr, nullptr, nullptr};  // pre-activations fp32 [M][out_p]
    bf16 *hb[2] = {nullptr, nullptr}, *ht[2] = {nullptr, nullptr};
    bf16 *dzb = nullptr, *dzt = nullptr;        // scratch for the current layer's dZ
    float *dz32 = nullptr;
    bf16 *dzb2 = nullptr, *dzt2 = nullptr;
    float *dz32b = nullptr;
    std::vector<void *> allocs;
    // forward + backward captured as one CUDA graph, replayed while the call
    // keeps the same batch, buffers and skip term (captured on the second
    // consecutive call with the same key)
    struct GraphKey {
        int batch = -1, Mcap = -1;
        const void *x = nullptr, *t = nullptr, *loss = nullptr, *J = nullptr;
        bool operator==(const GraphKey &o) const {
            return batch == o.batch && Mcap == o.Mcap && x == o.x && t == o.t && loss == o.loss && J == o.J;
        }
    } gkey;
    int gseen = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
    }
    ~cut_mlp() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        drop_graph();
        if (gstream) cudaStreamDestroy(gstream);
        for (void *p : allocs) cudaFree(p);
        cudaSetDevice(cur);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
        if (e == cudaSuccess) {
            allocs.push_back(*p);
            cudaMemset(*p, 0, count * sizeof(T));
        }
        return e;
    }
};

static uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static cut_status ensure_batch(cut_mlp *m, int Mp) {
    if (Mp <= m->Mcap) return CUT_OK;
    const int H = m->L[0].out_p, O = m->L[2].out_p, I = m->L[0].in_p;
    const int F = std::max(std::max(H, O), I);
    bool ok = m->alloc(&m->xb, (size_t)Mp * I) == cudaSuccess && m->alloc(&m->xt, (size_t)Mp * I) == cudaSuccess;
    for (int l = 0; l < 3 && ok; l++) ok = m->alloc(&m->z[l], (size_t)Mp * m->L[l].out_p) == cudaSuccess;
    for (int l = 0; l < 2 && ok; l++)
        ok = m->alloc(&m->hb[l], (size_t)Mp * H) == cudaSuccess && m->alloc(&m->ht[l], (size_t)Mp * H) == cudaSuccess;
    ok = ok && m->alloc(&m->dzb, (size_t)Mp * F) == cudaSuccess && m->alloc(&m->dzt, (size_t)Mp * F) == cudaSuccess &&
         m->alloc(&m->dz32, (size_t)Mp * F) == cudaSuccess && m->alloc(&m->dzb2, (size_t)Mp * F) == cudaSuccess &&
         m->alloc(&m->dzt2, (size_t)Mp * F) == cudaSuccess && m->alloc(&m->dz32b, (size_t)Mp * F) == cudaSuccess;
    if (!ok) return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp: activation buffers");
    m->Mcap = Mp;
    return CUT_OK;
}

static int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 148 * 8)); }

// forward: Z_l, H_l (bf16 + transposes); returns the output pre-affine in z[2]
static cut_status forward(cut_mlp *m, int batch, const float *x, cudaStream_t s, const float *post_scale,
                          const float *post_shift, float *y_out) {
    const int Mp = pad_to(batch, 128);
    cut_status st = ensure_batch(m, Mp);
    if (st != CUT_OK) return st;
    pdl_launch(mlpk::pack_input, grid_of((int64_t)Mp * m->L[0].in_p), 256, 0, s, x, batch, m->n_in, m->L[0].in_p, Mp, m->xb,
                                                                          m->xt);
    const bf16 *in = m->xb;
    for (int l = 0; l < 3; l++) {
        Layer &Ly = m->L[l];
        tc::Epi e = epi0(Mp, Ly.out_p, m->err);
        e.bias = Ly.b;
        e.out_f32 = m->z[l];
        e.ld_f32 = Ly.out_p;
        if (l < 2) {
            e.out_bf16 = m->hb[l];
            e.ld_bf16 = Ly.out_p;
            e.out_t = m->ht[l];
            e.ld_t = Mp;
            if (y_out) {
                // inference: the pre-activations and the transposed
                // activations serve only the backward pass, which runs its
                // own forward pass
                e.out_f32 = nullptr;
                e.out_t = nullptr;
            }
        } else if (y_out) {
            // inference: valid region only, with the output affine and skip
            e.M = batch;
            e.N = m->n_out;
            e.post_scale = post_scale;
            e.post_shift = post_shift;
            e.lin_J = m->J;
            e.lin_x = x;
            e.lin_k = m->n_in;
            e.out_f32 = y_out;
            e.ld_f32 = m->n_out;
        }
        st = gemm(in, Ly.wb, Mp, Ly.out_p, Ly.in_p, e, s, 1, l < 2);   // GELU on the hidden layers
        if (st != CUT_OK) return st;
        if (l < 2) in = m->hb[l];
    }
    return CUT_OK;
}

extern "C" {

cut_status cut_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, int device, cut_mlp **out) {
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 65536)
        return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_create: bad sizes");
    std::unique_ptr<cut_mlp> m(new cut_mlp());
    m->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_create: bad device");
    m->n_in = n_in;
    m->n_hid = n_hidden;
    m->n_out = n_out;
    const int dims[4] = {n_in, n_hidden, n_hidden, n_out};
    uint64_t rs = seed;
    for (int l = 0; l < 3; l++) {
        Layer &Ly = m->L[l];
        Ly.in = dims[l];
        Ly.out = dims[l + 1];
        // a layer's padded input width is the previous layer's padded output
        // width, so that activation buffers chain without re-striding
        Ly.in_p = l == 0 ? pad_to(Ly.in, 64) : m->L[l - 1].out_p;
        Ly.out_p = pad_to(Ly.out, 128);
        const size_t cnt = (size_t)Ly.in_p * Ly.out_p;
        bool ok = m->alloc(&Ly.w, cnt) == cudaSuccess && m->alloc(&Ly.gw, cnt) == cudaSuccess &&
                  m->alloc(&Ly.mw, cnt) == cudaSuccess && m->alloc(&Ly.vw, cnt) == cudaSuccess &&
                  m->alloc(&Ly.b, Ly.out_p) == cudaSuccess && m->alloc(&Ly.gb, Ly.out_p) == cudaSuccess &&
                  m->alloc(&Ly.mb, Ly.out_p) == cudaSuccess && m->alloc(&Ly.vb, Ly.out_p) == cudaSuccess &&
                  m->alloc(&Ly.wb, cnt) == cudaSuccess && m->alloc(&Ly.wt, cnt) == cudaSuccess;
        if (!ok) return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_create: parameters");
        // uniform(-1/sqrt(in), 1/sqrt(in)) from a counter-based generator
        std::vector<float> hw(cnt, 0.0f);
        const float a = 1.0f / std::sqrt((float)Ly.in);
        for (int o = 0; o < Ly.out; o++)
            for (int i = 0; i < Ly.in; i++) {
                const double u = (double)(splitmix(rs) >> 11) * (1.0 / 9007199254740992.0);
                hw[(size_t)o * Ly.in_p + i] = (float)((2.0 * u - 1.0) * a);
            }
        cudaMemcpy(Ly.w, hw.data(), cnt * 4, cudaMemcpyHostToDevice);
        pdl_launch(mlpk::to_bf16, grid_of(cnt), 256, 0, 0, Ly.w, cnt, Ly.in_p, Ly.out_p, Ly.wb, Ly.wt);
    }
    size_t wmax = 0;
    for (int l = 0; l < 3; l++) wmax = std::max(wmax, (size_t)m->L[l].in_p * m->L[l].out_p);
    if (m->alloc(&m->scale, m->L[2].out_p) != cudaSuccess || m->alloc(&m->shift, m->L[2].out_p) != cudaSuccess ||
        m->alloc(&m->err, 4) != cudaSuccess || m->alloc(&m->splitbuf, wmax * kMaxSplits) != cudaSuccess)
        return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_create: buffers");
    std::vector<float> one(m->L[2].out_p, 1.0f);
    cudaMemcpy(m->scale, one.data(), one.size() * 4, cudaMemcpyHostToDevice);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_create: ") + cudaGetErrorString(e));
    *out = m.release();
    return set_ok();
}

cut_status cut_mlp_free(cut_mlp *m) {
    delete m;
    return set_ok();
}

cut_status cut_mlp_set_output_affine(cut_mlp *m, const float *scale, const float *shift) {
    if (!m || !scale || !shift) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_set_output_affine: null argument");
    for (int c = 0; c < m->n_out; c++)
        if (!(scale[c] > 0.0f) || !std::isfinite(shift[c]))
            return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_set_output_affine: scale must be > 0, shift finite");
    cudaSetDevice(m->device);
    cudaMemcpy(m->scale, scale, m->n_out * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->shift, shift, m->n_out * 4, cudaMemcpyHostToDevice);
    return set_ok();
}

cut_status cut_mlp_get_output_affine(const cut_mlp *m, float *scale, float *shift) {
    if (!m || (!scale && !shift)) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_get_output_affine: null argument");
    cudaSetDevice(m->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && scale) e = cudaMemcpy(scale, m->scale, m->n_out * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && shift) e = cudaMemcpy(shift, m->shift, m->n_out * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(CUT_ERR_CUDA, std::string("cut_mlp_get_output_affine: ") + cudaGetErrorString(e));
    }
    return set_ok();
}

cut_status cut_mlp_set_linear(cut_mlp *m, const float *J) {
    if (!m) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_set_linear: null model");
    cudaSetDevice(m->device);
    if (!J) {
        m->J = nullptr;
        return set_ok();
    }
    if (!m->J) {
        float *d = nullptr;
        if (m->alloc(&d, (size_t)m->n_out * m->n_in) != cudaSuccess)
            return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_set_linear");
        m->J = d;
    }
    cudaMemcpy(m->J, J, (size_t)m->n_out * m->n_in * 4, cudaMemcpyHostToDevice);
    return set_ok();
}

cut_status cut_mlp_fit_linear(cut_mlp *m, int batch, const float *x, const double *t, const float *weight,
                              cut_stream_t stream) {
    TraceRange trace_("cut_mlp_fit_linear");
    if (!m || batch < 2 || !x || !t) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_fit_linear: bad argument");
    if (m->n_in + 1 > mlpk::kFitP) return set_error(CUT_ERR_UNSUPPORTED, "cut_mlp_fit_linear: more than 63 inputs");
    if (weight)
        for (int o = 0; o < m->n_out; o++)
            if (!(weight[o] > 0.0f) || !std::isfinite(weight[o]))
                return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_fit_linear: weights must be finite and > 0");
    cudaSetDevice(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!m->J) {
        float *d = nullptr;
        if (m->alloc(&d, (size_t)m->n_out * m->n_in) != cudaSuccess)
            return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_fit_linear: J");
        m->J = d;
    }
    const int P = m->n_in + 1, ncol = P + m->n_out;
    const int chunks = (int)std::min<int64_t>(128, std::max<int64_t>(1, batch / 256));
    const int64_t rpc = (batch + chunks - 1) / chunks;
    const size_t np_ = (size_t)chunks * P * ncol, nres = (size_t)chunks * m->n_out;
    double *buf = nullptr;
    cudaError_t e = cut::scratch_alloc(&buf, (np_ + (size_t)P * ncol + (size_t)P * m->n_out + nres + m->n_out) * 8 + 64, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_fit_linear: scratch");
    }
    double *partial = buf, *M = partial + np_, *coef = M + (size_t)P * ncol, *rp = coef + (size_t)P * m->n_out,
           *ss = rp + nres;
    float *w = nullptr;
    if (weight) {
        e = cut::scratch_alloc(&w, m->n_out * 4, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w, weight, m->n_out * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFreeAsync(buf, s);
            return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_mlp_fit_linear: weights");
        }
    }
    pdl_launch(mlpk::fit_gram_partials, dim3((ncol + 127) / 128, chunks), 128, 0, s, x, t, batch, m->n_in, m->n_out, rpc,
                                                                              partial);
    pdl_launch(mlpk::fit_reduce, grid_of((int64_t)P * ncol), 256, 0, s, partial, chunks, (int64_t)P * ncol, M);
    // a relative ridge of 1e-12 of the Gram matrix's scale keeps the solve
    // defined when an input never varies
    pdl_launch(mlpk::fit_solve, 1, 256, 0, s, M, m->n_in, m->n_out, 1e-12 * (double)batch, coef, nullptr);
    pdl_launch(mlpk::fit_resid_partials, dim3((m->n_out + 127) / 128, chunks), 128, 0, s, x, t, coef, batch, m->n_in,
                                                                                   m->n_out, rpc, rp);
    pdl_launch(mlpk::fit_reduce, grid_of(m->n_out), 256, 0, s, rp, chunks, m->n_out, ss);
    pdl_launch(mlpk::fit_write, grid_of(m->n_out), 256, 0, s, coef, ss, w, batch, m->n_in, m->n_out, m->scale, m->shift,
                                                      m->J);
    e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    if (w) cudaFreeAsync(w, s);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_fit_linear: ") + cudaGetErrorString(e));
    return set_ok();
}

cut_status cut_mlp_ensemble_stats(int K, int batch, int n_out, const float *const *preds, const uint8_t *mask,
                                  float *mean, float *spread, cut_stream_t stream) {
    if (K < 1 || K > 16 || batch < 0 || n_out < 1 || !preds || !mask || !spread)
        return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_ensemble_stats: bad argument (1 <= K <= 16)");
    mlpk::Members mb;
    for (int k = 0; k < K; k++) {
        if (!preds[k]) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_ensemble_stats: null member output");
        mb.p[k] = preds[k];
    }
    if (batch == 0) return set_ok();
    pdl_launch(mlpk::ensemble_stats, batch, 256, 0, (cudaStream_t)stream, mb, K, n_out, mask, mean, spread);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_ensemble_stats: ") + cudaGetErrorString(e));
    return set_ok();
}

int64_t cut_mlp_param_count(const cut_mlp *m) {
    if (!m) return -1;
    int64_t c = 0;
    for (int l = 0; l < 3; l++) c += (int64_t)m->L[l].in * m->L[l].out + m->L[l].out;
    return c;
}

// Copy parameters (or their gradients, which = 1) between the device and a
// flat host array W1, b1, W2, b2, W3, b3 (W row-major [out][in]).
static cut_status params_io(cut_mlp *m, float *host, int to_host, int which) {
    cudaSetDevice(m->device);
    int64_t off = 0;
    for (int l = 0; l < 3; l++) {
        Layer &Ly = m->L[l];
        float *W = which ? Ly.gw : Ly.w;
        float *B = which ? Ly.gb : Ly.b;
        for (int o = 0; o < Ly.out; o++) {
            cudaError_t e = to_host ? cudaMemcpy(host + off, W + (size_t)o * Ly.in_p, Ly.in * 4, cudaMemcpyDeviceToHost)
                                    : cudaMemcpy(W + (size_t)o * Ly.in_p, host + off, Ly.in * 4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, "cut_mlp params copy");
            off += Ly.in;
        }
        cudaError_t e = to_host ? cudaMemcpy(host + off, B, Ly.out * 4, cudaMemcpyDeviceToHost)
                                : cudaMemcpy(B, host + off, Ly.out * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, "cut_mlp params copy");
        off += Ly.out;
        if (!to_host && !which) {
            const size_t cnt = (size_t)Ly.in_p * Ly.out_p;
            pdl_launch(mlpk::to_bf16, grid_of(cnt), 256, 0, 0, Ly.w, cnt, Ly.in_p, Ly.out_p, Ly.wb, Ly.wt);
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp params: ") + cudaGetErrorString(e));
    return set_ok();
}

cut_status cut_mlp_get_params(cut_mlp *m, float *host, int grads) {
    if (!m || !host) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_get_params: null argument");
    return params_io(m, host, 1, grads ? 1 : 0);
}

cut_status cut_mlp_set_params(cut_mlp *m, const float *host) {
    if (!m || !host) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_set_params: null argument");
    return params_io(m, const_cast<float *>(host), 0, 0);
}

cut_status cut_mlp_forward(cut_mlp *m, int batch, const float *x, float *y, cut_stream_t stream) {
    TraceRange trace_("cut_mlp_forward");
    if (!m || batch < 1 || !x || !y) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_forward: bad argument");
    cudaSetDevice(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    cut_status st = forward(m, batch, x, s, m->scale, m->shift, y);
    if (st != CUT_OK) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_forward: ") + cudaGetErrorString(e));
    return set_ok();
}

}  // extern "C"

static cut_status backward_body(cut_mlp *m, int batch, const float *x, const float *target, float *loss,
                                cudaStream_t s) {
    cut_status st = forward(m, batch, x, s, nullptr, nullptr, nullptr);
    if (st != CUT_OK) return st;
    const int Mp = pad_to(batch, 128);
    Layer *L = m->L;
    // output layer
    pdl_launch(mlpk::mse_grad, dim3(L[2].out_p / 32, Mp / 32), dim3(32, 8), 0, s, 
        m->z[2], L[2].out_p, target, batch, m->n_out, m->scale, m->shift, Mp, L[2].out_p, m->dzb, m->dzt, m->dz32,
        loss, m->J, x, m->n_in);
    bf16 *dzb = m->dzb, *dzt = m->dzt, *nb = m->dzb2, *nt = m->dzt2;
    float *dz32 = m->dz32, *n32 = m->dz32b;
    for (int l = 2; l >= 0; l--) {
        Layer &Ly = L[l];
        // dW_l[out][in] = dZ^T[out][M] * IN^T[in][M]^T
        const bf16 *inT = l == 0 ? m->xt : m->ht[l - 1];
        // few output tiles and a long k (the batch): split k across CTAs so
        // that about one wave of SMs works on it, then sum the partials in
        // split order (deterministic)
        const int bn = Ly.in_p % 128 == 0 ? 128 : 64;
        const int tiles = (Ly.out_p / 128) * (Ly.in_p / bn);
        int splits = 1;
        while (splits < kMaxSplits && tiles * splits * 2 <= 148 && Mp % (64 * splits * 2) == 0 &&
               Mp / (splits * 2) >= 256)
            splits *= 2;
        tc::Epi e = epi0(Ly.out_p, Ly.in_p, m->err);
        e.out_f32 = splits > 1 ? m->splitbuf : Ly.gw;
        e.ld_f32 = Ly.in_p;
        e.split_stride = (int64_t)Ly.out_p * Ly.in_p;
        st = gemm(dzt, inT, Ly.out_p, Ly.in_p, Mp, e, s, splits);
        if (st != CUT_OK) return st;
        if (splits > 1)
            pdl_launch(mlpk::sum_splits, grid_of(e.split_stride), 256, 0, s, m->splitbuf, splits, e.split_stride, Ly.gw);
        pdl_launch(mlpk::col_sum, (Ly.out_p + 31) / 32, dim3(32, mlpk::kColSumGroups), 0, s, dz32, Ly.out_p, batch, Ly.out_p,
                                                                                   Ly.gb);
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
        Layer &Lp = L[l - 1];
        tc::Epi d = epi0(Mp, Lp.out_p, m->err);
        d.dgelu_z = m->z[l - 1];
        d.ldz = Lp.out_p;
        d.out_f32 = n32;
        d.ld_f32 = Lp.out_p;
        d.out_bf16 = nb;
        d.ld_bf16 = Lp.out_p;
        d.out_t = nt;
        d.ld_t = Mp;
        st = gemm(dzb, Ly.wt, Mp, Lp.out_p, Ly.out_p, d, s);
        if (st != CUT_OK) return st;
        std::swap(dzb, nb);
        std::swap(dzt, nt);
        std::swap(dz32, n32);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_backward: ") + cudaGetErrorString(e));
    return set_ok();
}

extern "C" {
cut_status cut_mlp_backward(cut_mlp *m, int batch, const float *x, const float *target, float *loss,
                            cut_stream_t stream) {
    TraceRange trace_("cut_mlp_backward");
    if (!m || batch < 1 || !x || !target) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_backward: bad argument");
    cudaSetDevice(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    cut_status st = ensure_batch(m, pad_to(batch, 128));   // no allocation inside a capture
    if (st != CUT_OK) return st;
    cut_mlp::GraphKey key;
    key.batch = batch;
    key.Mcap = m->Mcap;
    key.x = x;
    key.t = target;
    key.loss = loss;
    key.J = m->J;
    if (!(key == m->gkey)) {
        m->drop_graph();
        m->gkey = key;
        m->gseen = 0;
    }
    m->gseen++;
    if (!m->gexec && m->gseen >= 2) {
        if (!m->gstream) cudaStreamCreateWithFlags(&m->gstream, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(m->gstream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            st = backward_body(m, batch, x, target, loss, m->gstream);
            e = cudaStreamEndCapture(m->gstream, &graph);
            if (st == CUT_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&m->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (st != CUT_OK || e != cudaSuccess) m->drop_graph();
        }
        cudaGetLastError();   // a failed capture falls back to direct launches
    }
    if (m->gexec) {
        cudaError_t e = cudaGraphLaunch(m->gexec, s);
        if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_backward: ") + cudaGetErrorString(e));
        return set_ok();
    }
    return backward_body(m, batch, x, target, loss, s);
}

cut_status cut_mlp_adamw_step(cut_mlp *m, float lr, float beta1, float beta2, float eps, float weight_decay,
                              cut_stream_t stream) {
    TraceRange trace_("cut_mlp_adamw_step");
    if (!m || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_adamw_step: bad hyper-parameters");
    cudaSetDevice(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    m->t++;
    const float bc1 = 1.0f - (float)std::pow((double)beta1, (double)m->t);
    const float bc2 = 1.0f - (float)std::pow((double)beta2, (double)m->t);
    // weights in tiles (with both BF16 copies), biases element by element
    mlpk::AdamTiles tw;
    memset(&tw, 0, sizeof(tw));
    mlpk::AdamSegs segs;
    memset(&segs, 0, sizeof(segs));
    int64_t start = 0;
    for (int l = 0; l < 3; l++) {
        Layer &Ly = m->L[l];
        tw.s[l] = {Ly.w, Ly.gw, Ly.mw, Ly.vw, Ly.wb, Ly.wt, (int64_t)Ly.in_p * Ly.out_p, 0, Ly.in_p, Ly.out_p,
                   weight_decay};
        tw.tiles_x[l] = (Ly.in_p + 31) / 32;
        tw.tile_start[l + 1] = tw.tile_start[l] + (int64_t)tw.tiles_x[l] * ((Ly.out_p + 31) / 32);
        mlpk::AdamSeg &B = segs.s[segs.n++];
        B = {Ly.b, Ly.gb, Ly.mb, Ly.vb, nullptr, nullptr, (int64_t)Ly.out_p, start, 1, 1, 0.0f};
        start += B.count;
    }
    segs.total = start;
    pdl_launch(mlpk::adamw_tiles, (int)std::min<int64_t>(tw.tile_start[3], 148 * 8), dim3(32, 8), 0, s, 
        tw, lr, beta1, beta2, eps, bc1, bc2);
    pdl_launch(mlpk::adamw_all, grid_of(start), 256, 0, s, segs, lr, beta1, beta2, eps, bc1, bc2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_adamw_step: ") + cudaGetErrorString(e));
    return set_ok();
}

cut_status cut_mlp_status(cut_mlp *m) {
    if (!m) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_status: null");
    cudaSetDevice(m->device);
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, m->err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_status: ") + cudaGetErrorString(e));
    if (h) {
        const int zero = 0;   // reported once: later calls start clean
        cudaMemcpy(m->err, &zero, 4, cudaMemcpyHostToDevice);
        return set_error(CUT_ERR_TIMEOUT, "cut_mlp: a tensor-core pipeline wait timed out");
    }
    return set_ok();
}

cut_status cut_mlp_inject_stall(cut_mlp *m, int on) {
    if (!m) return set_error(CUT_ERR_INVALID_ARG, "cut_mlp_inject_stall: null");
    cudaSetDevice(m->device);
    cudaError_t e = cudaDeviceSynchronize();
    const int v = on ? 1 : 0;
    if (e == cudaSuccess) e = cudaMemcpy(m->err + 1, &v, 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_mlp_inject_stall: ") + cudaGetErrorString(e));
    return set_ok();
}

}  // extern "C"
