// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory, operands staged by TMA).
//
//   C[M, N] = A[M, K] * B[N, K]^T     (both operands K-major, row-major in HBM)
//
// One CTA of 128 threads computes a 128 x BN tile:
//   warp 0, lane 0 : TMA producer, ST-deep ring of 128x64 / BNx64 tiles
//                    (128-byte swizzle), one mbarrier pair per stage;
//   warp 1, lane 0 : issues tcgen05.mma (M=128, N=BN, K=16 per instruction)
//                    and tcgen05.commit to release each stage;
//   all 4 warps    : epilogue, tcgen05.ld of their 32 TMEM lanes (rows),
//                    staged through shared memory so that every global
//                    access is coalesced; fused bias / GELU / GELU-derivative /
//                    output affine / FP32 linear skip / transposed stores.
// Every mbarrier wait is bounded; on expiry the kernel records an error,
// still frees its tensor memory and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pdl.cuh"

namespace cut {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;          // one 128-byte swizzle row of BF16
// Ring depth: 3 stages (97 KB at BN = 128) let two CTAs share an SM, for
// grids of more than one wave; a grid of at most one CTA per SM takes 6
// (193 KB, one CTA per SM), so that each CTA keeps twice the operand copies
// in flight over its k loop.
constexpr int STAGES = 3;
constexpr int STAGES_DEEP = 6;
constexpr int kThreads = 256;          // 8 warps: two per TMEM lane quarter share the epilogue
constexpr long long kSpinLimit = 1ll << 26;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // a pipeline wait gives up after 1 s

struct Epi {
    const float *bias;          // [N] or null
    const float *dgelu_z;       // ACT == kGeluGrad: multiply by GELU'(z), z row-major [M][ldz]
    int ldz;
    float alpha;                // scale of the product
    const float *post_scale;    // optional per-column affine after bias: v * scale + shift
    const float *post_shift;
    const float *lin_J;         // optional linear skip: + sum_k J[col][k] x[row][k] (FP32)
    const float *lin_x;
    int lin_k;
    float *out_f32;             // [M][ld_f32] or null (split k: [splits][M][ld_f32])
    int ld_f32;
    int64_t split_stride;       // split k (gridDim.z > 1): floats between the partial products
    __nv_bfloat16 *out_bf16;    // [M][ld_bf16] or null
    int ld_bf16;
    __nv_bfloat16 *out_t;       // transposed [N][ld_t] or null
    int ld_t;
    int M, N;                   // valid extent (rows, columns) written
    int *err;                   // set to 1 when a wait timed out
    const int *stall;           // failure injection for tests: while *stall != 0 the
                                // producer issues no operand copies, so the MMA
                                // issuer's wait runs out (no fault, no hang)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on the phase with the given parity; false once it has waited
// kWaitLimitNs (or kSpinLimit polls), whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (long long it = 0; it < kSpinLimit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 0) {
            const unsigned long long t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;          // start address
    d |= (uint64_t)1 << 16;                // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;                // version
    d |= (uint64_t)2 << 61;                // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float dgelu(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// Epilogue activation, fixed at compile time so that the row loop carries
// only the arithmetic it needs (a runtime choice let the compiler evaluate
// the error function on every element).
enum EpiAct { kLinear = 0, kGelu = 1, kGeluGrad = 2 };

template <int BN, int ACT, int ST = STAGES>
__global__ void __launch_bounds__(kThreads, ST <= STAGES ? 2 : 1)
    gemm_bf16_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K, Epi ep) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile ring
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    unsigned char *sA = base;
    unsigned char *sB = base + ST * A_BYTES;
    __shared__ __align__(8) uint64_t full[ST], empty[ST], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // column tiles fastest: the CTAs that share a row tile of A run together,
    // so a large A is read from DRAM once and B stays in L2
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int KT = K / BK;                 // K columns per split; split z starts at z K
    const int kbase = blockIdx.z * K;

    if (threadIdx.x == 0) {
        // start fetching both tensor maps while the barriers and TMEM are set up
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        for (int s = 0; s < ST; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // the barriers and the accumulator are set up while the previous kernel
    // on the stream may still run; no global memory is touched before this
    pdl_enter();

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // producer
        const bool stall = ep.stall && *ep.stall;
        for (int kt = 0; kt < KT && !failed && !stall; kt++) {
            const int s = kt % ST;
            if (kt >= ST && !mbar_wait(&empty[s], ((kt / ST) - 1) & 1)) { failed = 1; break; }
            mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
            tma_load_2d(sA + s * A_BYTES, &tmA, &full[s], kbase + kt * BK, m0);
            tma_load_2d(sB + s * B_BYTES, &tmB, &full[s], kbase + kt * BK, n0);
            issued = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN);
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % ST;
            if (!mbar_wait(&full[s], (kt / ST) & 1)) { failed = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++) {
                const uint64_t da = smem_desc(sA + s * A_BYTES + kk * 32);
                const uint64_t db = smem_desc(sB + s * B_BYTES + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    __syncwarp();
    // every thread waits for the accumulator
    const bool ok = mbar_wait(&done, 0);
    if (!ok) failed = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();

    if (!failed) {
        // Epilogue through shared memory (the operand ring is idle once the
        // accumulator is complete): each warp reads 32 rows x 32 columns of
        // TMEM (thread = row), stages them transposed, and applies the
        // epilogue with lane = column, so loads of bias / z and row-major
        // stores are coalesced; the transposed output is written back from
        // the row layout, where it is coalesced too.
        static_assert(BN % 32 == 0, "epilogue works on 32-column slices");
        static_assert(kThreads / 32 * 2 * 32 * 33 * 4 <= ST * (A_BYTES + B_BYTES), "staging fits in the ring");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        float *stile = reinterpret_cast<float *>(base) + warp * (2 * 32 * 33);
        float *ltile = stile + 32 * 33;        // linear-skip terms, same layout
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (its rows); the warps
        // sharing a lane quarter take alternate 32-column slices
        constexpr int kQuarterWarps = kThreads / 128;
        const int quarter = warp & 3, part = warp >> 2;
        const int rbase = m0 + quarter * 32;
        const int myrow = rbase + lane;
        float *const out_f32 = ep.out_f32 ? ep.out_f32 + (int64_t)blockIdx.z * ep.split_stride : nullptr;
#pragma unroll 1
        for (int c0 = part * 32; c0 < BN; c0 += 32 * kQuarterWarps) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 32; i++) stile[lane * 33 + i] = __uint_as_float(r[i]);
            if (ep.lin_J) {
                // skip terms sum_k J[col][k] x[row][k] in the row layout (J
                // broadcast), 16 columns per pass to bound the registers
#pragma unroll 1
                for (int h = 0; h < 32; h += 16) {
                    float l[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) l[i] = 0.0f;
                    if (myrow < ep.M) {
                        for (int k = 0; k < ep.lin_k; k++) {
                            const float xv = ep.lin_x[(int64_t)myrow * ep.lin_k + k];
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                const int col = n0 + c0 + h + i;
                                if (col < ep.N) l[i] = fmaf(ep.lin_J[(int64_t)col * ep.lin_k + k], xv, l[i]);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; i++) ltile[lane * 33 + h + i] = l[i];
                }
            }
            __syncwarp();
            const int col = n0 + c0 + lane;
            const bool colok = col < ep.N;
            const float bias = (ep.bias && colok) ? ep.bias[col] : 0.0f;
            const float psc = (ep.post_scale && colok) ? ep.post_scale[col] : 1.0f;
            const float psh = (ep.post_scale && colok) ? ep.post_shift[col] : 0.0f;
            // every row's GELU-derivative input in flight at once, parked in
            // the second tile (the skip term and the GELU derivative are
            // never used by the same GEMM)
            if constexpr (ACT == kGeluGrad) {
                float zr[32];
#pragma unroll
                for (int rr = 0; rr < 32; rr++)
                    zr[rr] = (colok && rbase + rr < ep.M) ? ep.dgelu_z[(int64_t)(rbase + rr) * ep.ldz + col] : 0.0f;
#pragma unroll
                for (int rr = 0; rr < 32; rr++) ltile[rr * 33 + lane] = zr[rr];
            }
            // partly unrolled: a fully unrolled row loop with the GELU (or
            // its derivative) overflows the instruction cache
            constexpr int kRowUnroll = ACT == kLinear ? 8 : 2;
#pragma unroll(kRowUnroll)
            for (int rr = 0; rr < 32; rr++) {
                const int row = rbase + rr;
                if (!colok || row >= ep.M) continue;
                float v = stile[rr * 33 + lane] * ep.alpha + bias;
                if (ep.post_scale) v = v * psc + psh;
                if (ep.lin_J) v += ltile[rr * 33 + lane];
                if constexpr (ACT == kGeluGrad) v *= dgelu(ltile[rr * 33 + lane]);
                if (out_f32) out_f32[(int64_t)row * ep.ld_f32 + col] = v;
                float a = v;
                if constexpr (ACT == kGelu) a = gelu(v);
                if (ep.out_bf16) ep.out_bf16[(int64_t)row * ep.ld_bf16 + col] = __float2bfloat16(a);
                stile[rr * 33 + lane] = a;
            }
            __syncwarp();
            if (ep.out_t && myrow < ep.M) {
#pragma unroll 8
                for (int i = 0; i < 32; i++) {
                    const int cc = n0 + c0 + i;
                    if (cc < ep.N) ep.out_t[(int64_t)cc * ep.ld_t + myrow] = __float2bfloat16(stile[lane * 33 + i]);
                }
            }
            __syncwarp();
        }
    } else {
        if (threadIdx.x == 0) {
            // let the copies this thread issued land before the CTA exits
            for (int kt = issued - ST < 0 ? 0 : issued - ST; kt < issued; kt++)
                mbar_wait(&full[kt % ST], (kt / ST) & 1);
            if (ep.err) atomicExch(ep.err, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

template <int BN, int ST = STAGES>
constexpr size_t gemm_smem_bytes() {
    return 1024 + (size_t)ST * (BM * BK * 2 + BN * BK * 2);
}

}  // namespace tc
}  // namespace cut
