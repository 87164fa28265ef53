// cut_lib.cu -- C ABI of the graph engine: load/upload, right-hand side,
// adjoint, flows (paper Sec. 2.2-2.4).  See include/cut.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "alloc.h"
#include "bundle.h"
#include "cut.h"
#include "flow_kernels.cuh"
#include "kernels.cuh"
#include "status.h"
#include "trace.h"

namespace cut {

static thread_local std::string g_err;
cut_status set_error(cut_status s, const std::string &msg) {
    g_err = msg;
    return s;
}
cut_status set_ok() { return CUT_OK; }

// On failure: report, and clear the runtime's record of a non-sticky error
// (an allocation that did not fit) so that later calls start clean.
#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess) {                                                                \
            (void)cudaGetLastError();                                                           \
            return set_error(_e == cudaErrorMemoryAllocation ? CUT_ERR_OUT_OF_MEMORY : CUT_ERR_CUDA, \
                             std::string(#expr) + ": " + cudaGetErrorString(_e));               \
        }                                                                                       \
    } while (0)

static void *current_context();

// One pool per device, remade when the device's context changes (a device
// reset invalidates the old handle).
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[256] = {nullptr};
static void *g_pool_ctx[256] = {nullptr};

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        void *ctx = current_context();
        if (!g_pool[dev] || !ctx || ctx != g_pool_ctx[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            unsigned long long keep = kScratchKeepBytes;
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            g_pool[dev] = np;
            g_pool_ctx[dev] = current_context();
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

struct DevCSR {
    uint64_t *rp = nullptr;
    uint2 *rec = nullptr;
    int64_t rows = 0, R = 0;
    // long rows split into pieces (transposed orders only): rp then bounds
    // the `rows` pieces, and pieces vr[r] .. vr[r+1]-1 make up row r
    uint64_t *vr = nullptr;
    int64_t real_rows = 0;
    // forward commutator stage of a graph with few, long rows: the same
    // records cut into `pieces` pieces (prp bounds them, pvr[r] is the first
    // piece of row r) so that enough lane groups share the work; rp and
    // rows keep describing whole rows
    uint64_t *prp = nullptr, *pvr = nullptr;
    int64_t pieces = 0;
    int64_t lane_rows = 0;   // rows of the whole stage: picks the lanes per row, so
                             // a shard sums each row exactly as the whole graph does
};

}  // namespace cut

struct cut_graph {
    int device = 0;
    cut::HostGraph host;
    cut::DevCSR st[3];             // forward stages (2: outside space, optional)
    cut::DevCSR tx, txi, th;       // transposed orders (adjoint), built lazily
    bool have_T = false;
    double *wtab = nullptr;        // exact factors as doubles
    float *wtab32 = nullptr;
    unsigned long long *wsign = nullptr;  // sign bit per code
    double wmag = 1.0;             // common magnitude when all factors share it
    int wuniform = 0;
    uint32_t wnegmask = 0;         // bit c set when factor c < 0 (codes < 32)
    int arith = CUT_ARITH_FP64;    // arithmetic of the commutator stage
    int shard_rank = 0, shard_world = 0;   // world > 0: only rows [lo, hi) of stages 0, 1 resident
    int64_t lo[2] = {0, 0}, hi[2] = {0, 0};
    int64_t device_bytes = 0;
    std::mutex mu;
    ~cut_graph() {
        if (device < 0) return;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        for (auto *c : {&st[0], &st[1], &st[2], &tx, &txi, &th}) {
            cudaFree(c->rp);
            cudaFree(c->rec);
            cudaFree(c->vr);
            cudaFree(c->prp);
            cudaFree(c->pvr);
        }
        cudaFree(wtab);
        cudaFree(wtab32);
        cudaFree(wsign);
        cudaSetDevice(cur);
    }
};

namespace cut {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

static int grid_for_rows(int64_t rows) {
    int64_t b = (rows + k::kWarpsPerBlock - 1) / k::kWarpsPerBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 16));
}
static int grid_for_len(int64_t len) {
    int64_t b = (len + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 8));
}

static cut_status upload_csr(DevCSR &d, const std::vector<uint64_t> &rp, const std::vector<uint32_t> &rec,
                             int64_t &bytes) {
    d.rows = (int64_t)rp.size() - 1;
    d.lane_rows = d.rows;
    d.R = (int64_t)rec.size() / 2;
    CUDA_TRY(cudaMalloc(&d.rp, rp.size() * 8));
    CUDA_TRY(cudaMemcpy(d.rp, rp.data(), rp.size() * 8, cudaMemcpyHostToDevice));
    size_t rb = std::max<size_t>(8, rec.size() * 4);
    CUDA_TRY(cudaMalloc(&d.rec, rb));
    if (!rec.empty()) CUDA_TRY(cudaMemcpy(d.rec, rec.data(), rec.size() * 4, cudaMemcpyHostToDevice));
    bytes += (int64_t)(rp.size() * 8 + rec.size() * 4);
    return CUT_OK;
}

static cut_status upload_weights(cut_graph *g);
static cut_status ensure_transposes(cut_graph *g);

// Entry points that traverse the whole graph refuse a shard handle.
static cut_status whole_graph(const cut_graph *g, const char *fn) {
    if (g && g->shard_world > 0)
        return set_error(CUT_ERR_INVALID_ARG, std::string(fn) + ": the handle holds one shard of the graph; use the "
                                                                "cut_shard_* entry points");
    return CUT_OK;
}


// Few long rows (fewer than kManyRows rows holding kPieceAvg records or more
// on average, as in the Pauli-boson graphs): cut every row of the forward
// commutator stage into pieces of about kFwdPiece records.  The cut of a row
// depends only on its own length, so a shard holding whole rows cuts them
// exactly as the whole graph does.  rp: the whole stage's row pointers;
// rows [lo, hi) are the resident ones, record offsets rebased to rp[lo].
constexpr int64_t kManyRowsForPieces = 16384;
constexpr uint64_t kPieceAvg = 512, kFwdPiece = 256;

static cut_status add_pieces(DevCSR &d, const std::vector<uint64_t> &rp, int64_t lo, int64_t hi, int64_t &bytes) {
    const int64_t rows = (int64_t)rp.size() - 1;
    if (rows <= 0 || rows >= kManyRowsForPieces || rp[rows] < (uint64_t)rows * kPieceAvg || hi <= lo) return CUT_OK;
    std::vector<uint64_t> prp{0}, pvr(hi - lo + 1);
    for (int64_t r = lo; r < hi; r++) {
        pvr[r - lo] = prp.size() - 1;
        const uint64_t b = rp[r] - rp[lo], len = rp[r + 1] - rp[r];
        const uint64_t np = std::max<uint64_t>(1, (len + kFwdPiece - 1) / kFwdPiece);
        for (uint64_t q = 1; q <= np; q++) prp.push_back(b + len * q / np);
    }
    pvr[hi - lo] = prp.size() - 1;
    CUDA_TRY(cudaMalloc(&d.prp, prp.size() * 8));
    CUDA_TRY(cudaMemcpy(d.prp, prp.data(), prp.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&d.pvr, pvr.size() * 8));
    CUDA_TRY(cudaMemcpy(d.pvr, pvr.data(), pvr.size() * 8, cudaMemcpyHostToDevice));
    d.pieces = (int64_t)prp.size() - 1;
    bytes += (int64_t)(prp.size() + pvr.size()) * 8;
    return CUT_OK;
}

// ----------------------------------------------------------------- RHS core
// dx_o (o < nops) for operands x_o, given xi; operands processed 4 at a time.
static k::Weights weights_of(const cut_graph *g) {
    k::Weights w;
    w.val = g->wtab;
    w.sign = g->wsign;
    w.mag = g->wmag;
    w.n_codes = (int)g->host.num.size();
    w.uniform = g->wuniform;
    return w;
}

// lanes per CSR segment.  With many outputs, 8 lanes per commutator row
// (4 per generator row) keep lanes busy and the closing reductions short;
// with few outputs (a few thousand) a whole warp per row is needed to fill
// the GPU's ~7000 resident warps.
constexpr int kManyRows = 16384;
static int comm_lanes(int64_t rows) { return rows >= kManyRows ? 8 : 32; }
static int gen_lanes(int64_t rows) { return rows >= kManyRows ? 4 : 8; }

static int grid_for_groups(int64_t rows, int lanes) {
    return grid_for_rows((rows + (32 / lanes) - 1) / (32 / lanes));
}

template <int M, int L>
static void comm_launch(const DevCSR &c, const k::Weights &w, const double *xi, const k::Ops<M> &ops,
                        cudaStream_t s, const int *done) {
    const int grid = grid_for_groups(c.rows, L);
    if (w.uniform)
        pdl_launch(k::comm_stage<M, true, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, ops, c.rows, done);
    else
        pdl_launch(k::comm_stage<M, false, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, ops, c.rows, done);
}

template <int M, int L>
static void comm_launch_x4(const DevCSR &c, const k::Weights &w, const double *xi, const k::Ops<M> &ops,
                           const double *X4, cudaStream_t s, const int *done) {
    const int grid = grid_for_groups(c.rows, L);
    if (w.uniform)
        pdl_launch(k::comm_stage_x4<M, true, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, X4, ops, c.rows, done);
    else
        pdl_launch(k::comm_stage_x4<M, false, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, X4, ops, c.rows, done);
}

// X4: optional scratch of n x 64 bytes on a 32-byte boundary.  With it, and
// at most eight operands, they go through pack_x4 + comm_stage_x4 in one
// pass over the records (one 256-bit gather per four operands and record);
// otherwise through comm_stage (one gather per operand, eight operands per
// pass).  Both give the same bits.
static void launch_comm(const cut_graph *g, const double *xi, int nops, const double *const *xs,
                        double *const *dxs, cudaStream_t s, const int *done, int stage = 1,
                        double *X4 = nullptr, const DevCSR *csr = nullptr, double *piece = nullptr,
                        bool prepacked = false) {
    const DevCSR &c = csr ? *csr : g->st[stage];
    const k::Weights w = weights_of(g);
    const int lanes = comm_lanes(c.lane_rows);
    if (X4 && nops <= 8 && c.prp && piece) {
        // few long rows: 8 lanes per piece, piece sums reduced row by row in
        // piece order
        const int64_t n = g->host.n();
        DevCSR pc = c;
        pc.rp = c.prp;
        pc.rows = c.pieces;
        switch (nops) {
#define CASE(M)                                                                                       \
    case M: {                                                                                         \
        k::Ops<M> ops;                                                                                \
        for (int t = 0; t < M; t++) { ops.x[t] = xs[t]; ops.dx[t] = piece + t * c.pieces; }            \
        if (!prepacked) pdl_launch(k::pack_x4<M>, grid_for_len(n), 256, 0, s, ops, n, X4, done);               \
        comm_launch_x4<M, 8>(pc, w, xi, ops, X4, s, done);                                             \
    } break;
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        }
        k::Ops<8> red;
        for (int t = 0; t < nops; t++) { red.x[t] = piece + t * c.pieces; red.dx[t] = dxs[t]; }
        pdl_launch(k::piece_reduce, grid_for_len(c.rows * nops), 256, 0, s, c.pvr, c.rows, red, nops, nullptr);
        return;
    }
    if (X4 && nops <= 8) {
        const int64_t n = g->host.n();
        for (int o0 = 0; o0 < nops; o0 += 8) {
            const int m = std::min(8, nops - o0);
            switch (m) {
#define CASE(M)                                                                                       \
    case M: {                                                                                         \
        k::Ops<M> ops;                                                                                \
        for (int t = 0; t < M; t++) { ops.x[t] = xs[o0 + t]; ops.dx[t] = dxs[o0 + t]; }                 \
        if (!prepacked) pdl_launch(k::pack_x4<M>, grid_for_len(n), 256, 0, s, ops, n, X4, done);               \
        if (lanes == 8) comm_launch_x4<M, 8>(c, w, xi, ops, X4, s, done);                              \
        else comm_launch_x4<M, 32>(c, w, xi, ops, X4, s, done);                                        \
    } break;
                CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
            }
        }
        return;
    }
    // up to eight operands share one pass over the records
    for (int o0 = 0; o0 < nops; o0 += 8) {
        int m = std::min(8, nops - o0);
        switch (m) {
#define CASE(M)                                                                        \
    case M: {                                                                          \
        k::Ops<M> ops;                                                                 \
        for (int t = 0; t < M; t++) { ops.x[t] = xs[o0 + t]; ops.dx[t] = dxs[o0 + t]; }  \
        if (lanes == 8) comm_launch<M, 8>(c, w, xi, ops, s, done);                     \
        else comm_launch<M, 32>(c, w, xi, ops, s, done);                               \
    } break;
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        }
    }
}

template <int L>
static void gen_launch(const DevCSR &c, const k::Weights &w, const double *h, double *xi, cudaStream_t s,
                       const int *done) {
    const int grid = grid_for_groups(c.rows, L);
    if (w.uniform)
        pdl_launch(k::gen_stage<true, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, h, xi, c.rows, done);
    else
        pdl_launch(k::gen_stage<false, L>, grid, k::kBlock, 0, s, c.rp, c.rec, w, h, xi, c.rows, done);
}

static void launch_gen(const cut_graph *g, const double *h, double *xi, cudaStream_t s, const int *done) {
    const DevCSR &c = g->st[0];
    const k::Weights w = weights_of(g);
    if (gen_lanes(c.lane_rows) == 4) gen_launch<4>(c, w, h, xi, s, done);
    else gen_launch<8>(c, w, h, xi, s, done);
}

// The generator of h = xs[0] and, when the commutator stage will read packed
// FP64 blocks (X4 given, at most eight operands, FP64 arithmetic), the
// packing of xs into X4, in one launch.  Returns whether X4 was packed.
static bool launch_gen_pack(const cut_graph *g, const double *const *xs, int nops, double *xi, double *X4,
                            cudaStream_t s, const int *done) {
    if (!X4 || nops > 8 || g->arith != CUT_ARITH_FP64) {
        launch_gen(g, xs[0], xi, s, done);
        return false;
    }
    const DevCSR &c = g->st[0];
    const k::Weights w = weights_of(g);
    const int64_t n = g->host.n();
    const int gl = gen_lanes(c.lane_rows);
    const int grid = std::max(grid_for_len(n), grid_for_groups(c.rows, gl));
    switch (nops) {
#define CASE(M)                                                                                       \
    case M: {                                                                                         \
        k::Ops<M> ops;                                                                                \
        for (int t = 0; t < M; t++) { ops.x[t] = xs[t]; ops.dx[t] = nullptr; }                        \
        if (w.uniform && gl == 4) pdl_launch(k::gen_pack<M, true, 4>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, c.rows, ops, n, X4, done); \
        else if (w.uniform) pdl_launch(k::gen_pack<M, true, 8>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, c.rows, ops, n, X4, done); \
        else if (gl == 4) pdl_launch(k::gen_pack<M, false, 4>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, c.rows, ops, n, X4, done); \
        else pdl_launch(k::gen_pack<M, false, 8>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi, c.rows, ops, n, X4, done); \
    } break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    return true;
}

// Double-float commutator stage: split xi and up to three operands at a time
// into FP32 pairs (xi2[n_g], X2[n][4]) and apply the records on the FP32 pipes.
static void launch_comm_df(const cut_graph *g, const double *xi, float2 *xi2, float2 *X2, int nops,
                           const double *const *xs, double *const *dxs, cudaStream_t s, const int *done,
                           double *piece = nullptr) {
    const DevCSR &rows_c = g->st[1];
    const bool pieces = rows_c.prp && piece;
    DevCSR c = rows_c;
    if (pieces) { c.rp = rows_c.prp; c.rows = rows_c.pieces; }
    const int64_t n = g->host.n(), ng = g->host.n_g();
    const k::Weights w = weights_of(g);
    // lanes per row as the FP64 stage (a whole warp per row shares a few
    // more L1 lines per instruction, but measured within run-to-run noise
    // of 8 lanes on the 16-orbital graph: 1.68-1.81 ms against 1.68-1.73);
    // 8 lanes per piece when few long rows are cut into pieces
    const int lanes = pieces ? 8 : comm_lanes(c.lane_rows);
    const int grid = grid_for_groups(c.rows, lanes);
    if (ng > 0) pdl_launch(k::split_pairs, grid_for_len(ng), 256, 0, s, xi, ng, xi2, 1, 0, done);
    for (int o0 = 0; o0 < nops; o0 += 3) {
        const int m = std::min(3, nops - o0);
        for (int t = 0; t < m; t++) pdl_launch(k::split_pairs, grid_for_len(n), 256, 0, s, xs[o0 + t], n, X2, 4, t, done);
        const float4 *X4 = reinterpret_cast<const float4 *>(X2);
        switch (m) {
#define CASE(M)                                                                                                   \
    case M: {                                                                                                     \
        k::Ops<M> ops;                                                                                            \
        for (int t = 0; t < M; t++) {                                                                             \
            ops.x[t] = xs[o0 + t];                                                                                \
            ops.dx[t] = pieces ? piece + t * c.rows : dxs[o0 + t];                                                \
        }                                                                                                         \
        if (lanes == 8)                                                                                           \
            pdl_launch(k::comm_stage_df<M, 8>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi2, X4, ops, c.rows, done);        \
        else                                                                                                      \
            pdl_launch(k::comm_stage_df<M, 32>, grid, k::kBlock, 0, s, c.rp, c.rec, w, xi2, X4, ops, c.rows, done);       \
    } break;
            CASE(1) CASE(2) CASE(3)
#undef CASE
        }
        if (pieces) {
            k::Ops<8> red;
            for (int t = 0; t < m; t++) { red.x[t] = piece + t * c.rows; red.dx[t] = dxs[o0 + t]; }
            pdl_launch(k::piece_reduce, grid_for_len(rows_c.rows * m), 256, 0, s, rows_c.pvr, rows_c.rows, red, m, nullptr);
        }
    }
}

// piece sums of the forward stage: after the n x 64-byte operand blocks
static double *piece_area(const cut_graph *g, float2 *X2) {
    return X2 ? reinterpret_cast<double *>(X2) + 8 * g->host.n() : nullptr;
}

// L(h) x_o for given xi (either arithmetic); df buffers may be null for FP64
static void apply_L(const cut_graph *g, const double *xi, float2 *xi2, float2 *X2, int nops,
                    const double *const *xs, double *const *dxs, cudaStream_t s, const int *done,
                    bool prepacked = false) {
    // without scratch (adjoint recomputation) the stage runs in FP64 with one
    // gather per operand
    if (g->arith == CUT_ARITH_DF64 && xi2 && X2)
        launch_comm_df(g, xi, xi2, X2, nops, xs, dxs, s, done, piece_area(g, X2));
    else
        launch_comm(g, xi, nops, xs, dxs, s, done, 1, reinterpret_cast<double *>(X2), nullptr, piece_area(g, X2),
                    prepacked);
}

static size_t operand_scratch_bytes(const cut_graph *g) {
    return (size_t)(std::max<int64_t>(1, g->host.n_g()) + 8 * g->host.n() + 8 * g->st[1].pieces) * 8 + 64;
}

// Operand scratch of the commutator stage: xi2[n_g] pairs (double-float
// only), then, on a 32-byte boundary, up to 64 bytes per input index:
// X2[n][4] FP32 pairs in double-float arithmetic, X4[n][4 NB] doubles in
// FP64 (NB = 1 or 2 blocks of 32 bytes; the stages read a block with one
// 256-bit load).
static float2 *operand_blocks(const cut_graph *g, void *df) {
    if (!df) return nullptr;
    const uintptr_t p = (uintptr_t)((float2 *)df + std::max<int64_t>(1, g->host.n_g()));
    return (float2 *)((p + 31) & ~(uintptr_t)31);
}

// f(Y) for the stacked state Y[nops][n] into DY[nops][n].  df: scratch of
// operand_scratch_bytes(g) bytes (operand scratch; null: operands gathered one by one).
static void stacked_rhs(const cut_graph *g, const double *Y, double *DY, int nops, double *xi,
                        cudaStream_t s, const int *done, void *df = nullptr) {
    const int64_t n = g->host.n();
    const double *xs[64];
    double *dxs[64];
    for (int o = 0; o < nops; o++) { xs[o] = Y + o * n; dxs[o] = DY + o * n; }
    float2 *X2 = operand_blocks(g, df);
    const bool packed = launch_gen_pack(g, xs, nops, xi, reinterpret_cast<double *>(X2), s, done);
    apply_L(g, xi, (float2 *)df, X2, nops, xs, dxs, s, done, packed);
}

}  // namespace cut

using namespace cut;

extern "C" {

const char *cut_last_error(void) { return g_err.c_str(); }
const char *cut_version(void) { return "cutgraph-b300 0.1 (sm_103a)"; }

cut_status cut_graph_load(const char *path, int device, unsigned flags, cut_graph **out) {
    TraceRange trace_("cut_graph_load");
    if (!path || !out) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load: null argument");
    if (flags & ~(unsigned)CUT_LOAD_ADJOINT) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load: unknown flags");
    *out = nullptr;
    if (device < -1) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load: bad device");
    if (device >= 0) {
        int ndev = 0;
        CUDA_TRY(cudaGetDeviceCount(&ndev));
        if (device >= ndev) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load: bad device");
    }
    std::unique_ptr<cut_graph> g(new cut_graph());
    g->device = device;
    std::string err;
    TraceRange read("cut_graph_load/read_verify");
    int rc = read_bundle(path, g->host, &err);
    read.end();
    if (rc != 0) return set_error((cut_status)rc, "cut_graph_load: " + err);
    if (device == -1) {  // host-only handle: query, labels, weights, records
        g->st[0].rows = g->host.n_g(); g->st[0].R = g->host.R(0);
        g->st[1].rows = g->host.n(); g->st[1].R = g->host.R(1);
        g->st[2].rows = g->host.n_out(); g->st[2].R = g->host.R(2);
        *out = g.release();
        return set_ok();
    }
    DeviceGuard dg(device);
    int64_t bytes = 0;
    TraceRange upload("cut_graph_load/upload");
    for (int s = 0; s < 3; s++) {
        cut_status st = upload_csr(g->st[s], g->host.rp[s], g->host.rec[s], bytes);
        if (st != CUT_OK) return st;
    }
    cut_status st = add_pieces(g->st[1], g->host.rp[1], 0, g->host.n(), bytes);
    if (st != CUT_OK) return st;
    st = upload_weights(g.get());
    if (st != CUT_OK) return st;
    g->device_bytes += bytes;
    upload.end();
    if (flags & CUT_LOAD_ADJOINT) {
        TraceRange tr("cut_graph_load/transposes");
        st = ensure_transposes(g.get());
        if (st != CUT_OK) return st;
    }
    *out = g.release();
    return set_ok();
}

}  // extern "C"

namespace cut {
// The exact factors as doubles, FP32 and sign bits on the graph's device
// (current device), and the uniform-magnitude flags.
static cut_status upload_weights(cut_graph *g) {
    std::vector<double> w(g->host.num.size());
    std::vector<float> w32(w.size());
    std::vector<unsigned long long> sg(w.size());
    g->wuniform = 1;
    for (size_t c = 0; c < w.size(); c++) {
        w[c] = (double)g->host.num[c] / (double)g->host.den[c];
        w32[c] = (float)w[c];
        sg[c] = w[c] < 0 ? 0x8000000000000000ull : 0ull;
        if (w[c] < 0 && c < 32) g->wnegmask |= 1u << c;
        if (std::fabs(w[c]) != std::fabs(w[0]) || w[c] == 0.0) g->wuniform = 0;
    }
    g->wmag = std::fabs(w[0]);
    CUDA_TRY(cudaMalloc(&g->wsign, sg.size() * 8));
    CUDA_TRY(cudaMemcpy(g->wsign, sg.data(), sg.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&g->wtab, w.size() * 8));
    CUDA_TRY(cudaMemcpy(g->wtab, w.data(), w.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&g->wtab32, w.size() * 4));
    CUDA_TRY(cudaMemcpy(g->wtab32, w32.data(), w.size() * 4, cudaMemcpyHostToDevice));
    g->device_bytes += (int64_t)w.size() * 20;
    return CUT_OK;
}
}  // namespace cut

extern "C" {

cut_status cut_graph_free(cut_graph *g) {
    delete g;
    return set_ok();
}

cut_status cut_graph_query(const cut_graph *g, cut_graph_desc *out) {
    if (!g || !out) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_query: null argument");
    memset(out, 0, sizeof(*out));
    out->algebra = g->host.algebra;
    out->nmodes = g->host.nmodes;
    out->max_rank = g->host.max_rank;
    out->n_codes = (int)g->host.num.size();
    out->n = g->host.n();
    out->n_g = g->host.n_g();
    out->R_g = g->st[0].R;
    out->R_L = g->st[1].R;
    memcpy(out->sha256, g->host.sha, 32);
    out->device_bytes = g->device_bytes;
    out->record_bytes = 8;
    out->n_out = g->host.n_out();
    out->R_C = g->st[2].R;
    out->shard_rank = g->shard_rank;
    out->shard_world = g->shard_world;
    out->gen_lo = g->shard_world ? g->lo[0] : 0;
    out->gen_hi = g->shard_world ? g->hi[0] : g->host.n_g();
    out->comm_lo = g->shard_world ? g->lo[1] : 0;
    out->comm_hi = g->shard_world ? g->hi[1] : g->host.n();
    return set_ok();
}

cut_status cut_graph_outside_labels(const cut_graph *g, uint64_t *out) {
    if (!g || !out) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_outside_labels: null argument");
    memcpy(out, g->host.out_labels.data(), g->host.out_labels.size() * 8);
    return set_ok();
}

cut_status cut_rhs_outside(const cut_graph *g, const double *h, int n_obs, const double *x, double *c,
                           cut_stream_t stream) {
    TraceRange trace_("cut_rhs_outside");
    if (whole_graph(g, "cut_rhs_outside") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || !c || n_obs < 0 || n_obs > 63 || (n_obs > 0 && !x))
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_outside: bad argument");
    if (g->host.n_out() == 0)
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_outside: the graph was built without diagnostics");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n(), nout = g->host.n_out();
    double *xi = nullptr;
    CUDA_TRY(scratch_alloc(&xi, std::max<int64_t>(1, g->host.n_g()) * 8, s));
    launch_gen(g, h, xi, s, nullptr);
    const double *xs[64];
    double *cs[64];
    xs[0] = h;
    cs[0] = c;
    for (int o = 0; o < n_obs; o++) { xs[o + 1] = x + o * n; cs[o + 1] = c + (o + 1) * nout; }
    launch_comm(g, xi, n_obs + 1, xs, cs, s, nullptr, 2);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaFreeAsync(xi, s));
    return set_ok();
}

cut_status cut_graph_labels(const cut_graph *g, uint64_t *labels, uint64_t *gen_labels, uint8_t *diag) {
    if (!g) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_labels: null graph");
    if (labels) memcpy(labels, g->host.labels.data(), g->host.labels.size() * 8);
    if (gen_labels) memcpy(gen_labels, g->host.gen_labels.data(), g->host.gen_labels.size() * 8);
    if (diag) memcpy(diag, g->host.diag.data(), g->host.diag.size());
    return set_ok();
}

cut_status cut_graph_weights(const cut_graph *g, int32_t *num, int32_t *den) {
    if (!g) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_weights: null graph");
    if (num) memcpy(num, g->host.num.data(), g->host.num.size() * 4);
    if (den) memcpy(den, g->host.den.data(), g->host.den.size() * 4);
    return set_ok();
}

cut_status cut_graph_records(const cut_graph *g, int stage, int64_t *row_ptr, int32_t *in1, int32_t *in2,
                             uint8_t *code) {
    if (!g || stage < 0 || stage > 2) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_records: bad argument");
    const auto &rp = g->host.rp[stage];
    const auto &rc = g->host.rec[stage];
    if (rc.size() / 2 != (size_t)g->st[stage].R)
        return set_error(CUT_ERR_UNSUPPORTED, "cut_graph_records: host copy of the records was released");
    if (row_ptr) for (size_t r = 0; r < rp.size(); r++) row_ptr[r] = (int64_t)rp[r];
    for (size_t e = 0; e < rc.size() / 2; e++) {
        if (in1) in1[e] = (int32_t)(rc[2 * e] & kIndexMask);
        if (in2) in2[e] = (int32_t)rc[2 * e + 1];
        if (code) code[e] = (uint8_t)(rc[2 * e] >> kIndexBits);
    }
    return set_ok();
}

cut_status cut_rhs(const cut_graph *g, const double *h, int n_obs, const double *x, double *dh, double *dx,
                   double *xi_out, cut_stream_t stream) {
    TraceRange trace_("cut_rhs");
    if (whole_graph(g, "cut_rhs") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || !dh || n_obs < 0 || n_obs > 63 || (n_obs > 0 && (!x || !dx)))
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs: bad argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n();
    double *xi = xi_out;
    if (!xi) CUDA_TRY(scratch_alloc(&xi, std::max<int64_t>(1, g->host.n_g()) * 8, s));
    void *df = nullptr;
    CUDA_TRY(scratch_alloc(&df, operand_scratch_bytes(g), s));
    const double *xs[64];
    double *dxs[64];
    xs[0] = h;
    dxs[0] = dh;
    for (int o = 0; o < n_obs; o++) { xs[o + 1] = x + o * n; dxs[o + 1] = dx + o * n; }
    float2 *X2 = operand_blocks(g, df);
    const bool packed = launch_gen_pack(g, xs, n_obs + 1, xi, reinterpret_cast<double *>(X2), s, nullptr);
    apply_L(g, xi, (float2 *)df, X2, n_obs + 1, xs, dxs, s, nullptr, packed);
    CUDA_TRY(cudaGetLastError());
    if (!xi_out) CUDA_TRY(cudaFreeAsync(xi, s));
    if (df) CUDA_TRY(cudaFreeAsync(df, s));
    return set_ok();
}

cut_status cut_graph_set_arithmetic(cut_graph *g, int arith) {
    if (!g || (arith != CUT_ARITH_FP64 && arith != CUT_ARITH_DF64))
        return set_error(CUT_ERR_INVALID_ARG, "cut_graph_set_arithmetic: unknown arithmetic");
    if (arith == CUT_ARITH_DF64 && !g->wuniform)
        return set_error(CUT_ERR_UNSUPPORTED, "cut_graph_set_arithmetic: double-float needs factors of one magnitude");
    g->arith = arith;
    return set_ok();
}

cut_status cut_apply_L(const cut_graph *g, const double *xi, int n_ops, const double *x, double *dx,
                       cut_stream_t stream) {
    TraceRange trace_("cut_apply_L");
    if (whole_graph(g, "cut_apply_L") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !xi || n_ops < 1 || n_ops > 64 || !x || !dx)
        return set_error(CUT_ERR_INVALID_ARG, "cut_apply_L: bad argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n();
    void *df = nullptr;
    CUDA_TRY(scratch_alloc(&df, operand_scratch_bytes(g), s));
    const double *xs[64];
    double *dxs[64];
    for (int o = 0; o < n_ops; o++) { xs[o] = x + o * n; dxs[o] = dx + o * n; }
    apply_L(g, xi, (float2 *)df, operand_blocks(g, df), n_ops, xs, dxs, s, nullptr);
    CUDA_TRY(cudaGetLastError());
    if (df) CUDA_TRY(cudaFreeAsync(df, s));
    return set_ok();
}

}  // extern "C"

// ----------------------------------------------------------------- assembly
extern "C" cut_status cut_assemble(int n_src, int64_t n, const double *X, int n_out, const double *C, double *out,
                                   cut_stream_t stream) {
    TraceRange trace_("cut_assemble");
    if (n_src < 1 || n_src > 3000 || n < 1 || n_out < 1 || !X || !C || !out)
        return set_error(CUT_ERR_INVALID_ARG, "cut_assemble: bad argument (1 <= n_src <= 3000)");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = (size_t)n_src * 32 * 8;
    if (smem > 48 * 1024)
        CUDA_TRY(cudaFuncSetAttribute(k::assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = (n + 31) / 32;
    pdl_launch(k::assemble, (unsigned)blocks, 256, smem, s, X, n_src, n, C, n_out, out);
    CUDA_TRY(cudaGetLastError());
    return set_ok();
}

// ----------------------------------------------------------------- tangent
extern "C" cut_status cut_rhs_jvp(const cut_graph *g, const double *h, int n_obs, const double *x, const double *dh,
                                  const double *dx, double *out_h, double *out_x, cut_stream_t stream) {
    TraceRange trace_("cut_rhs_jvp");
    if (whole_graph(g, "cut_rhs_jvp") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || !dh || !out_h || n_obs < 0 || n_obs > 63 ||
        (n_obs > 0 && (!x || !dx || !out_x)))
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_jvp: bad argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n(), ng = std::max<int64_t>(1, g->host.n_g());
    double *buf = nullptr;
    CUDA_TRY(scratch_alloc(&buf, 2 * ng * 8, s));
    double *xi = buf, *dxi = buf + ng;
    const k::Weights w = weights_of(g);
    launch_gen(g, h, xi, s, nullptr);
    const DevCSR &c0 = g->st[0], &c1 = g->st[1];
    pdl_launch(k::gen_jvp, grid_for_rows(c0.rows), k::kBlock, 0, s, c0.rp, c0.rec, w, h, dh, dxi, c0.rows);
    const int nops = n_obs + 1;
    const double *xs[64], *dxs[64];
    double *outs[64];
    xs[0] = h;
    dxs[0] = dh;
    outs[0] = out_h;
    for (int o = 0; o < n_obs; o++) { xs[o + 1] = x + o * n; dxs[o + 1] = dx + o * n; outs[o + 1] = out_x + o * n; }
    for (int o0 = 0; o0 < nops; o0 += 4) {
        const int m = std::min(4, nops - o0);
        switch (m) {
#define CASE(M)                                                                                     \
    case M: {                                                                                       \
        k::TanOps<M> t;                                                                             \
        for (int u = 0; u < M; u++) { t.x[u] = xs[o0 + u]; t.dx[u] = dxs[o0 + u]; t.out[u] = outs[o0 + u]; } \
        pdl_launch(k::comm_jvp<M>, grid_for_rows(c1.rows), k::kBlock, 0, s, c1.rp, c1.rec, w, xi, dxi, t, c1.rows); \
    } break;
            CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
        }
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaFreeAsync(buf, s));
    return set_ok();
}

// ----------------------------------------------------------------- adjoint
namespace cut {

// Counting sort of records into a new CSR keyed by `row_of(e)`, payload
// (code | first(e), second(e)).  The input rows are split into T contiguous
// blocks, one host thread each: counts per (block, output row), then every
// block writes its records after those of the blocks before it, so each
// output row lists its records in input order, as a sequential pass would.
template <class RowF, class AF, class BF>
static void transpose(const std::vector<uint64_t> &rp, const std::vector<uint32_t> &rec, int64_t rows_out,
                      RowF row_of, AF first, BF second, std::vector<uint64_t> &orp,
                      std::vector<uint32_t> &orec) {
    const int64_t rows_in = (int64_t)rp.size() - 1;
    const uint64_t R = rows_in > 0 ? rp[rows_in] : 0;
    int T = (int)std::min<uint64_t>(std::max(1u, std::thread::hardware_concurrency()), 16);
    if (R < (1u << 20)) T = 1;
    std::vector<int64_t> blk(T + 1);
    blk[0] = 0;
    for (int t = 1; t < T; t++)
        blk[t] = std::max(blk[t - 1], (int64_t)(std::lower_bound(rp.begin(), rp.end(), R * t / T) - rp.begin()));
    blk[T] = rows_in;
    std::vector<std::vector<uint64_t>> cnt(T, std::vector<uint64_t>(rows_out + 1, 0));
    auto par = [&](auto fn) {
        std::vector<std::thread> th;
        for (int t = 0; t < T; t++) th.emplace_back(fn, t);
        for (auto &x : th) x.join();
    };
    par([&](int t) {
        auto &c = cnt[t];
        for (int64_t r = blk[t]; r < std::min(blk[t + 1], rows_in); r++)
            for (uint64_t e = rp[r]; e < rp[r + 1]; e++) c[row_of(r, rec[2 * e], rec[2 * e + 1])]++;
    });
    // offsets: output row major, block minor
    orp.assign(rows_out + 1, 0);
    uint64_t acc = 0;
    for (int64_t o = 0; o < rows_out; o++) {
        orp[o] = acc;
        for (int t = 0; t < T; t++) {
            const uint64_t c = cnt[t][o];
            cnt[t][o] = acc;
            acc += c;
        }
    }
    orp[rows_out] = acc;
    orec.assign(rec.size(), 0);
    par([&](int t) {
        auto &cur = cnt[t];
        for (int64_t r = blk[t]; r < std::min(blk[t + 1], rows_in); r++)
            for (uint64_t e = rp[r]; e < rp[r + 1]; e++) {
                const uint32_t w0 = rec[2 * e], w1 = rec[2 * e + 1];
                const uint64_t p = cur[row_of(r, w0, w1)]++;
                orec[2 * p] = ((w0 >> kIndexBits) << kIndexBits) | first(r, w0, w1);
                orec[2 * p + 1] = second(r, w0, w1);
            }
    });
}

// Rows much longer than the mean keep one lane group busy long after the
// others finish.  Split every row of more than kSplitAbove records into
// pieces of about kPiece records: the kernels sum pieces like rows, and
// piece_reduce adds the pieces of each row in order (fixed sum order).
constexpr uint64_t kSplitAbove = 2048, kPiece = 1024;

static cut_status upload_split(DevCSR &d, const std::vector<uint64_t> &rp, const std::vector<uint32_t> &rc,
                               int64_t &bytes) {
    const int64_t rows = (int64_t)rp.size() - 1;
    std::vector<uint64_t> vrp{0}, vr(rows + 1);
    for (int64_t r = 0; r < rows; r++) {
        vr[r] = vrp.size() - 1;
        const uint64_t b = rp[r], len = rp[r + 1] - b;
        const uint64_t np = len > kSplitAbove ? (len + kPiece - 1) / kPiece : 1;
        for (uint64_t q = 1; q <= np; q++) vrp.push_back(b + len * q / np);
    }
    vr[rows] = vrp.size() - 1;
    cut_status st = upload_csr(d, vrp, rc, bytes);
    if (st != CUT_OK) return st;
    d.real_rows = rows;
    CUDA_TRY(cudaMalloc(&d.vr, vr.size() * 8));
    CUDA_TRY(cudaMemcpy(d.vr, vr.data(), vr.size() * 8, cudaMemcpyHostToDevice));
    bytes += (int64_t)vr.size() * 8;
    return CUT_OK;
}

// Sort the records of every row by (first input, second input), rows split
// over host threads (the order is fixed, so the sums stay reproducible).
static void sort_rows_by_first(const std::vector<uint64_t> &rp, std::vector<uint32_t> &rc) {
    const int64_t rows = (int64_t)rp.size() - 1;
    const int T = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16);
    std::vector<std::thread> th;
    for (int t = 0; t < T; t++)
        th.emplace_back([&, t]() {
            std::vector<uint64_t> key;
            for (int64_t r = t; r < rows; r += T) {
                const uint64_t b = rp[r], e = rp[r + 1];
                key.resize(e - b);
                for (uint64_t q = b; q < e; q++)
                    key[q - b] = ((uint64_t)(rc[2 * q] & kIndexMask) << 32 | rc[2 * q + 1]) << 8 |
                                 (rc[2 * q] >> kIndexBits);
                std::sort(key.begin(), key.end());
                for (uint64_t q = b; q < e; q++) {
                    const uint64_t k2 = key[q - b];
                    rc[2 * q] = (uint32_t)((k2 & 0xff) << kIndexBits) | (uint32_t)(k2 >> 40);
                    rc[2 * q + 1] = (uint32_t)((k2 >> 8) & 0xffffffffu);
                }
            }
        });
    for (auto &x : th) x.join();
}

static cut_status ensure_transposes(cut_graph *g) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->have_T) return CUT_OK;
    const auto &H = g->host;
    const int64_t n = H.n(), ng = H.n_g();
    std::vector<uint64_t> rp;
    std::vector<uint32_t> rc;
    int64_t bytes = 0;
    // rows j, entries (code|a, k), each row sorted by (a, k) like the forward
    // rows, so that neighbouring lanes gather neighbouring generator entries
    transpose(H.rp[1], H.rec[1], n, [](int64_t, uint32_t, uint32_t w1) { return (int64_t)w1; },
              [](int64_t, uint32_t w0, uint32_t) { return w0 & kIndexMask; },
              [](int64_t k, uint32_t, uint32_t) { return (uint32_t)k; }, rp, rc);
    sort_rows_by_first(rp, rc);
    cut_status st = upload_split(g->tx, rp, rc, bytes);
    if (st != CUT_OK) return st;
    // rows a, entries (code|k, j)
    transpose(H.rp[1], H.rec[1], ng, [](int64_t, uint32_t w0, uint32_t) { return (int64_t)(w0 & kIndexMask); },
              [](int64_t k, uint32_t, uint32_t) { return (uint32_t)k; },
              [](int64_t, uint32_t, uint32_t w1) { return w1; }, rp, rc);
    st = upload_split(g->txi, rp, rc, bytes);
    if (st != CUT_OK) return st;
    // rows r (both inputs of a generator record), entries (code|a, partner)
    {
        std::vector<uint64_t> orp(n + 1, 0);
        const auto &grp = H.rp[0];
        const auto &grc = H.rec[0];
        for (int64_t a = 0; a < ng; a++)
            for (uint64_t e = grp[a]; e < grp[a + 1]; e++) {
                orp[(grc[2 * e] & kIndexMask) + 1]++;
                orp[grc[2 * e + 1] + 1]++;
            }
        for (int64_t r = 0; r < n; r++) orp[r + 1] += orp[r];
        std::vector<uint64_t> cur(orp.begin(), orp.end() - 1);
        std::vector<uint32_t> orc(2 * orp[n]);
        for (int64_t a = 0; a < ng; a++)
            for (uint64_t e = grp[a]; e < grp[a + 1]; e++) {
                uint32_t w0 = grc[2 * e], w1 = grc[2 * e + 1];
                uint32_t code = w0 >> kIndexBits, i = w0 & kIndexMask, j = w1;
                uint64_t p = cur[i]++;
                orc[2 * p] = (code << kIndexBits) | (uint32_t)a;
                orc[2 * p + 1] = j;
                p = cur[j]++;
                orc[2 * p] = (code << kIndexBits) | (uint32_t)a;
                orc[2 * p + 1] = i;
            }
        st = upload_split(g->th, orp, orc, bytes);
        if (st != CUT_OK) return st;
    }
    g->device_bytes += bytes;
    g->have_T = true;
    return CUT_OK;
}

// X4[j][4 NB] = Y[o][j] for the nops (<= 8) operands of a stacked vector
static void pack_operands(const cut_graph *g, const double *Y, int nops, double *X4, cudaStream_t s) {
    const int64_t n = g->host.n();
    switch (nops) {
#define CASE(M)                                                                       \
    case M: {                                                                         \
        k::Ops<M> ops;                                                                \
        for (int t = 0; t < M; t++) { ops.x[t] = Y + t * n; ops.dx[t] = nullptr; }      \
        pdl_launch(k::pack_x4<M>, grid_for_len(n), 256, 0, s, ops, n, X4, nullptr);           \
    } break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
}

// bytes of the packed adjoint scratch: two blocks of n x 64 bytes, 32-byte aligned
// operand blocks (two of n x 64 bytes) and the piece sums of the split
// transposed passes (up to 8 operands)
static size_t adjoint_scratch_bytes(const cut_graph *g) {
    const int64_t pieces = std::max(std::max(g->tx.rows, g->txi.rows), g->th.rows);
    return (size_t)g->host.n() * 128 + (size_t)pieces * 64 + 128;
}

// VJP of the stacked RHS at Y with cotangent W: YB = J(Y)^T W.  xi, xib:
// scratch [n_g]; xbar0: scratch [n]; pk: adjoint_scratch_bytes(g) of scratch
// (packed operand blocks and the piece sums of split rows).
static void stacked_vjp(const cut_graph *g, const double *Y, const double *W, double *YB, int nops, double *xi,
                        double *xib, double *xbar0, cudaStream_t s, void *pk) {
    const int64_t n = g->host.n(), ng = g->host.n_g();
    const int nc = (int)g->host.num.size();
    launch_gen(g, Y, xi, s, nullptr);
    if (nops <= 8) {
        // operand transposes: x_bar_o[j] = sum beta xi[a] w_o[k] is the forward
        // commutator's form over the rows-by-j records (W packed into W4)
        double *W4 = reinterpret_cast<double *>(((uintptr_t)pk + 31) & ~(uintptr_t)31);
        double *X4 = W4 + 8 * n;
        double *piece = X4 + 8 * n;   // piece sums [nops][pieces]
        const double *ws[8];
        double *xb[8];
        const int64_t ptx = g->tx.rows;
        for (int o = 0; o < nops; o++) { ws[o] = W + o * n; xb[o] = piece + o * ptx; }
        launch_comm(g, xi, nops, ws, xb, s, nullptr, 1, W4, &g->tx);
        {
            k::Ops<8> red;
            for (int o = 0; o < nops; o++) { red.x[o] = piece + o * ptx; red.dx[o] = o == 0 ? xbar0 : YB + o * n; }
            pdl_launch(k::piece_reduce, grid_for_len(n * nops), 256, 0, s, g->tx.vr, n, red, nops, nullptr);
        }
        pack_operands(g, Y, nops, X4, s);
        const k::Weights w = weights_of(g);
        const DevCSR &cx = g->txi, &ch = g->th;
        const int lx = comm_lanes(cx.rows), lh = gen_lanes(ch.rows);
        double *xpiece = piece, *hpiece = piece + std::max<int64_t>(cx.rows, 1);
        switch (nops) {
#define CASE(M)                                                                                                 \
    case M:                                                                                                     \
        if (w.uniform) {                                                                                        \
            if (lx == 8) pdl_launch(k::commT_xi_x4<M, true, 8>, grid_for_groups(cx.rows, 8), k::kBlock, 0, s, cx.rp, cx.rec, w, W4, X4, xpiece, cx.rows); \
            else pdl_launch(k::commT_xi_x4<M, true, 32>, grid_for_groups(cx.rows, 32), k::kBlock, 0, s, cx.rp, cx.rec, w, W4, X4, xpiece, cx.rows); \
        } else {                                                                                                \
            if (lx == 8) pdl_launch(k::commT_xi_x4<M, false, 8>, grid_for_groups(cx.rows, 8), k::kBlock, 0, s, cx.rp, cx.rec, w, W4, X4, xpiece, cx.rows); \
            else pdl_launch(k::commT_xi_x4<M, false, 32>, grid_for_groups(cx.rows, 32), k::kBlock, 0, s, cx.rp, cx.rec, w, W4, X4, xpiece, cx.rows); \
        }                                                                                                       \
        break;
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        }
        {
            k::Ops<8> red;
            red.x[0] = xpiece;
            red.dx[0] = xib;
            pdl_launch(k::piece_reduce, grid_for_len(ng), 256, 0, s, cx.vr, ng, red, 1, nullptr);
        }
        // the rows of the diagonal coordinates hold most of the generator
        // records (every generator record has one diagonal input) and are
        // split into pieces like the other transposed orders
        // a whole warp per piece: each record here is two dependent gathers
        // and one FMA, so a lane's chain of records is all latency
        (void)lh;
        if (w.uniform)
            pdl_launch(k::genT_lanes<true, 32>, grid_for_groups(ch.rows, 32), k::kBlock, 0, s, ch.rp, ch.rec, w, xib, Y, nullptr, hpiece, ch.rows);
        else
            pdl_launch(k::genT_lanes<false, 32>, grid_for_groups(ch.rows, 32), k::kBlock, 0, s, ch.rp, ch.rec, w, xib, Y, nullptr, hpiece, ch.rows);
        {
            k::Ops<8> red;
            red.x[0] = hpiece;
            red.dx[0] = YB;
            pdl_launch(k::piece_reduce, grid_for_len(n), 256, 0, s, ch.vr, n, red, 1, xbar0);
        }
        return;
    }
    // more than eight operands: one gather per operand, four operands per
    // pass, over the same pieces
    double *piece = reinterpret_cast<double *>(((uintptr_t)pk + 31) & ~(uintptr_t)31) + 16 * n;
    const int64_t ptx = g->tx.rows, pxi = g->txi.rows, pth = g->th.rows;
    for (int o0 = 0; o0 < nops; o0 += 4) {
        int m = std::min(4, nops - o0);
        switch (m) {
#define CASE(M)                                                                              \
    case M: {                                                                                \
        k::Ops<M> ops;                                                                       \
        for (int t = 0; t < M; t++) { ops.x[t] = W + (o0 + t) * n; ops.dx[t] = piece + t * ptx; } \
        pdl_launch(k::commT_x<M>, grid_for_rows(ptx), k::kBlock, 0, s, g->tx.rp, g->tx.rec, g->wtab, nc, xi, ops, ptx); \
    } break;
            CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
        }
        k::Ops<8> red;
        for (int t = 0; t < m; t++) {
            red.x[t] = piece + t * ptx;
            red.dx[t] = (o0 + t == 0) ? xbar0 : YB + (o0 + t) * n;
        }
        pdl_launch(k::piece_reduce, grid_for_len(n * m), 256, 0, s, g->tx.vr, n, red, m, nullptr);
    }
    for (int o0 = 0; o0 < nops; o0 += 4) {
        int m = std::min(4, nops - o0);
        switch (m) {
#define CASE(M)                                                                              \
    case M: {                                                                                \
        k::Pairs<M> pr;                                                                      \
        for (int t = 0; t < M; t++) { pr.x[t] = Y + (o0 + t) * n; pr.w[t] = W + (o0 + t) * n; } \
        pdl_launch(k::commT_xi<M>, grid_for_rows(pxi), k::kBlock, 0, s, g->txi.rp, g->txi.rec, g->wtab, nc, pr, piece, pxi, o0 > 0); \
    } break;
            CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
        }
    }
    {
        k::Ops<8> red;
        red.x[0] = piece;
        red.dx[0] = xib;
        pdl_launch(k::piece_reduce, grid_for_len(ng), 256, 0, s, g->txi.vr, ng, red, 1, nullptr);
    }
    pdl_launch(k::genT, grid_for_rows(pth), k::kBlock, 0, s, g->th.rp, g->th.rec, g->wtab, nc, xib, Y, nullptr, piece, pth);
    {
        k::Ops<8> red;
        red.x[0] = piece;
        red.dx[0] = YB;
        pdl_launch(k::piece_reduce, grid_for_len(n), 256, 0, s, g->th.vr, n, red, 1, xbar0);
    }
}

}  // namespace cut

extern "C" cut_status cut_rhs_adjoint(const cut_graph *g, const double *h, int n_obs, const double *x,
                                      const double *w_h, const double *w_x, double *h_bar, double *x_bar,
                                      cut_stream_t stream) {
    TraceRange trace_("cut_rhs_adjoint");
    if (whole_graph(g, "cut_rhs_adjoint") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || !w_h || !h_bar || n_obs < 0 || n_obs > 63 || (n_obs > 0 && (!x || !w_x || !x_bar)))
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_adjoint: bad argument");
    DeviceGuard dg(g->device);
    cut_status st = ensure_transposes(const_cast<cut_graph *>(g));
    if (st != CUT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n(), ng = std::max<int64_t>(1, g->host.n_g());
    const int nops = n_obs + 1;
    // stacked copies so that one code path serves single calls and flows
    double *buf = nullptr;
    const size_t L = (size_t)nops * n;
    CUDA_TRY(scratch_alloc(&buf, (3 * L + 2 * ng + n) * 8 + adjoint_scratch_bytes(g), s));
    double *Y = buf, *W = buf + L, *YB = buf + 2 * L, *xi = buf + 3 * L, *xib = xi + ng, *xb0 = xib + ng;
    void *pk = xb0 + n;
    CUDA_TRY(cudaMemcpyAsync(Y, h, n * 8, cudaMemcpyDeviceToDevice, s));
    if (n_obs) CUDA_TRY(cudaMemcpyAsync(Y + n, x, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(W, w_h, n * 8, cudaMemcpyDeviceToDevice, s));
    if (n_obs) CUDA_TRY(cudaMemcpyAsync(W + n, w_x, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s));
    stacked_vjp(g, Y, W, YB, nops, xi, xib, xb0, s, pk);
    CUDA_TRY(cudaMemcpyAsync(h_bar, YB, n * 8, cudaMemcpyDeviceToDevice, s));
    if (n_obs) CUDA_TRY(cudaMemcpyAsync(x_bar, YB + n, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaFreeAsync(buf, s));
    return set_ok();
}

// ----------------------------------------------------------------- flows
namespace cut {

static const double RK4_A[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
static const double RK4_B[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
// Dormand & Prince (1980) 5(4) tableau
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_BS[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                                1.0 / 40};

struct FlowWork {
    double *Y, *U, *Y5, *K[7], *xi;
    k::Control *ctl;
    double *replay, *record;
    int *flag;
    void *df = nullptr;            // commutator operand scratch (or null)
    void *base = nullptr;
};

static cut_status alloc_work(FlowWork &w, int64_t L, int64_t ng, int64_t nrec, cudaStream_t s,
                             size_t df_bytes = 0) {
    size_t doubles = (size_t)(3 + 7) * L + ng + 2 * nrec + 64 + df_bytes / 8 + 1;
    size_t bytes = doubles * 8 + sizeof(k::Control) + 64;
    CUDA_TRY(scratch_alloc(&w.base, bytes, s));
    double *p = (double *)w.base;
    w.Y = p; p += L;
    w.U = p; p += L;
    w.Y5 = p; p += L;
    for (int i = 0; i < 7; i++) { w.K[i] = p; p += L; }
    w.xi = p; p += std::max<int64_t>(1, ng);
    w.replay = p; p += nrec;
    w.record = p; p += nrec;
    w.flag = (int *)p; p += 8;
    w.df = df_bytes ? (void *)p : nullptr;
    p += df_bytes / 8 + 1;
    w.ctl = (k::Control *)p;
    return CUT_OK;
}

// U = Y + ds sum_j A[i][j] K_j
static void stage_input(const FlowWork &w, const double *A, int i, int64_t L, const double *dsp, double dsc,
                        cudaStream_t s, const int *done, double *out) {
    k::Combine cb;
    cb.base = w.Y;
    cb.nk = 0;
    for (int j = 0; j < i; j++)
        if (A[j] != 0.0) { cb.K[cb.nk] = w.K[j]; cb.c[cb.nk] = A[j]; cb.nk++; }
    pdl_launch(k::rk_combine, grid_for_len(L), 256, 0, s, cb, out, L, dsp, dsc, done);
}

// K_i = f(Y + ds sum_j A[j] K_j): the stage input, its packed operand
// blocks and the generator in one launch (stage_gen), then the commutator
// stage over the packed blocks; U_full (may be null) keeps the stage input.
// The fused generator forms each of a record's two inputs as Y + sum c K
// (1 + nk loads instead of 1), which only pays where the launches it saves
// dominate: a generator stage of at most kFuseGenRecords records (8-orbital
// model, 4.6e3 records: 15.7 us per right-hand side fused against 18.5 us;
// the 16-orbital stress graph, 3.5e6 records: 48 us per RK4 stage fused
// against 36 us separate).  Larger graphs, double-float arithmetic, more
// than eight operands or no operand scratch take the separate combination
// and right-hand-side launches.  Same bits either way.
constexpr int64_t kFuseGenRecords = 1 << 16;
static void fused_stage(const cut_graph *g, FlowWork &w, const double *A, int i, int nops, const double *dsp,
                        double dsc, cudaStream_t s, const int *done, double *U_full, double *Kout) {
    const int64_t n = g->host.n(), L = (int64_t)nops * n;
    double *X4 = reinterpret_cast<double *>(operand_blocks(g, w.df));
    if (g->arith != CUT_ARITH_FP64 || nops > 8 || !X4 || g->st[0].R > kFuseGenRecords) {
        double *U = U_full ? U_full : w.U;
        const double *in = w.Y;
        if (i > 0) {
            stage_input(w, A, i, L, dsp, dsc, s, done, U);
            in = U;
        } else if (U_full) {
            stage_input(w, A, 0, L, dsp, dsc, s, done, U);
        }
        stacked_rhs(g, in, Kout, nops, w.xi, s, done, w.df);
        return;
    }
    k::StageIn si;
    si.base = w.Y;
    si.nk = 0;
    for (int j = 0; j < i; j++)
        if (A[j] != 0.0) { si.K[si.nk] = w.K[j]; si.c[si.nk] = A[j]; si.nk++; }
    si.ds_ptr = dsp;
    si.ds_const = dsc;
    const DevCSR &c0 = g->st[0];
    const k::Weights wt = weights_of(g);
    const int gl = gen_lanes(c0.lane_rows);
    const int grid = std::max(grid_for_len(n), grid_for_groups(c0.rows, gl));
    switch (nops * 4 + (wt.uniform ? 2 : 0) + (gl == 4 ? 1 : 0)) {
#define CASE(M)                                                                                                 \
    case M * 4 + 0: pdl_launch(k::stage_gen<M, false, 8>, grid, k::kBlock, 0, s, si, n, X4, U_full, c0.rp, c0.rec, wt, w.xi, c0.rows, done); break; \
    case M * 4 + 1: pdl_launch(k::stage_gen<M, false, 4>, grid, k::kBlock, 0, s, si, n, X4, U_full, c0.rp, c0.rec, wt, w.xi, c0.rows, done); break; \
    case M * 4 + 2: pdl_launch(k::stage_gen<M, true, 8>, grid, k::kBlock, 0, s, si, n, X4, U_full, c0.rp, c0.rec, wt, w.xi, c0.rows, done); break; \
    case M * 4 + 3: pdl_launch(k::stage_gen<M, true, 4>, grid, k::kBlock, 0, s, si, n, X4, U_full, c0.rp, c0.rec, wt, w.xi, c0.rows, done); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    const double *xs[8];
    double *dxs[8];
    for (int o = 0; o < nops; o++) { xs[o] = nullptr; dxs[o] = Kout + o * n; }
    launch_comm(g, w.xi, nops, xs, dxs, s, done, 1, X4, nullptr, piece_area(g, reinterpret_cast<float2 *>(X4)), true);
}

// One RK4 step on w.Y (fixed ds), K/U scratch.
static void rk4_step(const cut_graph *g, FlowWork &w, int nops, double ds, cudaStream_t s) {
    const int64_t L = (int64_t)nops * g->host.n();
    for (int i = 0; i < 4; i++) fused_stage(g, w, RK4_A[i], i, nops, nullptr, ds, s, nullptr, nullptr, w.K[i]);
    k::Combine cb;
    cb.base = w.Y;
    cb.nk = 4;
    for (int j = 0; j < 4; j++) { cb.K[j] = w.K[j]; cb.c[j] = RK4_B[j]; }
    pdl_launch(k::rk_combine, grid_for_len(L), 256, 0, s, cb, w.Y, L, nullptr, ds, nullptr);
}

// One Dormand-Prince attempt under device control (w.K[0] holds f(Y)).
static void dp_attempt(const cut_graph *g, FlowWork &w, int nops, cudaStream_t s, bool replay,
                       int64_t record_cap) {
    const int64_t L = (int64_t)nops * g->host.n();
    const int *done = &w.ctl->done;
    const double *dsp = &w.ctl->ds;
    for (int i = 1; i < 6; i++) fused_stage(g, w, DP_A[i], i, nops, dsp, 0.0, s, done, nullptr, w.K[i]);
    fused_stage(g, w, DP_A[6], 6, nops, dsp, 0.0, s, done, w.Y5, w.K[6]);
    if (!replay) {
        k::ErrTerms et;
        for (int i = 0; i < 7; i++) { et.K[i] = w.K[i]; et.e[i] = DP_B[i] - DP_BS[i]; }
        pdl_launch(k::dp_error, grid_for_len(L), 256, 0, s, et, w.Y, w.Y5, L, w.ctl);
    }
    pdl_launch(k::dp_control, 1, 1, 0, s, w.ctl, replay ? w.replay : nullptr, w.record, record_cap);
    pdl_launch(k::dp_accept, grid_for_len(L), 256, 0, s, w.ctl, w.Y, w.Y5, w.K[0], w.K[6], L);
}

struct StreamPair {
    cudaStream_t user, work;
    cudaEvent_t ev;
};

static cut_status begin_work(StreamPair &sp) {
    CUDA_TRY(cudaStreamCreateWithFlags(&sp.work, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&sp.ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(sp.ev, sp.user));
    CUDA_TRY(cudaStreamWaitEvent(sp.work, sp.ev, 0));
    return CUT_OK;
}
static void end_work(StreamPair &sp) {
    cudaEventRecord(sp.ev, sp.work);
    cudaStreamWaitEvent(sp.user, sp.ev, 0);
    cudaStreamDestroy(sp.work);
    cudaEventDestroy(sp.ev);
}

// Capture `body` into a graph once and replay it `times` times.
template <class F>
static cut_status replay_graph(cudaStream_t s, int64_t times, F body) {
    if (times <= 0) return CUT_OK;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    body();
    CUDA_TRY(cudaStreamEndCapture(s, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    for (int64_t t = 0; t < times; t++) {
        e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) break;
    }
    cudaGraphExecDestroy(exec);
    CUDA_TRY(e);
    return CUT_OK;
}

static cut_status check_opts(const cut_flow_opts *o) {
    if (!o) return set_error(CUT_ERR_INVALID_ARG, "flow: null options");
    if (o->method != CUT_RK4 && o->method != CUT_DP45) return set_error(CUT_ERR_INVALID_ARG, "flow: unknown method");
    if (!(o->s1 >= o->s0) || !std::isfinite(o->s0) || !std::isfinite(o->s1))
        return set_error(CUT_ERR_INVALID_ARG, "flow: need finite s1 >= s0");
    if (o->method == CUT_RK4 && !(o->ds > 0)) return set_error(CUT_ERR_INVALID_ARG, "flow: RK4 needs ds > 0");
    if (o->method == CUT_DP45 && !o->replay_steps && (!(o->ds > 0) || !(o->rtol > 0) || o->atol < 0))
        return set_error(CUT_ERR_INVALID_ARG, "flow: DP45 needs ds > 0, rtol > 0, atol >= 0");
    if (o->replay_steps && o->n_replay <= 0) return set_error(CUT_ERR_INVALID_ARG, "flow: empty replay list");
    return CUT_OK;
}

static int64_t rk4_nsteps(const cut_flow_opts *o, double *ds_eff) {
    int64_t N = (int64_t)std::llround((o->s1 - o->s0) / o->ds);
    if (N < 1) N = (o->s1 > o->s0) ? 1 : 0;
    *ds_eff = N > 0 ? (o->s1 - o->s0) / (double)N : 0.0;
    return N;
}

}  // namespace cut

extern "C" cut_status cut_flow(const cut_graph *g, double *h, int n_obs, double *x, const cut_flow_opts *o,
                               cut_flow_stats *stats, cut_stream_t stream) {
    TraceRange trace_("cut_flow");
    if (whole_graph(g, "cut_flow") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || n_obs < 0 || n_obs > 63 || (n_obs > 0 && !x)) return set_error(CUT_ERR_INVALID_ARG, "cut_flow: bad argument");
    cut_status st = check_opts(o);
    if (st != CUT_OK) return st;
    DeviceGuard dg(g->device);
    const int64_t n = g->host.n(), ng = g->host.n_g();
    const int nops = n_obs + 1;
    const int64_t L = (int64_t)nops * n;
    StreamPair sp{(cudaStream_t)stream, nullptr, nullptr};
    st = begin_work(sp);
    if (st != CUT_OK) return st;
    cudaStream_t s = sp.work;
    const bool dp = o->method == CUT_DP45;
    const bool replay = dp && o->replay_steps;
    const int64_t max_steps = o->max_steps > 0 ? o->max_steps : 1000000;
    const int64_t nrec = dp ? (replay ? o->n_replay : std::min<int64_t>(max_steps, 1 << 22)) : 1;
    FlowWork w;
    st = alloc_work(w, L, ng, nrec, s, operand_scratch_bytes(g));
    if (st != CUT_OK) { end_work(sp); return st; }
    auto fail = [&](cut_status e) { cudaFreeAsync(w.base, s); end_work(sp); return e; };
    cudaMemcpyAsync(w.Y, h, n * 8, cudaMemcpyDeviceToDevice, s);
    if (n_obs) cudaMemcpyAsync(w.Y + n, x, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(w.flag, 0, 8, s);
    cut_flow_stats out;
    memset(&out, 0, sizeof(out));
    int status = CUT_OK;
    if (!dp) {
        double ds;
        int64_t N = rk4_nsteps(o, &ds);
        const int64_t chunk = 32;
        st = replay_graph(s, N / chunk, [&]() { for (int t = 0; t < chunk; t++) rk4_step(g, w, nops, ds, s); });
        if (st != CUT_OK) return fail(st);
        for (int64_t t = 0; t < N % chunk; t++) rk4_step(g, w, nops, ds, s);
        pdl_launch(k::scan_nonfinite, grid_for_len(L), 256, 0, s, w.Y, L, w.flag);
        int flag = 0;
        cudaMemcpyAsync(&flag, w.flag, 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(set_error(CUT_ERR_CUDA, std::string("cut_flow: ") + cudaGetErrorString(e)));
        if (flag) status = CUT_ERR_NONFINITE;
        out.steps = N;
        out.rhs_calls = 4 * N;
        out.s_final = o->s0 + ds * (double)N;
        out.ds_next = ds;
        out.finished = 1;
    } else {
        k::Control c;
        memset(&c, 0, sizeof(c));
        c.s = o->s0;
        c.s1 = o->s1;
        c.rtol = o->rtol;
        c.atol = o->atol;
        c.max_steps = max_steps;
        c.pause_after = replay ? 0 : std::max<int64_t>(0, o->pause_after);
        c.n_replay = replay ? o->n_replay : 0;
        c.ds = replay ? o->replay_steps[0] : std::min(o->ds, o->s1 - o->s0);
        c.done = (replay || o->s1 > o->s0) ? 0 : 1;
        cudaMemcpyAsync(w.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, s);
        if (replay) cudaMemcpyAsync(w.replay, o->replay_steps, o->n_replay * 8, cudaMemcpyHostToDevice, s);
        stacked_rhs(g, w.Y, w.K[0], nops, w.xi, s, nullptr, w.df);
        const int64_t chunk = 16;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(set_error(CUT_ERR_CUDA, "cut_flow: capture failed"));
        for (int t = 0; t < chunk; t++) dp_attempt(g, w, nops, s, replay, nrec);
        e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess) return fail(set_error(CUT_ERR_CUDA, "cut_flow: capture failed"));
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(set_error(CUT_ERR_CUDA, "cut_flow: graph instantiate failed"));
        k::Control hc;
        int64_t attempts_cap = replay ? o->n_replay : max_steps;
        for (int64_t launched = 0;; launched += chunk) {
            cudaGraphLaunch(exec, s);
            cudaMemcpyAsync(&hc, w.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s);
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess || hc.done || launched > attempts_cap + chunk) break;
        }
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fail(set_error(CUT_ERR_CUDA, std::string("cut_flow: ") + cudaGetErrorString(e)));
        status = hc.status;
        if (!hc.done && status == CUT_OK) status = CUT_ERR_MAX_STEPS;
        out.steps = hc.steps;
        out.rejects = hc.rejects;
        out.rhs_calls = 1 + 6 * hc.attempts;
        out.s_final = hc.s;
        out.ds_next = hc.ds;
        out.finished = hc.paused ? 0 : 1;
        if (o->record_steps && o->record_cap > 0) {
            int64_t m = std::min<int64_t>(std::min<int64_t>(hc.steps, o->record_cap), nrec);
            cudaMemcpyAsync(o->record_steps, w.record, m * 8, cudaMemcpyDeviceToHost, s);
        }
    }
    cudaMemcpyAsync(h, w.Y, n * 8, cudaMemcpyDeviceToDevice, s);
    if (n_obs) cudaMemcpyAsync(x, w.Y + n, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(w.base, s);
    cudaError_t e = cudaStreamSynchronize(s);
    end_work(sp);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_flow: ") + cudaGetErrorString(e));
    if (stats) *stats = out;
    if (status != CUT_OK) {
        static const char *names[] = {"", "", "", "", "", "", "", "non-finite state", "step size underflow",
                                      "step limit reached"};
        return set_error((cut_status)status, std::string("cut_flow: ") + (status < 10 ? names[status] : "error"));
    }
    return set_ok();
}

// ----------------------------------------------------------------- flow VJP
extern "C" cut_status cut_flow_vjp(const cut_graph *g, const double *h0, int n_obs, const double *x0,
                                   const cut_flow_opts *o, int checkpoint_every, const double *yb_h,
                                   const double *yb_x, double *gh, double *gx, cut_stream_t stream) {
    TraceRange trace_("cut_flow_vjp");
    if (whole_graph(g, "cut_flow_vjp") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h0 || !yb_h || !gh || n_obs < 0 || n_obs > 63 || (n_obs > 0 && (!x0 || !yb_x || !gx)) ||
        checkpoint_every < 1)
        return set_error(CUT_ERR_INVALID_ARG, "cut_flow_vjp: bad argument");
    cut_status st = check_opts(o);
    if (st != CUT_OK) return st;
    if (o->method == CUT_DP45 && !o->replay_steps)
        return set_error(CUT_ERR_INVALID_ARG, "cut_flow_vjp: DP45 needs the accepted steps in replay_steps");
    DeviceGuard dg(g->device);
    st = ensure_transposes(const_cast<cut_graph *>(g));
    if (st != CUT_OK) return st;
    const int64_t n = g->host.n(), ng = std::max<int64_t>(1, g->host.n_g());
    const int nops = n_obs + 1;
    const int64_t L = (int64_t)nops * n;
    // step list
    std::vector<double> steps;
    const double(*A)[6] = nullptr;
    const double *B = nullptr;
    int S = 0;
    double rkA[4][6] = {{0}};
    if (o->method == CUT_RK4) {
        double ds;
        int64_t N = rk4_nsteps(o, &ds);
        steps.assign(N, ds);
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) rkA[i][j] = RK4_A[i][j];
        A = rkA;
        B = RK4_B;
        S = 4;
    } else {
        steps.assign(o->replay_steps, o->replay_steps + o->n_replay);
        A = DP_A;
        B = DP_B;
        S = 6;
    }
    const int64_t N = (int64_t)steps.size();
    const int64_t C = checkpoint_every;
    const int64_t ncp = (N + C - 1) / C + 1;
    StreamPair sp{(cudaStream_t)stream, nullptr, nullptr};
    st = begin_work(sp);
    if (st != CUT_OK) return st;
    cudaStream_t s = sp.work;
    // memory: checkpoints [ncp][L], segment states [C+1][L], stages U[S][L],
    // K[S][L], kb[S][L], yb, ub, ybn, the fixed step input/output Ycur, Ynext,
    // xi, xib, xb0, the step sizes and the current one, packing scratch
    const size_t dfb = operand_scratch_bytes(g) / 8 + 4, pkb = adjoint_scratch_bytes(g) / 8 + 4;
    double *buf = nullptr;
    size_t tot = (size_t)(ncp + (C + 1) + 3 * S + 5) * L + 2 * ng + n + N + 1 + dfb + pkb;
    cudaError_t e = scratch_alloc(&buf, tot * 8, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        end_work(sp);
        return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_flow_vjp: workspace of " + std::to_string(tot * 8) +
                                                    " bytes: " + cudaGetErrorString(e));
    }
    double *cp = buf, *seg = cp + ncp * L, *U = seg + (C + 1) * L, *K = U + S * L, *KB = K + S * L;
    double *yb = KB + S * L, *ub = yb + L, *ybn = ub + L, *Ycur = ybn + L, *Ynext = Ycur + L;
    double *xi = Ynext + L, *xib = xi + ng, *xb0 = xib + ng, *steps_d = xb0 + n, *dsd = steps_d + N;
    void *df = dsd + 1, *pk = (double *)df + dfb;
    cudaMemcpyAsync(cp, h0, n * 8, cudaMemcpyDeviceToDevice, s);
    if (n_obs) cudaMemcpyAsync(cp + n, x0, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s);
    if (N) cudaMemcpyAsync(steps_d, steps.data(), N * 8, cudaMemcpyHostToDevice, s);
    // out = base + sum c_j (ds K_j) with ds read from the device (*dsd) or given
    auto combine = [&](double *out, const double *base, int nk, const double *const *Ks, const double *cs,
                       const double *dsp, double dsc) {
        k::Combine cb;
        cb.base = base;
        cb.nk = 0;
        for (int j = 0; j < nk; j++)
            if (cs[j] != 0.0) { cb.K[cb.nk] = Ks[j]; cb.c[cb.nk] = cs[j]; cb.nk++; }
        pdl_launch(k::rk_combine, grid_for_len(L), 256, 0, s, cb, out, L, dsp, dsc, nullptr);
    };
    // one explicit RK step Ycur -> Ynext of size *dsd, stages kept in U/K
    auto step = [&]() {
        const double *Ks[7];
        for (int j = 0; j < S; j++) Ks[j] = K + j * L;
        for (int i = 0; i < S; i++) {
            combine(U + i * L, Ycur, i, Ks, A[i], dsd, 0.0);
            // FP64 whatever the graph's arithmetic setting: the adjoint is FP64
            const double *xs[64];
            double *dxs[64];
            for (int o = 0; o < nops; o++) { xs[o] = U + i * L + o * n; dxs[o] = K + i * L + o * n; }
            launch_gen(g, U + i * L, xi, s, nullptr);
            launch_comm(g, xi, nops, xs, dxs, s, nullptr, 1, reinterpret_cast<double *>(operand_blocks(g, df)),
                        nullptr, piece_area(g, operand_blocks(g, df)));
        }
        combine(Ynext, Ycur, S, Ks, B, dsd, 0.0);
    };
    // the reverse of one step: k_bar_i = ds b_i y_bar, then stage by stage
    // u_bar_i = J(U_i)^T k_bar_i into y_bar and ds a_ij u_bar_i into k_bar_j
    auto back = [&]() {
        step();   // stage inputs U_i of this step
        for (int i = 0; i < S; i++) {
            cudaMemsetAsync(KB + i * L, 0, L * 8, s);
            const double *v[1] = {yb};
            const double c[1] = {B[i]};
            if (B[i] != 0.0) combine(KB + i * L, KB + i * L, 1, v, c, dsd, 0.0);
        }
        cudaMemcpyAsync(ybn, yb, L * 8, cudaMemcpyDeviceToDevice, s);
        for (int i = S - 1; i >= 0; i--) {
            stacked_vjp(g, U + i * L, KB + i * L, ub, nops, xi, xib, xb0, s, pk);
            const double *v[1] = {ub};
            const double one[1] = {1.0};
            combine(ybn, ybn, 1, v, one, nullptr, 1.0);
            for (int j = 0; j < i; j++) {
                const double c[1] = {A[i][j]};
                if (A[i][j] != 0.0) combine(KB + j * L, KB + j * L, 1, v, c, dsd, 0.0);
            }
        }
        cudaMemcpyAsync(yb, ybn, L * 8, cudaMemcpyDeviceToDevice, s);
    };
    // both bodies captured once as CUDA graphs; a step is then three
    // launches: its size and its start state copied in, the graph replayed
    cudaGraphExec_t gstep = nullptr, gback = nullptr;
    auto capture = [&](auto body, cudaGraphExec_t *exec) -> cudaError_t {
        cudaGraph_t graph;
        cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return ce;
        body();
        ce = cudaStreamEndCapture(s, &graph);
        if (ce != cudaSuccess) return ce;
        ce = cudaGraphInstantiate(exec, graph, 0);
        cudaGraphDestroy(graph);
        return ce;
    };
    e = capture(step, &gstep);
    if (e == cudaSuccess) e = capture(back, &gback);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (gstep) cudaGraphExecDestroy(gstep);
        cudaFreeAsync(buf, s);
        cudaStreamSynchronize(s);
        end_work(sp);
        return set_error(CUT_ERR_CUDA, std::string("cut_flow_vjp: graph capture: ") + cudaGetErrorString(e));
    }
    auto run_step = [&](int64_t t, const double *y, double *out) {
        cudaMemcpyAsync(dsd, steps_d + t, 8, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(Ycur, y, L * 8, cudaMemcpyDeviceToDevice, s);
        cudaGraphLaunch(gstep, s);
        cudaMemcpyAsync(out, Ynext, L * 8, cudaMemcpyDeviceToDevice, s);
    };
    // forward: the state at step c*C is kept as checkpoint c
    {
        double *cur = seg, *nxt = seg + L;
        cudaMemcpyAsync(cur, cp, L * 8, cudaMemcpyDeviceToDevice, s);
        for (int64_t t = 0; t < N; t++) {
            run_step(t, cur, nxt);
            std::swap(cur, nxt);
            if ((t + 1) % C == 0 && t + 1 < N) cudaMemcpyAsync(cp + ((t + 1) / C) * L, cur, L * 8, cudaMemcpyDeviceToDevice, s);
        }
    }
    // backward, segment by segment: recompute the segment's step-start
    // states from its checkpoint, then walk its steps in reverse
    cudaMemcpyAsync(yb, yb_h, n * 8, cudaMemcpyDeviceToDevice, s);
    if (n_obs) cudaMemcpyAsync(yb + n, yb_x, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s);
    for (int64_t c0 = N > 0 ? ((N - 1) / C) * C : -1; c0 >= 0; c0 -= C) {
        const int64_t c1 = std::min(N, c0 + C);
        cudaMemcpyAsync(seg, cp + (c0 / C) * L, L * 8, cudaMemcpyDeviceToDevice, s);
        for (int64_t t = c0; t < c1 - 1; t++) run_step(t, seg + (t - c0) * L, seg + (t - c0 + 1) * L);
        for (int64_t t = c1 - 1; t >= c0; t--) {
            cudaMemcpyAsync(dsd, steps_d + t, 8, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(Ycur, seg + (t - c0) * L, L * 8, cudaMemcpyDeviceToDevice, s);
            cudaGraphLaunch(gback, s);
        }
    }
    cudaGraphExecDestroy(gstep);
    cudaGraphExecDestroy(gback);
    cudaMemcpyAsync(gh, yb, n * 8, cudaMemcpyDeviceToDevice, s);
    if (n_obs) cudaMemcpyAsync(gx, yb + n, (size_t)n_obs * n * 8, cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(buf, s);
    e = cudaStreamSynchronize(s);
    end_work(sp);
    if (e != cudaSuccess) return set_error(CUT_ERR_CUDA, std::string("cut_flow_vjp: ") + cudaGetErrorString(e));
    return set_ok();
}

// ----------------------------------------------------------------- batched
namespace cut {
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
cut_status flow_batched_impl(const BatchedGraphView &v, int device, int batch, double *h, int n_obs, double *x,
                             int precision, const cut_flow_opts *o, int tile, int *steps_out, int *status_out,
                             cudaStream_t user, int *chosen_tile);
static thread_local int g_last_tile = 0;
}  // namespace cut

extern "C" cut_status cut_flow_batched(const cut_graph *g, int batch, double *h, int n_obs, double *x, int precision,
                                       const cut_flow_opts *o, int tile, int *steps_out, int *status_out,
                                       cut_stream_t stream) {
    TraceRange trace_("cut_flow_batched");
    if (whole_graph(g, "cut_flow_batched") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || batch < 1 || !h || n_obs < 0 || n_obs > 3 || (n_obs > 0 && !x) || !steps_out ||
        !status_out || (precision != CUT_FP64 && precision != CUT_FP32REC_FP64STATE) || tile < 0)
        return set_error(CUT_ERR_INVALID_ARG, "cut_flow_batched: bad argument (n_obs <= 3)");
    cut_status st = check_opts(o);
    if (st != CUT_OK) return st;
    if (o->replay_steps) return set_error(CUT_ERR_INVALID_ARG, "cut_flow_batched: replay is not supported");
    DeviceGuard dg(g->device);
    BatchedGraphView v{g->st[0].rp, g->st[1].rp, g->st[0].rec, g->st[1].rec, g->wtab,
                       (int)g->host.num.size(), g->host.n(), g->host.n_g(), g->host.sha,
                       g->st[0].R, g->st[1].R, g->wuniform, g->wmag, g->wnegmask};
    return flow_batched_impl(v, g->device, batch, h, n_obs, x, precision, o, tile, steps_out, status_out,
                             (cudaStream_t)stream, &g_last_tile);
}

extern "C" int cut_flow_batched_last_tile(void) { return g_last_tile; }

// ----------------------------------------------------------------- no-alloc RHS
// A right-hand side for callers that must not allocate device memory: the
// generator scratch lives in a fixed array inside the library's device image.
namespace cut {

constexpr int64_t kNoAllocMaxGen = CUT_RHS_NOALLOC_MAX_NG;
static __device__ __align__(256) double g_noalloc_xi[kNoAllocMaxGen];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[256] = {nullptr};
static void *g_noalloc_ctx[256] = {nullptr};   // context the address belongs to

// The calling thread's current CUDA context (driver entry point reached
// through the runtime, so the library does not link libcuda directly).
static void *current_context() {
    typedef int (*CtxGetCurrent)(void **);
    static CtxGetCurrent fn = []() -> CtxGetCurrent {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (CtxGetCurrent)f;
    }();
    void *ctx = nullptr;
    if (fn) fn(&ctx);
    return ctx;
}

// Device address of the scratch array in the current device's context,
// looked up once per device and context (the host-side name of the array is
// not a device address; a device reset or another context makes a new
// lookup).
static cut_status noalloc_scratch(int device, double **out) {
    if (device < 0 || device >= 256) return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    void *ctx = current_context();
    if (!g_noalloc_ptr[device] || !ctx || ctx != g_noalloc_ctx[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_xi);   // creates the context if needed
        if (e != cudaSuccess || !p)
            return set_error(CUT_ERR_CUDA, std::string("cut_rhs_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[device] = (double *)p;
        g_noalloc_ctx[device] = current_context();
    }
    *out = g_noalloc_ptr[device];
    return CUT_OK;
}

}  // namespace cut

extern "C" cut_status cut_rhs_noalloc(const cut_graph *g, const double *h, int n_obs, const double *x, double *dh,
                                      double *dx, cut_stream_t stream) {
    if (whole_graph(g, "cut_rhs_noalloc") != CUT_OK) return CUT_ERR_INVALID_ARG;
    if (!g || g->device < 0 || !h || !dh || n_obs < 0 || n_obs > 63 || (n_obs > 0 && (!x || !dx)))
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_noalloc: bad argument");
    if (g->host.n_g() > kNoAllocMaxGen)
        return set_error(CUT_ERR_INVALID_ARG, "cut_rhs_noalloc: the graph has " + std::to_string(g->host.n_g()) +
                                                  " generator coordinates, more than the fixed scratch holds (" +
                                                  std::to_string(kNoAllocMaxGen) + "); use cut_rhs");
    DeviceGuard dg(g->device);
    double *xi = nullptr;
    cut_status st = noalloc_scratch(g->device, &xi);
    if (st != CUT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n();
    // every generator coordinate is written by the generator stage before the
    // commutator stage reads it, so the scratch needs no clearing
    launch_gen(g, h, xi, s, nullptr);
    const double *xs[64];
    double *dxs[64];
    xs[0] = h;
    dxs[0] = dh;
    for (int o = 0; o < n_obs; o++) { xs[o + 1] = x + o * n; dxs[o + 1] = dx + o * n; }
    launch_comm(g, xi, n_obs + 1, xs, dxs, s, nullptr);
    CUDA_TRY(cudaGetLastError());
    return set_ok();
}

// ----------------------------------------------------------------- target-range shards
// Sec. 2.2: records are grouped by output, so the outputs of each stage can
// be split into contiguous ranges that hold about equal numbers of records;
// a rank holding one range of each stage computes its generator
// coordinates and its outputs from full input vectors, and the ranks
// exchange those pieces (an all-gather of xi, then of the right-hand side).
namespace cut {

// bounds[0..parts]: row r of the stage goes to part p when
// bounds[p] <= r < bounds[p+1]; part p starts at the first row whose record
// offset reaches p R / parts (deterministic, independent of the caller).
static void partition_rows(const std::vector<uint64_t> &rp, int parts, int64_t *bounds) {
    const int64_t rows = (int64_t)rp.size() - 1;
    const uint64_t R = rows > 0 ? rp[rows] : 0;
    bounds[0] = 0;
    for (int p = 1; p < parts; p++) {
        const uint64_t target = (uint64_t)(((unsigned __int128)R * (unsigned)p) / (unsigned)parts);
        int64_t b = (int64_t)(std::lower_bound(rp.begin(), rp.end(), target) - rp.begin());
        b = std::min(b, rows);
        bounds[p] = std::max(b, bounds[p - 1]);
    }
    bounds[parts] = std::max<int64_t>(rows, 0);
}

// the rows [lo, hi) of a stage, row pointers rebased to start at 0
static cut_status upload_rows(DevCSR &d, const std::vector<uint64_t> &rp, const std::vector<uint32_t> &rec,
                              int64_t lo, int64_t hi, int64_t &bytes) {
    std::vector<uint64_t> lrp(hi - lo + 1);
    for (int64_t r = lo; r <= hi; r++) lrp[r - lo] = rp[r] - rp[lo];
    std::vector<uint32_t> lrec(rec.begin() + 2 * rp[lo], rec.begin() + 2 * rp[hi]);
    cut_status st = upload_csr(d, lrp, lrec, bytes);
    d.lane_rows = (int64_t)rp.size() - 1;
    return st;
}

}  // namespace cut

extern "C" cut_status cut_graph_partition(const cut_graph *g, int stage, int parts, int64_t *bounds) {
    if (!g || stage < 0 || stage > 1 || parts < 1 || parts > 65536 || !bounds)
        return set_error(CUT_ERR_INVALID_ARG, "cut_graph_partition: bad argument");
    if (g->shard_world > 0 || g->host.rp[stage].empty())
        return set_error(CUT_ERR_INVALID_ARG, "cut_graph_partition: needs a handle of the whole graph");
    partition_rows(g->host.rp[stage], parts, bounds);
    return set_ok();
}

extern "C" cut_status cut_graph_load_shard(const char *path, int device, int rank, int world, unsigned flags,
                                           cut_graph **out) {
    TraceRange trace_("cut_graph_load_shard");
    if (!path || !out || device < 0 || world < 1 || world > 65536 || rank < 0 || rank >= world || flags != 0)
        return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load_shard: bad argument");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device >= ndev) return set_error(CUT_ERR_INVALID_ARG, "cut_graph_load_shard: bad device");
    std::unique_ptr<cut_graph> g(new cut_graph());
    g->device = device;
    std::string err;
    int rc = read_bundle(path, g->host, &err);
    if (rc != 0) return set_error((cut_status)rc, "cut_graph_load_shard: " + err);
    DeviceGuard dg(device);
    int64_t bytes = 0;
    std::vector<int64_t> b(world + 1);
    for (int s = 0; s < 2; s++) {
        partition_rows(g->host.rp[s], world, b.data());
        g->lo[s] = b[rank];
        g->hi[s] = b[rank + 1];
        cut_status st = upload_rows(g->st[s], g->host.rp[s], g->host.rec[s], g->lo[s], g->hi[s], bytes);
        if (st != CUT_OK) return st;
        if (s == 1) st = add_pieces(g->st[1], g->host.rp[1], g->lo[1], g->hi[1], bytes);
        if (st != CUT_OK) return st;
    }
    cut_status st = upload_weights(g.get());
    if (st != CUT_OK) return st;
    g->device_bytes += bytes;
    g->shard_rank = rank;
    g->shard_world = world;
    *out = g.release();
    return set_ok();
}

extern "C" cut_status cut_shard_generator(const cut_graph *g, const double *h, double *xi_part, cut_stream_t stream) {
    TraceRange trace_("cut_shard_generator");
    if (!g || g->device < 0 || g->shard_world < 1 || !h || (!xi_part && g->hi[0] > g->lo[0]))
        return set_error(CUT_ERR_INVALID_ARG, "cut_shard_generator: bad argument (needs a shard handle)");
    if (g->hi[0] == g->lo[0]) return set_ok();
    DeviceGuard dg(g->device);
    launch_gen(g, h, xi_part, (cudaStream_t)stream, nullptr);
    CUDA_TRY(cudaGetLastError());
    return set_ok();
}

extern "C" cut_status cut_shard_commutator(const cut_graph *g, const double *xi, int n_ops, const double *x,
                                           double *dx_part, cut_stream_t stream) {
    TraceRange trace_("cut_shard_commutator");
    if (!g || g->device < 0 || g->shard_world < 1 || !xi || n_ops < 1 || n_ops > 64 || !x ||
        (!dx_part && g->hi[1] > g->lo[1]))
        return set_error(CUT_ERR_INVALID_ARG, "cut_shard_commutator: bad argument (needs a shard handle)");
    const int64_t rows = g->hi[1] - g->lo[1];
    if (rows == 0) return set_ok();
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->host.n();
    void *df = nullptr;
    CUDA_TRY(scratch_alloc(&df, operand_scratch_bytes(g), s));
    const double *xs[64];
    double *dxs[64];
    for (int o = 0; o < n_ops; o++) { xs[o] = x + o * n; dxs[o] = dx_part + o * rows; }
    apply_L(g, xi, (float2 *)df, operand_blocks(g, df), n_ops, xs, dxs, s, nullptr);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaFreeAsync(df, s));
    return set_ok();
}

extern "C" cut_status cut_combine(int64_t len, const double *base, int nk, const double *const *K, const double *c,
                                  double ds, double *out, cut_stream_t stream) {
    if (len < 0 || !base || !out || nk < 0 || nk > 7 || (nk > 0 && (!K || !c)))
        return set_error(CUT_ERR_INVALID_ARG, "cut_combine: bad argument (nk <= 7)");
    if (len == 0) return set_ok();
    k::Combine cb;
    cb.base = base;
    cb.nk = 0;
    for (int s = 0; s < nk; s++) {
        if (!K[s]) return set_error(CUT_ERR_INVALID_ARG, "cut_combine: null slope");
        if (c[s] != 0.0) { cb.K[cb.nk] = K[s]; cb.c[cb.nk] = c[s]; cb.nk++; }
    }
    pdl_launch(k::rk_combine, grid_for_len(len), 256, 0, (cudaStream_t)stream, cb, out, len, nullptr, ds, nullptr);
    CUDA_TRY(cudaGetLastError());
    return set_ok();
}
