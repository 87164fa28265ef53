/*
 * cut.h -- C ABI of the compile-once CUT operation-graph engine (B300, sm_103a).
 *
 * The library evaluates the projected continuous-unitary-transformation flow
 *     dH/ds = P[eta(H), H],   dX/ds = P[eta(H), X],   eta = [H_d, H_od]
 * (paper Sec. 2.1, Eqs. coflow, block-generator, projected-flow) by applying
 * a stored operation graph (Sec. 2.2, Eq. graph-actions):
 *     xi_a(h)  = sum_{e in E_eta(a)} alpha_e (Dh)_{i_e} ((I-D)h)_{j_e}
 *     F_k(h,x) = sum_{e in E_L(k)}   beta_e  xi_{a_e}(h) x_{j_e}
 * Records are grouped by output (Sec. 2.2, last paragraph), stored once on
 * disk (Sec. 2.3) and traversed forward and in reverse (Sec. 2.4).
 *
 * Conventions shared by every entry point
 *   - Coefficients are real doubles.  For Pauli strings H = sum_k h_k P_k with
 *     Hermitian P_k and eta = i sum_a xi_a G_a; for fermion monomials
 *     H = sum_k h_k O_k and eta = sum_a xi_a G_a; for Pauli-boson monomials
 *     (Sec. 2.1, Eq. monomial) the Pauli factor is taken from the real basis
 *     {I, X, iY, Z}, so H = sum_k h_k B_k and eta = sum_a xi_a G_a with real
 *     coefficients as well.  All stored factors are exact integers (or
 *     rationals num/den), never rounded.
 *   - A coefficient vector has n entries in the order of the registry the
 *     graph was built from (cut_graph_labels); xi has n_g entries in the
 *     order of the generator registry.
 *   - "device" pointers are CUDA device memory on the graph's device,
 *     owned by the caller; the library keeps no pointer after a call
 *     returns, but kernels it queued on `stream` may still read or write
 *     them until the stream reaches that point.  "host" pointers are
 *     ordinary CPU memory, read or written before the call returns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - The library's kernels are launched with programmatic stream serialization
 *     and let the next grid on the stream be scheduled as soon as they
 *     start.  Work the caller queues with ordinary launches, copies or
 *     events still waits for them to complete.  A kernel the caller
 *     launches right after a call with that attribute set must wait on the
 *     device (cudaGridDependencySynchronize) before it reads the call's
 *     outputs.
 *   - "Scratch from the stream-ordered allocator" below means the library's
 *     own memory pool of the graph's device (cudaMallocFromPoolAsync; freed
 *     with cudaFreeAsync on the call's stream).  The pool keeps up to 1 GiB
 *     of freed scratch reserved between calls, so that repeated calls map
 *     no new device memory; the reserve is released when the process ends
 *     (or the device's context is destroyed).  Allocations beyond what the
 *     device can give fail with CUT_ERR_OUT_OF_MEMORY.
 *   - Phases (compile, reload, each traversal or flow) are marked as NVTX
 *     ranges named after the entry point ("cut_flow", "cut_graph_load/upload",
 *     ...).  With the environment variable CUT_LOG=1 each also writes one
 *     line "[cut] <name> <ms> ms" to stderr when it ends.
 *   - No entry point throws; each returns a cut_status and, on failure,
 *     leaves a message for cut_last_error() (thread-local).  Arguments are
 *     validated before anything is queued: on CUT_ERR_INVALID_ARG nothing
 *     was written.
 */
#ifndef CUT_H
#define CUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cut_graph cut_graph; /* opaque; owned by the library until cut_graph_free */
typedef void *cut_stream_t;         /* cudaStream_t */

typedef enum {
    CUT_OK = 0,
    CUT_ERR_INVALID_ARG = 1,
    CUT_ERR_IO = 2,
    CUT_ERR_FORMAT = 3,
    CUT_ERR_CHECKSUM = 4,
    CUT_ERR_OUT_OF_MEMORY = 5,
    CUT_ERR_CUDA = 6,
    CUT_ERR_NONFINITE = 7,
    CUT_ERR_STEP_UNDERFLOW = 8,
    CUT_ERR_MAX_STEPS = 9,
    CUT_ERR_TIMEOUT = 10,
    CUT_ERR_UNSUPPORTED = 11
} cut_status;

enum { CUT_ALG_PAULI = 0, CUT_ALG_FERMION = 1, CUT_ALG_PAULI_BOSON = 2 };
enum { CUT_RK4 = 0, CUT_DP45 = 1 };
enum { CUT_FP64 = 0, CUT_FP32REC_FP64STATE = 1 };
enum { CUT_ARITH_FP64 = 0, CUT_ARITH_DF64 = 1 };

/* Message of the last failing call on this thread ("" if none). */
const char *cut_last_error(void);
const char *cut_version(void);

/* ------------------------------------------------------------------ */
/* Compile (Sec. 2.2-2.3): registry -> two-traversal build -> bundle    */
/* ------------------------------------------------------------------ */
typedef struct {
    int algebra;   /* CUT_ALG_PAULI, CUT_ALG_FERMION or CUT_ALG_PAULI_BOSON */
    int nmodes;    /* qubits / spin-orbitals 1..32, boson modes 1..6 */
    int max_rank;  /* fermion: highest rank of generator coordinates kept
                      (terms of eta of higher rank cannot reach a registry of
                      that rank); 0 = the registry's highest rank */
    int threads;   /* host threads, 0 = all cores */
    int diagnostics; /* 1: also store the outside-space records gamma of
                        Eq. graph-actions (terms of [eta, X] outside the
                        registry, Eq. projected-flow), with eta exact */
} cut_build_opts;

typedef struct {
    int64_t n, n_g, R_g, R_L; /* registry size, generator size, records */
    int n_codes;              /* distinct exact factors */
    double seconds_count, seconds_write, seconds_total;
    int64_t bytes_stored;     /* bundle size on disk */
    int64_t peak_rss_bytes;   /* process peak resident set after the build */
} cut_build_stats;

/* Build the operation graph of the registry `labels` (host, n entries,
 * distinct, every label number-conserving for fermions) and write the bundle
 * to `path`.  Two deterministic traversals: the first counts records per
 * output, the second writes each record into its final slot (Sec. 2.3).
 * Records of one output are sorted by (input a, input b); the same input
 * gives a bitwise-identical file.  `stats` (host) may be NULL.
 * Errors: INVALID_ARG (bad options, duplicate or malformed label, an index
 * beyond 2^24), IO (cannot write), OUT_OF_MEMORY. */
cut_status cut_build(const cut_build_opts *opts, int64_t n, const uint64_t *labels,
                     const char *path, cut_build_stats *stats);

/* ------------------------------------------------------------------ */
/* Load / query (Sec. 2.3: validated reload in any process)            */
/* ------------------------------------------------------------------ */
/* Read `path`, verify its SHA-256 and structure, upload to CUDA device
 * `device`.  device == -1 gives a host-only handle (no CUDA call is made):
 * query, labels, weights and records work, every traversal returns
 * INVALID_ARG.  flags: 0, or CUT_LOAD_ADJOINT to build the transposed record
 * orders of the reverse traversal (Sec. 2.4) now, on the host threads, and
 * upload them (about twice the graph's device memory more); without it they
 * are built at the first adjoint call.  Errors: IO, FORMAT (bad header or
 * inconsistent arrays), CHECKSUM (payload digest mismatch), CUDA,
 * OUT_OF_MEMORY, INVALID_ARG (unknown flag). */
enum { CUT_LOAD_ADJOINT = 1 };
cut_status cut_graph_load(const char *path, int device, unsigned flags, cut_graph **out);
cut_status cut_graph_free(cut_graph *g);

typedef struct {
    int algebra, nmodes, max_rank, n_codes;
    int64_t n, n_g, R_g, R_L;
    uint8_t sha256[32];      /* digest of the bundle payload */
    int64_t device_bytes;    /* graph bytes resident on the device */
    int64_t record_bytes;    /* bytes of one stored record (both stages) */
    int64_t n_out, R_C;      /* outside-space labels and records (0 without diagnostics) */
    int shard_rank, shard_world; /* shard handles (cut_graph_load_shard): its
                                    rank and the number of shards; 0, 0 for a
                                    whole graph.  R_g and R_L then count the
                                    shard's own records. */
    int64_t gen_lo, gen_hi;      /* generator rows held: [gen_lo, gen_hi) */
    int64_t comm_lo, comm_hi;    /* commutator rows held: [comm_lo, comm_hi) */
} cut_graph_desc;

cut_status cut_graph_query(const cut_graph *g, cut_graph_desc *out);
/* host out: labels[n], gen_labels[n_g], diag[n] (1 = block-diagonal
 * coordinate, the mask D of Sec. 2.2); any pointer may be NULL. */
cut_status cut_graph_labels(const cut_graph *g, uint64_t *labels, uint64_t *gen_labels, uint8_t *diag);
/* host out: the outside-space labels out[n_out] (diagnostic graphs). */
cut_status cut_graph_outside_labels(const cut_graph *g, uint64_t *out);
/* host out: exact factor table, value of code c = num[c] / den[c]. */
cut_status cut_graph_weights(const cut_graph *g, int32_t *num, int32_t *den);
/* host out: the stored records of one stage (0 = generator, rows are
 * generator coordinates a, inputs (i, j); 1 = commutator, rows are outputs
 * k, inputs (a, j); 2 = outside space, rows are outside labels q, inputs
 * (a, j)).  row_ptr[rows+1], in1[R], in2[R], code[R]. */
cut_status cut_graph_records(const cut_graph *g, int stage, int64_t *row_ptr, int32_t *in1,
                             int32_t *in2, uint8_t *code);

/* ------------------------------------------------------------------ */
/* One right-hand side (Eq. graph-actions)                              */
/* ------------------------------------------------------------------ */
/* dh = P[eta(h), H], dx_o = P[eta(h), X_o] for o < n_obs.
 * device in : h[n], x[n_obs][n] (NULL if n_obs == 0)
 * device out: dh[n], dx[n_obs][n], xi_out[n_g] (optional, NULL = not kept)
 * Runs asynchronously on `stream`; takes its scratch (the packed operand
 * blocks, n x 64 bytes, and the generator when xi_out is NULL) from the
 * stream-ordered allocator and returns it on the same stream.  On a graph
 * with few long rows (fewer than 16384 rows of 512 or more records on
 * average) the commutator stage cuts each row into pieces of about 256
 * records, sums the pieces and then each row's pieces in order (64 more
 * bytes of scratch per piece); a row's cut depends only on its length, so
 * the result is the same on every run and on every shard.
 * Errors: INVALID_ARG, CUDA. */
cut_status cut_rhs(const cut_graph *g, const double *h, int n_obs, const double *x, double *dh,
                   double *dx, double *xi_out, cut_stream_t stream);

/* Arithmetic of the commutator stage for cut_rhs, cut_apply_L and cut_flow
 * on this graph (a host-side setting of the handle; not thread-safe against
 * calls in flight on other threads).
 *   CUT_ARITH_FP64 (default): FP64 products and sums.
 *   CUT_ARITH_DF64: products and sums as unevaluated pairs of FP32 numbers
 *     (about 48 significant bits, error-free two-product and two-sum), run on
 *     the FP32 pipes, which on B300 far outnumber the FP64 pipe that bounds
 *     the FP64 stage.  Results agree with FP64 to about 1e-14 relative to the
 *     largest term of a sum; coefficients below ~1e-38 lose relative
 *     precision (FP32 range).  The generator stage, the RK state, the
 *     adjoint and the batched path stay FP64 as documented there.
 * Errors: INVALID_ARG (unknown mode), UNSUPPORTED (DF64 needs all stored
 * factors of one magnitude, true for Pauli and fermion graphs). */
cut_status cut_graph_set_arithmetic(cut_graph *g, int arith);

/* The linear action L(h) x (Sec. 2.4, Eq. forward-coeff) for given generator
 * coordinates: dx_o = sum_e beta_e xi[a_e] x_o[j_e] for n_ops operands, i.e.
 * the commutator stage alone (xi from cut_rhs's xi_out).
 * device in: xi[n_g], x[n_ops][n]; device out: dx[n_ops][n].
 * Errors: INVALID_ARG, CUDA. */
cut_status cut_apply_L(const cut_graph *g, const double *xi, int n_ops, const double *x, double *dx,
                       cut_stream_t stream);

/* Outside-space diagnostic action (Eq. graph-actions, third line; Eq.
 * projected-flow): C_q = sum_e gamma_e xi_{a_e} x_{j_e} for the operands
 * X_0 = H and X_1.. of cut_rhs, for every label q outside the registry that
 * [eta, X] generates.  Needs a graph built with diagnostics; it neither
 * reads nor changes anything the retained flow uses.
 * device in : h[n], x[n_obs][n]; device out: c[(1 + n_obs)][n_out]
 * Errors: INVALID_ARG (no diagnostic records), CUDA. */
cut_status cut_rhs_outside(const cut_graph *g, const double *h, int n_obs, const double *x, double *c,
                           cut_stream_t stream);

/* Multi-operator assembly (Sec. 2.4, last paragraph): from a library of
 * already transformed source operators X_i (coefficient vectors), form
 * out_m = sum_i C[m][i] X_i for n_out combinations, without touching the
 * graph.  The sum runs over i in index order with FMA, so results are the
 * same bits on every run.  Uses the current CUDA device.
 * device in : X[n_src][n], C[n_out][n_src]; device out: out[n_out][n]
 * Errors: INVALID_ARG (1 <= n_src <= 3000), CUDA. */
cut_status cut_assemble(int n_src, int64_t n, const double *X, int n_out, const double *C, double *out,
                        cut_stream_t stream);

/* Forward tangent (Sec. 2.4, Eq. directional-derivative): the directional
 * derivative of cut_rhs along (dh, dx),
 *   d F_o = dF_o/dh . dh + L(h) dx_o      (X_0 = H, so dx_0 = dh),
 * including the induced variation of the generator.
 * device in : h[n], x[n_obs][n], dh[n], dx[n_obs][n]
 * device out: out_h[n], out_x[n_obs][n]
 * Errors: INVALID_ARG, CUDA. */
cut_status cut_rhs_jvp(const cut_graph *g, const double *h, int n_obs, const double *x, const double *dh,
                       const double *dx, double *out_h, double *out_x, cut_stream_t stream);

/* Allocation-free variant of cut_rhs.  The paper has no counterpart; it
 * exists for callers that may not allocate device memory while they run
 * (for example a real-time or serving loop whose memory is fixed up front,
 * or code whose allocator is owned by someone else), since cut_rhs takes
 * temporary buffers from the stream-ordered allocator (the generator when
 * xi_out is NULL, and up to 64 bytes per coordinate into which the
 * operands are packed).  Here the generator buffer is a fixed array of
 * CUT_RHS_NOALLOC_MAX_NG
 * doubles (8 MiB) compiled into the library: every GPU that loads the
 * library holds it until the process exits.
 *   - Same inputs, outputs and results as cut_rhs with xi_out = NULL, always
 *     in FP64 arithmetic; the operands are gathered one by one instead of
 *     from packed blocks, with the same sums in the same order (same bits;
 *     on graphs with few long rows, which cut_rhs cuts into pieces, the
 *     rows are summed whole here, so the two agree to rounding).
 *   - Graphs with more than CUT_RHS_NOALLOC_MAX_NG generator coordinates are
 *     rejected with CUT_ERR_INVALID_ARG before anything is queued.
 *   - Makes no cudaMalloc, cudaFree or other allocating call.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept per device and CUDA
 *     context: after a device reset, or with another context current, the
 *     next call looks it up again (again outside any capture).
 *   - All calls on a device share the one array and it keeps what the last
 *     call left there (every entry is rewritten before it is read, so nothing
 *     needs clearing): calls whose kernels overlap on the GPU (different
 *     streams, no ordering between them) race on it and give wrong results. */
#define CUT_RHS_NOALLOC_MAX_NG (1 << 20)
cut_status cut_rhs_noalloc(const cut_graph *g, const double *h, int n_obs, const double *x, double *dh,
                           double *dx, cut_stream_t stream);

/* Reverse traversal (Sec. 2.4): vector-Jacobian product of cut_rhs.
 * With L = <w_h, dh> + sum_o <w_x[o], dx_o>:
 *   h_bar = dL/dh (through eta and through X_0 = H),  x_bar[o] = dL/dx_o.
 * device in : h[n], x[n_obs][n], w_h[n], w_x[n_obs][n]
 * device out: h_bar[n], x_bar[n_obs][n]
 * The transposed record orders come from cut_graph_load(.., CUT_LOAD_ADJOINT)
 * or are built on the host at the first call (synchronous), then kept with
 * the graph.  With at most eight operands the transposed passes gather the
 * operands as packed 32-byte blocks (scratch n x 128 bytes from the
 * stream-ordered allocator).  Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY. */
cut_status cut_rhs_adjoint(const cut_graph *g, const double *h, int n_obs, const double *x,
                           const double *w_h, const double *w_x, double *h_bar, double *x_bar,
                           cut_stream_t stream);

/* ------------------------------------------------------------------ */
/* Target-range shards (Sec. 2.2: records grouped by output)            */
/* ------------------------------------------------------------------ */
/* Because every output's records are stored together, the outputs of each
 * stage split into contiguous row ranges that hold about equal numbers of
 * records.  A shard holds one range of the generator stage and one of the
 * commutator stage; per right-hand side the shards of a group compute their
 * pieces from full input vectors and exchange them (all-gather of xi, then
 * of the outputs).  Each row is summed exactly as the whole graph sums it,
 * so the assembled pieces equal cut_rhs bit for bit.
 *
 * Record-balanced bounds of stage 0 (generator rows) or 1 (commutator rows)
 * split into `parts`: host out bounds[parts + 1]; part p holds rows
 * [bounds[p], bounds[p+1]) and starts at the first row whose record offset
 * reaches p * R / parts.  Needs a whole-graph handle (host-only works).
 * Errors: INVALID_ARG. */
cut_status cut_graph_partition(const cut_graph *g, int stage, int parts, int64_t *bounds);

/* Load shard `rank` of `world` onto `device`: the records of generator rows
 * [gen_lo, gen_hi) and commutator rows [comm_lo, comm_hi) of
 * cut_graph_partition(.., world, ..) are resident (about 1/world of the
 * graph); labels and factors are kept whole on the host.  The handle serves
 * cut_shard_generator, cut_shard_commutator, the query and host-side calls;
 * whole-graph traversals (cut_rhs, cut_flow, ...) return INVALID_ARG on it.
 * Errors: as cut_graph_load, INVALID_ARG (rank, world, device). */
cut_status cut_graph_load_shard(const char *path, int device, int rank, int world, unsigned flags,
                                cut_graph **out);

/* Generator stage of the shard's rows (Eq. graph-actions, line 1):
 * device in h[n] (whole vector); device out xi_part[gen_hi - gen_lo], entry
 * r - gen_lo = xi_r.  Errors: INVALID_ARG, CUDA. */
cut_status cut_shard_generator(const cut_graph *g, const double *h, double *xi_part, cut_stream_t stream);

/* Commutator stage of the shard's rows (Eq. graph-actions, line 2) for n_ops
 * operands: device in xi[n_g] (all generator coordinates), x[n_ops][n];
 * device out dx_part[n_ops][comm_hi - comm_lo].  Takes the operand-packing
 * scratch (n x 64 bytes) from the stream-ordered allocator like cut_rhs.
 * Errors: INVALID_ARG, CUDA. */
cut_status cut_shard_commutator(const cut_graph *g, const double *xi, int n_ops, const double *x, double *dx_part,
                                cut_stream_t stream);

/* Runge-Kutta combination out[i] = base[i] + sum_s (c[s] ds) K[s][i] for
 * len entries (terms with c[s] == 0 skipped), the same kernel and rounding
 * as the stage inputs and updates of cut_flow, so a flow driven step by step
 * through the shard calls reproduces cut_flow's RK4 bit for bit.  host in:
 * K[nk] (device pointers), c[nk]; nk <= 7; device in/out: base, out (may be
 * the same).  Uses the current device.  Errors: INVALID_ARG, CUDA. */
cut_status cut_combine(int64_t len, const double *base, int nk, const double *const *K, const double *c, double ds,
                       double *out, cut_stream_t stream);

/* ------------------------------------------------------------------ */
/* Flows                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    int method;              /* CUT_RK4 (fixed ds) or CUT_DP45 (adaptive) */
    double s0, s1;           /* flow interval */
    double ds;               /* RK4 step; DP45 first trial step */
    double rtol, atol;       /* DP45 tolerances */
    int64_t max_steps;       /* DP45: limit on attempted steps (0 = 10^6) */
    const double *replay_steps; /* host, DP45 only: if non-NULL, take exactly
                                   these n_replay steps, all accepted */
    int64_t n_replay;
    double *record_steps;    /* host, optional: accepted step sizes out */
    int64_t record_cap;      /* capacity of record_steps (cut_flow), or per
                                instance of batch_record_steps (cut_flow_batched) */
    double *batch_record_steps; /* device, cut_flow_batched only, optional:
                                   [batch][record_cap], row b receives the
                                   accepted step sizes of instance b in order
                                   (entries past its step count are untouched) */
    int64_t pause_after;     /* cut_flow, DP45 only: > 0 stops the flow after
                                that many attempts with status OK (a
                                checkpoint, see cut_flow) */
} cut_flow_opts;

typedef struct {
    int64_t steps, rejects, rhs_calls;
    double s_final;
    double ds_next;          /* DP45: the step size the next attempt would take */
    int finished;            /* 1: reached s1; 0: paused (pause_after) */
} cut_flow_stats;

/* Integrate the stacked state [h; x_1..x_nobs] from s0 to s1.
 * device in/out: h[n], x[n_obs][n].  host out: stats (may be NULL).
 * RK4: nsteps = round((s1-s0)/ds) steps of exactly ds (the last one lands
 * on s1).  DP45: Dormand-Prince 5(4), error ratio
 * max_k |e_k| / (atol + rtol max(|y_k|, |y5_k|)), accept when <= 1,
 * ds *= clamp(0.9 r^-1/5, 0.2, 5) (growth capped at 1 after a rejection).
 * Synchronises `stream` before returning.
 * Checkpoint and resume (DP45): with opts->pause_after = m the flow stops
 * after m attempts and returns OK with the state in h, x and stats->s_final,
 * stats->ds_next, finished = 0.  The controller's next decision depends only
 * on (state, s, ds), and every kernel is deterministic, so calling cut_flow
 * again with s0 = s_final and ds = ds_next (same s1, rtol, atol) continues
 * exactly where the uninterrupted flow would be: the same accepted steps and
 * the same bits at s1.
 * Errors: INVALID_ARG, CUDA, NONFINITE (a non-finite state was produced),
 * STEP_UNDERFLOW (ds fell below 1e-14 |s|), MAX_STEPS. */
cut_status cut_flow(const cut_graph *g, double *h, int n_obs, double *x, const cut_flow_opts *opts,
                    cut_flow_stats *stats, cut_stream_t stream);

/* Gradient through a flow: the discrete adjoint of the RK steps that
 * cut_flow took (pass its accepted steps in opts->replay_steps for DP45;
 * RK4 recomputes its uniform steps).  Given y_bar = dJ/dy(s1) for the
 * stacked final state, returns dJ/dy(s0).  The forward states are stored
 * every `checkpoint_every` steps and recomputed segment by segment.
 * device in : h0[n], x0[n_obs][n] (initial state, unchanged),
 *             yb_h[n], yb_x[n_obs][n]
 * device out: gh[n], gx[n_obs][n]
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY. */
cut_status cut_flow_vjp(const cut_graph *g, const double *h0, int n_obs, const double *x0,
                        const cut_flow_opts *opts, int checkpoint_every, const double *yb_h,
                        const double *yb_x, double *gh, double *gx, cut_stream_t stream);

/* Many coefficient sets through one graph read per record (batched flows).
 * device in/out: h[batch][n], x[batch][n_obs][n] (instance-major, as a user
 * holds them; the library transposes internally).
 * precision: CUT_FP64 or CUT_FP32REC_FP64STATE (records, products and sums
 * in FP32, including the stage sums sum_j a_ij K_j of the FP32 slopes and
 * the error estimate; the RK state and its updates Y + ds * (stage sum), the
 * flow coordinate and the step size stay FP64).
 * Each instance has its own adaptive step sequence (DP45) and stops at s1.
 * device out: steps_out[batch] accepted steps, status_out[batch] cut_status,
 * and, when opts->batch_record_steps is set, each instance's accepted step
 * sizes (so that a reference can replay that instance's path).
 * host in: opts (replay_steps and the host record_steps are ignored).  `tile` chooses the instance
 * tile width (0 = autotuned: a short probe of every width that fits, the
 * choice remembered per graph, batch, operands, precision, method and GPU;
 * with the environment variable CUT_TUNE_CACHE naming a file, choices are
 * read from it and new ones appended, one line each: "<graph SHA-256 hex>
 * <batch> <operands> <fp32 0|1> <method> <tile> <GPU name>").
 * Synchronises `stream` before returning.
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY. */
cut_status cut_flow_batched(const cut_graph *g, int batch, double *h, int n_obs, double *x,
                            int precision, const cut_flow_opts *opts, int tile, int *steps_out,
                            int *status_out, cut_stream_t stream);
/* Tile width the calling thread's last cut_flow_batched call ran with (0 if
 * none). */
int cut_flow_batched_last_tile(void);

/* ------------------------------------------------------------------ */
/* Measured roofs                                                       */
/* ------------------------------------------------------------------ */
/* Fused multiply-add throughput of CUDA device `device` in TFLOP/s (2 flops
 * per FMA), FP64 (fp64 != 0) or FP32: independent FMA chains in every thread
 * of 8 CTAs x 256 threads per SM; the loop length grows until one launch
 * takes about seconds / 4, then the best of three timed launches (CUDA
 * events) is reported.  The FP64 graph traversal on B300 is bound by this
 * rate, not by HBM.  host out: tflops.  Errors: INVALID_ARG, CUDA. */
cut_status cut_measure_fma_rate(int device, int fp64, double seconds, double *tflops);

/* ------------------------------------------------------------------ */
/* Learned surrogate of the flow map (the paper has no counterpart: a   */
/* warm start and screen in front of the graph flow, which stays the    */
/* fallback and the judge of its error)                                 */
/* ------------------------------------------------------------------ */
/* MLP n_in -> n_hidden -> n_hidden -> n_out, GELU after the two hidden
 * layers, BF16 operands with FP32 accumulation on the tensor cores
 * (tcgen05), FP32 master weights, AdamW.  Targets are standardised per
 * output, t_hat = (t - shift) / scale; the forward pass returns
 * y = scale * y_hat + shift.  Weights start uniform in +-1/sqrt(fan_in)
 * from `seed`, biases 0, scale 1, shift 0. */
typedef struct cut_mlp cut_mlp;
cut_status cut_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, int device, cut_mlp **out);
cut_status cut_mlp_free(cut_mlp *m);
/* host in: scale[n_out] (> 0), shift[n_out] */
cut_status cut_mlp_set_output_affine(cut_mlp *m, const float *scale, const float *shift);
/* host out: scale[n_out], shift[n_out] (either may be NULL, not both), the
 * output affine in use (after cut_mlp_fit_linear: the residual RMS of each
 * output over sqrt(weight), and the intercept).  Waits for the device's
 * queued work first.  Errors: INVALID_ARG, CUDA. */
cut_status cut_mlp_get_output_affine(const cut_mlp *m, float *scale, float *shift);
/* Optional linear skip term: y = scale * y_hat + shift + J x with
 * J[n_out][n_in] (host, FP32, copied), applied in FP32 on the CUDA cores in
 * the last layer's epilogue and removed from the targets in training
 * (t_hat = (t - shift - J x) / scale), so that the network learns only what
 * a linear model misses.  J = NULL removes it. */
cut_status cut_mlp_set_linear(cut_mlp *m, const float *J);
/* Fit the linear skip term and the output affine from training data on the
 * device, in FP64: the least-squares affine map (1, x) -> t over the batch
 * (normal equations, Cholesky with a 1e-12 relative ridge) gives shift =
 * intercept and J = slopes; scale = the residual RMS of each output divided
 * by sqrt(weight[o]) (host, optional, > 0: a larger weight makes that
 * output's error count more in the loss).  The network then learns only
 * what the affine map misses.  device in: x[batch][n_in] (FP32),
 * t[batch][n_out] (FP64).  At most 63 inputs.  Errors: INVALID_ARG,
 * UNSUPPORTED, OUT_OF_MEMORY, CUDA. */
cut_status cut_mlp_fit_linear(cut_mlp *m, int batch, const float *x, const double *t, const float *weight,
                              cut_stream_t stream);
/* Statistics of an ensemble of K independently trained networks on the same
 * queries, the error signal of the surrogate's gate: mean[b][o] = average
 * of the K outputs (members summed in order; mean may be NULL) and
 * spread[b] = max over the outputs with mask[o] != 0 of (max_k - min_k).
 * host in: preds[K] (device pointers to [batch][n_out] FP32 outputs);
 * device in: mask[n_out]; device out: mean, spread[batch].  1 <= K <= 16.
 * Uses the current device.  Errors: INVALID_ARG, CUDA. */
cut_status cut_mlp_ensemble_stats(int K, int batch, int n_out, const float *const *preds, const uint8_t *mask,
                                  float *mean, float *spread, cut_stream_t stream);
/* number of parameters in the flat layout W1, b1, W2, b2, W3, b3 (W [out][in]) */
int64_t cut_mlp_param_count(const cut_mlp *m);
/* host out: parameters (grads = 0) or the gradients of the last backward
 * (grads = 1), flat layout above.  Synchronous. */
cut_status cut_mlp_get_params(cut_mlp *m, float *host, int grads);
/* host in: parameters, flat layout above.  Synchronous. */
cut_status cut_mlp_set_params(cut_mlp *m, const float *host);
/* device in: x[batch][n_in] (FP32); device out: y[batch][n_out] (FP32). */
cut_status cut_mlp_forward(cut_mlp *m, int batch, const float *x, float *y, cut_stream_t stream);
/* Gradients of the mean squared error over batch x n_out of the
 * standardised targets, kept inside m.  device in: x[batch][n_in],
 * target[batch][n_out]; device in/out: loss (one float, the loss is ADDED,
 * may be NULL). */
cut_status cut_mlp_backward(cut_mlp *m, int batch, const float *x, const float *target, float *loss,
                            cut_stream_t stream);
/* One AdamW update (decoupled weight decay, none on biases) from the last
 * backward's gradients. */
cut_status cut_mlp_adamw_step(cut_mlp *m, float lr, float beta1, float beta2, float eps, float weight_decay,
                              cut_stream_t stream);
/* Synchronises; TIMEOUT if a tensor-core pipeline wait gave up since the
 * last call (each wait gives up after about one second; the kernel then
 * writes nothing, waits for its own copies, frees its tensor memory and
 * returns, so the context stays usable).  The flag is cleared once reported. */
cut_status cut_mlp_status(cut_mlp *m);
/* Failure injection for tests (no fault, no hang): while `on` is nonzero
 * every GEMM of m issues no operand copies, so its pipeline wait runs out
 * after about a second and cut_mlp_status reports TIMEOUT; outputs of those
 * calls are undefined.  Synchronises the device.  Errors: INVALID_ARG, CUDA. */
cut_status cut_mlp_inject_stall(cut_mlp *m, int on);

#ifdef __cplusplus
}
#endif
#endif /* CUT_H */
