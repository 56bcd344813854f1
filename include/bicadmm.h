/*
 * bicadmm.h - C ABI of the B300 Bi-cADMM solver library (libbicadmm.so).
 *
 * Solves the sparse machine-learning problem of Sec. 2, eq. (p:SML):
 *
 *     minimise_x  sum_i l_i(A_i x; b_i) + ||x||_2^2 / (2 gamma)   subject to  ||x||_0 <= kappa,
 *
 * with the bi-linear consensus ADMM of Sec. 3 (iterations block, eqs. x-min-step ..
 * global-lambda-updae, scaled form eqs. u-update and v-update).  The rows of A are split
 * into N sample shards (the paper's nodes, eq. p:bi-convex) and each shard's local prox
 * (eq. p:x-subp) is evaluated by the feature-split sharing ADMM of Sec. 3.1 over M column
 * blocks (eqs. p:GPU;x, p:GPU;omega, p:GPU;nu; Algorithm 2).  All shards and blocks live on
 * one GPU; there is no inter-process communication.
 *
 * Conventions shared by every call:
 *  - Matrices are row-major.  A is the full m x n data matrix; shard i is a contiguous row
 *    range and block j a contiguous column range, the first (m mod N) shards and
 *    (n mod M) blocks one longer than the rest.
 *  - Every call returns a status code (BICADMM_OK = 0, negative on error); no C++
 *    exception crosses this boundary.  After an error, bicadmm_last_error() describes it.
 *  - All GPU work is ordered on the CUDA stream given to bicadmm_create().  Calls that
 *    return host data (get_x, get_state, step/solve with an info pointer) synchronise that
 *    stream before returning.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef BICADMM_H
#define BICADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bicadmm_ctx* bicadmm_t;

/* Loss l(q; b) of a row (Sec. 2 lists the models; squared as eq. p:sls, without 1/2).
 * SQUARED: (q - b)^2.  LOGISTIC: log(1 + exp(-b q)), b in {-1,+1}.
 * SQHINGE: max(0, 1 - b q)^2, b in {-1,+1}.
 * SOFTMAX (sparse softmax regression, K = 2..16 classes): the model is an n x K matrix W,
 *   q = a_r W is a K-vector, l(q; y) = logsumexp(q) - q_y with y in {0, .., K-1} given as
 *   b_r (an integral value).  Every n-space array (x_i, u_i, z, s, the model returned by
 *   bicadmm_get_x) holds W flattened feature-major, entry (c, k) at c*K + k; kappa bounds
 *   the number of nonzero entries of W (entrywise sparsity, ties to the lowest flat index).
 *   omega and nu are m x K, row-major. */
enum {
  BICADMM_LOSS_SQUARED = 0,
  BICADMM_LOSS_LOGISTIC = 1,
  BICADMM_LOSS_SOFTMAX = 2,
  BICADMM_LOSS_SQHINGE = 3
};

/* Precision of the stored A and of the per-row arithmetic on the A products.
 * FP64: everything in FP64.  FP32: A, A x and A'd in FP32; the n-space state, the block
 * factors and all residuals stay in FP64; the Gram matrices A_ij'A_ij of the setup run on
 * the tensor cores in TF32 with each element split into a TF32 pair hi + lo (three
 * products per pair, about 22 bits of A), accumulated in FP32.  BF16: A stored in BF16
 * (rounded to nearest even at setup; half the bytes of FP32), its products accumulated in
 * FP32, everything else as in FP32 mode.  TF32: A stored in 32-bit words rounded to TF32
 * (10 mantissa bits, nearest even) at setup, the precision the tensor cores multiply in;
 * one TF32 product per pair forms the Gram matrices exactly in the FP32 accumulator; the
 * rest as in FP32 mode (the A x and A'd GEMVs of K = 1 read 4 bytes per element on the
 * CUDA cores either way).  The Gram matrices, factors and polish use the stored (rounded) A. */
enum { BICADMM_PREC_FP64 = 0, BICADMM_PREC_FP32 = 1, BICADMM_PREC_BF16 = 2, BICADMM_PREC_TF32 = 3 };

/* Element type of caller buffers passed to bicadmm_setup(). */
enum { BICADMM_DTYPE_F64 = 0, BICADMM_DTYPE_F32 = 1, BICADMM_DTYPE_BF16 = 2 };

enum {
  BICADMM_OK = 0,
  BICADMM_ERR_ARG = -1,         /* invalid argument or size */
  BICADMM_ERR_OOM = -2,         /* device allocation failed */
  BICADMM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  BICADMM_ERR_STATE = -4,       /* call out of order (e.g. step before setup) */
  BICADMM_ERR_NUMERIC = -5,     /* non-positive pivot, NaN/Inf in a residual */
  BICADMM_ERR_TIMEOUT = -6,     /* a device-side wait hit its limit */
  BICADMM_ERR_UNSUPPORTED = -7  /* valid request this build does not implement */
};

/* Fields readable with bicadmm_get_state(); lengths in doubles. */
enum {
  BICADMM_FIELD_X = 0,      /* N x nK: local estimates x_i (row i = shard i)          */
  BICADMM_FIELD_U = 1,      /* N x nK: scaled consensus duals u_i (eq. u-update)      */
  BICADMM_FIELD_Z = 2,      /* nK: consensus variable z                               */
  BICADMM_FIELD_S = 3,      /* nK: bi-linear variable s in S^kappa                    */
  BICADMM_FIELD_OMEGA = 4,  /* m x K: omega-bar of eq. (p:GPU;omega), shard-major rows */
  BICADMM_FIELD_NU = 5,     /* m x K: sharing duals nu of eq. (p:GPU;nu)              */
  BICADMM_FIELD_SCALARS = 6, /* 3: t, v (scaled bi-linear dual, eq. v-update), tau   */
  BICADMM_FIELD_P = 7        /* sum over (i, j) of n_j^2: the block inverses
                                (rho_l A_ij'A_ij + c0 I)^-1 of the x_ij solve, shard-major
                                then block, each n_j x n_j row-major (setup's output)   */
};

typedef struct {
  int32_t loss;          /* BICADMM_LOSS_*                                              */
  int32_t precision;     /* BICADMM_PREC_*                                              */
  int64_t m, n;          /* rows and columns of A                                       */
  int64_t K;             /* classes: 2..16 for SOFTMAX, 1 for every other loss          */
  int32_t N_shards;      /* N >= 1 sample shards (1 <= N <= m)                          */
  int32_t M_blocks;      /* M >= 1 feature blocks per shard (1 <= M <= n)               */
  int64_t kappa;         /* sparsity level, 1 <= kappa <= n K                           */
  double gamma;          /* ridge weight, > 0                                           */
  double rho_c;          /* consensus penalty, > 0                                      */
  double rho_b;          /* bi-linear penalty, > 0 (0 selects 0.5 rho_c)                */
  double rho_l;          /* sharing (feature-split) penalty, > 0 (0 selects rho_c)      */
  int32_t inner_iters;   /* J: sharing-ADMM sweeps per outer iteration, >= 1            */
  int32_t newton_iters;  /* cap on Newton steps of the logistic / softmax omega prox   */
  int32_t max_iters;     /* outer-iteration cap of bicadmm_solve()                      */
  int32_t check_every;   /* solve(): read residuals back every this many iterations     */
  double tol_rel;        /* solve(): stop when max(p_rel, d_rel, b_rel, i_rel) <= tol   */
  int32_t pass_rows;     /* tuning: rows per staged panel of the A pass (0 = auto; for
                            BF16 storage with K > 1 and n <= 2048 the tensor-core pass:
                            128 = on pairs of SMs (a two-CTA cluster splits the columns;
                            chosen by auto when n > 128), 64 = on single SMs (chosen by
                            auto when n <= 128); 8 = its CUDA-core pass)               */
  int32_t pass_stages;   /* tuning: panels in flight per CTA (0 = auto)                 */
} bicadmm_params;

typedef struct {
  int32_t iters;         /* outer iterations run since setup                            */
  int32_t converged;     /* 1 if the stop rule held at the last check                   */
  double p_r, d_r, b_r;  /* primal, dual, bi-linear residuals (Sec. 3, Termination)     */
  double i_r;            /* inner sharing residual ||Axbar - omega||                   */
  double p_rel, d_rel, b_rel, i_rel;  /* relative forms used by the stop rule           */
  double t, v, tau;      /* bi-linear scalars and the l1 multiplier / (N rho_c)         */
  int64_t kernel_launches;  /* iteration kernels this handle has launched since create
                               (step/solve; the objective's kernels are not counted)   */
  double objective;      /* F(z) = sum_r l(a_r z; b_r) + ||z||^2 / (2 gamma), problem
                            (p:SML) of Sec. 2 at the consensus iterate z, with the stored
                            (rounded) A and b and every product and sum in FP64.  Computed on the
                            device when info is returned (three small launches; a row
                            product runs only over the features where z is nonzero).     */
} bicadmm_info;

/* Fill *p with defaults: squared loss, FP64, gamma 10, rho_c 1, rho_b = rho_c/2,
 * rho_l = rho_c, J = 1, 50 Newton steps, 10000 iterations, tol 1e-6, check every 10.
 * Sizes (m, n, N, M, kappa) are zero and must be set by the caller. */
int bicadmm_default_params(bicadmm_params* p);

/* Validate *params and allocate all device buffers for that problem size (n K <= 32768).
 * stream: a cudaStream_t (NULL = legacy default stream), not owned by the handle.
 * On success *out owns the buffers until bicadmm_destroy().  Errors: ERR_ARG for an
 * invalid size or penalty, ERR_OOM if the device buffers do not fit, ERR_UNSUPPORTED for
 * a loss or width this build does not implement. */
int bicadmm_create(const bicadmm_params* params, void* stream, bicadmm_t* out);

/* A sparsity path (not part of the paper; the paper's kappa of eq. (p:SML) is what a user
 * sweeps): `count` = 2..16 instances of one problem that differ only in kappa (kappas[q],
 * 1 <= kappas[q] <= n), solved together on one copy of A.  *params describes the shared
 * problem (loss squared, logistic or squared hinge, K = 1; params->kappa is ignored) and
 * n * count <= 32768.  The instances are the columns of the multi-column kernels: one pass
 * over A per inner sweep forms A X and A'D for all of them (skinny GEMMs; on the tensor
 * cores for BF16 storage and n <= 2048, as the softmax pass), each row's omega prox of eq.
 * (p:GPU;omega) runs per column, the block solve of eq. (p:GPU;x) takes the count right-hand
 * sides, and each instance has its own consensus step (its own kappa, t, v, residual
 * records), run by its own CTA.  Setup, step, solve, set_graph, get_state (x, u, z, s as n x
 * count, feature-major: entry (c, q) at c count + q) and destroy work as for any handle; step
 * and solve report instance 0 in *info and solve stops when every instance meets tol_rel.
 * The shard sums p_r and the inner residual i_r cover every instance together.  Each
 * instance's iterates are those of its own handle up to rounding of the shared sums.
 * bicadmm_path_info fills *info for one instance (with its objective); bicadmm_path_get_x
 * copies its z (n doubles) and, when support_out is non-NULL, its kappas[q] largest |z|
 * (ascending indices, ties to the lowest).  bicadmm_get_x with polished = 1 or a support is
 * ERR_UNSUPPORTED on a path (no polish for paths in this build). */
int bicadmm_create_path(const bicadmm_params* params, int32_t count, const int64_t* kappas,
                        void* stream, bicadmm_t* out);
int bicadmm_path_info(bicadmm_t h, int32_t instance, bicadmm_info* info);
int bicadmm_path_get_x(bicadmm_t h, int32_t instance, double* x_host, int64_t len,
                       int64_t* support_out);

/* Load the data and build the per-block factors; resets the iteration state to zero.
 * A: m rows of n values with row stride lda (elements, lda >= n), type A_dtype, in host
 *    memory (A_on_device = 0) or device memory (1).  b: m values of type b_dtype (targets
 *    for SQUARED, class indices 0..K-1 for SOFTMAX, labels +/-1 otherwise), host or device;
 *    b_dtype BF16 is not accepted.  Invalid softmax labels give ERR_ARG.  Both are copied (and converted
 *    to the handle's precision); the caller keeps ownership and may free them on return.
 * Builds G_ij = A_ij' A_ij and the inverse of rho_l G_ij + (1/(N gamma) + rho_c) I, the
 * matrix of the x_ij solve of eq. (p:GPU;x), in FP64.  Errors: ERR_ARG, ERR_CUDA,
 * ERR_NUMERIC (a block matrix is not positive definite). */
int bicadmm_setup(bicadmm_t h, const void* A, int32_t A_dtype, int64_t lda, int32_t A_on_device,
                  const void* b, int32_t b_dtype, int32_t b_on_device);

/* Run exactly n_iters >= 0 outer iterations (each with J inner sweeps).  If info is
 * non-NULL the stream is synchronised and *info filled; with info NULL the call only
 * enqueues work.  Errors: ERR_STATE before setup, ERR_TIMEOUT / ERR_NUMERIC reported by
 * the device (checked whenever info is requested). */
int bicadmm_step(bicadmm_t h, int32_t n_iters, bicadmm_info* info);

/* Iterate until the stop rule holds (checked every check_every iterations) or max_iters
 * iterations have run in this call.  Not converging is not an error: info->converged = 0. */
int bicadmm_solve(bicadmm_t h, bicadmm_info* info);

/* Replay outer iterations from a CUDA graph: with iters_per_graph > 0, bicadmm_step (and so
 * bicadmm_solve) runs its first iteration eagerly, captures iters_per_graph iterations of
 * this handle into a graph once (recorded, not run), then runs the requested iterations as
 * whole replays plus an eager remainder.  The iterates are those of eager stepping; only
 * the host launch cost changes (it dominates small problems).  0 switches replay off and
 * frees the graph.  Needs a non-default stream (ERR_ARG otherwise); ignored while
 * profiling is on. */
int bicadmm_set_graph(bicadmm_t h, int32_t iters_per_graph);

/* Copy the model to host memory x_host[len], len = n K (the flattened n x K W for SOFTMAX).
 * polished = 0: the consensus iterate z.  polished = 1: the solution of the problem
 * restricted to S = the kappa largest |z_r| (ties to the lowest index), solved in FP64 by
 * damped Newton on the device (not part of the paper's algorithm; kappa <= 1024, else
 * ERR_UNSUPPORTED; ERR_NUMERIC if the restricted Hessian is not positive definite).
 * For SOFTMAX the support is the kappa largest entries of the flattened W and the restricted
 * problem is the cross-entropy over those entries (the rest of W held at zero).
 * support_out (kappa entries, ascending) receives S when non-NULL.  Synchronises the
 * stream; the first polished call allocates the polish buffers (kappa x m doubles; twice
 * that plus 4 m K doubles for SOFTMAX). */
int bicadmm_get_x(bicadmm_t h, double* x_host, int64_t len, int32_t polished, int64_t* support_out);

/* Copy one state field (BICADMM_FIELD_*) to host memory out_host[len]; len must equal the
 * field's length.  Synchronises the stream.  For tests, checkpoints and diagnostics. */
int bicadmm_get_state(bicadmm_t h, int32_t field, double* out_host, int64_t len);

/* Per-iteration residual trace: copies the records of the last min(iterations, 4096,
 * max_records) outer iterations, oldest first, to out_host (15 doubles per record:
 * iteration, p_r, d_r, b_r, i_r, p_rel, d_rel, b_rel, i_rel, t, v, tau, ||z||, the number
 * of Newton steps of the (z,t) root solve, and 1 when that step visited only the entry
 * lists of the all-SM prep kernel (K > 1, warm-started), else 0), and their count to
 * *n_out.  The
 * records are written on the device every iteration (Sec. 3, Termination) and read only
 * here.  Synchronises the stream. */
int bicadmm_get_trace(bicadmm_t h, double* out_host, int64_t max_records, int64_t* n_out);

/* Profiling with CUDA events on the handle's stream.  on = 1: every launch of the fused
 * A-pass kernel is bracketed; on = 2: every kernel of the iteration (pass, x-update, dual,
 * extra right-hand-side sweeps); on = 0: off.  Switching resets the records.
 * bicadmm_get_kernel_times() synchronises and writes, per kernel kind (0 pass, 1 x-update,
 * 2 dual, 3 right-hand side), the summed device time in ms to ms_out[4] and the launch
 * count to launches_out[4] (either may be NULL); reset != 0 clears the records.
 * bicadmm_get_pass_time() returns the pass's entries and clears the records. */
int bicadmm_set_profiling(bicadmm_t h, int32_t on);
int bicadmm_get_kernel_times(bicadmm_t h, double* ms_out, int64_t* launches_out, int32_t reset);
int bicadmm_get_pass_time(bicadmm_t h, double* ms_out, int64_t* launches_out);

/* Fault injection for tests (the paper has no counterpart; no effect unless called).
 * From the next K = 1 A-pass launch on, the load of panel `panel` (a global panel index,
 * 0 <= panel < the handle's panel count) is never posted: neither its expected byte count
 * nor its copy is issued, so the CTA that owns it waits at most wait_limit_cycles (>= 1000
 * SM cycles) on that stage, records BICADMM_ERR_TIMEOUT, lets the copies it did post land
 * and exits; no other CTA waits on it and nothing faults.  The handle's iterates are then
 * invalid: destroy it.  panel < 0 disarms the hook and restores the normal wait limit
 * (about 2 s).  Errors: ERR_ARG (no such panel, K > 1, limit too small), ERR_STATE with
 * graph replay on. */
int bicadmm_inject_pass_stall(bicadmm_t h, int64_t panel, int64_t wait_limit_cycles);

/* Allocation-free consensus update.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc when they call in, such as code running while a
 * stream is captured into a CUDA graph, services whose device memory belongs to another
 * allocator or pool, and latency-bound loops that must avoid the implicit synchronisation
 * of cudaMalloc/cudaFree.  It runs the same (z, t) root solve, top-kappa s update and v
 * update as one outer iteration of bicadmm_step, on caller buffers, and allocates nothing:
 * its scratch (about 1 MB: breakpoints, their coefficients and sort keys for up to 32768
 * entries, scalars and a status word) is a file-scope device array in the library, held by
 * every GPU that loads the library until the process exits.
 *   w    device, n doubles, in:  (1/N) sum_i (x_i + u_i)
 *   z    device, n doubles, in: z^k (for the dual residual), out: z^{k+1}
 *   s    device, n doubles, in: s^k, out: s^{k+1}
 *   tvt  device, 4 doubles, in: tvt[1] = v^k; out: t^{k+1}, v^{k+1}, tau, device status
 *        (0 = ok, nonzero = the root iteration hit its bound)
 *   n <= 32768, 1 <= kappa <= n, N_shards >= 1, rho_c > 0, rho_b > 0; larger n is rejected
 *   with BICADMM_ERR_ARG.  stream: cudaStream_t (NULL = legacy default stream).
 * Work is enqueued on stream; the call does not synchronise.  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress) for that device; make
 * that first call before any stream capture.  Every call on a device shares the one scratch
 * array and overwrites it, so calls that may overlap on the GPU (other streams, other host
 * threads) race: order them on one stream.  Returns BICADMM_ERR_ARG / BICADMM_ERR_CUDA on
 * failure (no handle, so no last-error text). */
int bicadmm_consensus_step_noalloc(const double* w, double* z, double* s, double* tvt, int64_t n,
                                   int64_t kappa, int32_t N_shards, double rho_c, double rho_b,
                                   void* stream);

/* Batched execution (not part of the paper): advance several independent, set-up handles
 * together, one launch per kernel kind per outer iteration for all of them (x-update, one
 * persistent A pass over a panel list spanning every instance's shards, consensus step,
 * dual update).  Each instance's iterates are those of bicadmm_step up to rounding (the
 * A'd partial sums are grouped differently).  Requirements: every handle set up, all of
 * one precision and device, inner_iters = 1, K = 1.  The batch references the handles (it does
 * not own them); destroy the batch before any of its handles.  Handles may still be stepped
 * alone between batch steps.
 * flags: BICADMM_BATCH_GRAPH captures one iteration into a CUDA graph and replays it (needs
 * a non-default stream); BICADMM_BATCH_PROFILE times each launch (not with GRAPH);
 * BICADMM_BATCH_AUTOTUNE spends the first iterations timing each
 * tiling that fits — shared-memory stage size (16..96 KB; each instance's panels take as
 * many rows as fit in a stage, at most 8, or at most 8 per row group for instances whose
 * rows hold at most 128 16-byte vectors, which run in a second pass launch) and stage
 * count (1..4; one stage only from 32 KB) — 2 iterations each (ordinary iterations of every
 * instance), and keeps the fastest.  Kind 0 of bicadmm_batch_kernel_times covers both pass launches.
 * stream: cudaStream_t used for all batch work.
 * bicadmm_batch_step runs n_iters iterations of every instance (does not synchronise) and
 * writes the batch's kernel-launch count so far to *launches_out when non-NULL.
 * bicadmm_batch_tiling reports the stage size in KB and the stage count in use.  Errors with a NULL batch
 * are described by bicadmm_batch_last_error(NULL). */
typedef struct bicadmm_batch_ctx* bicadmm_batch_t;
enum { BICADMM_BATCH_GRAPH = 1, BICADMM_BATCH_AUTOTUNE = 2, BICADMM_BATCH_PROFILE = 4 };
int bicadmm_batch_create(bicadmm_t* handles, int32_t count, void* stream, int32_t flags,
                         bicadmm_batch_t* out);
int bicadmm_batch_step(bicadmm_batch_t b, int32_t n_iters, int64_t* launches_out);
int bicadmm_batch_tiling(bicadmm_batch_t b, int32_t* stage_kb_out, int32_t* stages_out);
/* With BICADMM_BATCH_PROFILE (eager launches only) every batched launch is bracketed by CUDA
 * events; this synchronises and writes per kernel kind (0 pass, 1 x-update, 2 dual,
 * 3 consensus) the summed ms and launch counts since the last call, then clears them. */
int bicadmm_batch_kernel_times(bicadmm_batch_t b, double* ms_out, int64_t* launches_out);
int bicadmm_batch_destroy(bicadmm_batch_t b);
const char* bicadmm_batch_last_error(bicadmm_batch_t b);

/* Device bytes a handle with these parameters allocates (including one polished get_x),
 * and the extra bytes its setup holds temporarily.  Needs a current CUDA device. */
int bicadmm_estimate_bytes(const bicadmm_params* params, int64_t* device_bytes,
                           int64_t* setup_extra_bytes);

/* Serving (not part of the paper): a request loop with continuous batching.  Requests are
 * complete solves (A, b and parameters) submitted with an arrival time on the server's
 * clock (seconds since bicadmm_server_create, bicadmm_server_clock).  bicadmm_server_run
 * works in rounds until every submitted request is finished (or, with no request active,
 * the next arrival is later than `until`):
 *   - admit: arrived requests, in arrival order, get a handle (device copy of A and b,
 *     factors, iteration state) while the estimated device bytes stay within
 *     hbm_budget_bytes and at most max_active are active; a request that can never fit
 *     finishes with BICADMM_ERR_OOM;
 *   - one batched round (bicadmm_batch_step over every active request, CUDA graph when
 *     use_graph) of up to iters_per_round iterations, cut short so no request passes its
 *     max_iters; requests arriving meanwhile are admitted while the round runs;
 *   - retire: a request whose residuals meet its tol_rel (checked at round ends) or that
 *     reached max_iters is polished (when `polish`), copied to host and its memory freed.
 * Each request's iterates are those of solving it alone up to rounding (the batch only
 * regroups partial sums).  The caller keeps A and b of a request valid until it finishes.
 * All requests use the server's precision and inner_iters = 1.
 * Threads: bicadmm_server_run works on one host thread; bicadmm_server_submit, _set_open,
 * _result, _timing, _stats and _clock may be called from other threads at the same time
 * (requests that arrive while a run loops are admitted by it).  Create and destroy are not
 * concurrent with anything else.  Errors of submit and result are returned as codes only
 * (no last-error text, which belongs to the run thread). */
typedef struct bicadmm_server_ctx* bicadmm_server_t;
typedef struct {
  int64_t hbm_budget_bytes;  /* device bytes the active requests may hold              */
  int32_t max_active;        /* requests in flight at most                             */
  int32_t iters_per_round;   /* iterations per batched round                           */
  int32_t precision;         /* BICADMM_PREC_* of every request                        */
  int32_t use_graph;         /* replay rounds from a captured CUDA graph               */
  int32_t polish;            /* results are polished (kappa <= 1024)                   */
  int32_t pad;
} bicadmm_server_params;
int bicadmm_server_create(const bicadmm_server_params* sp, bicadmm_server_t* out);
double bicadmm_server_clock(bicadmm_server_t s);
int bicadmm_server_submit(bicadmm_server_t s, const bicadmm_params* p, const void* A,
                          int32_t A_dtype, int64_t lda, int32_t A_on_device, const void* b,
                          int32_t b_dtype, int32_t b_on_device, double arrival, int64_t* id_out);
int bicadmm_server_run(bicadmm_server_t s, double until, int64_t* completed_out);
/* open != 0: bicadmm_server_run does not return when nothing is active or waiting; it waits
 * for submissions (polling every 0.5 ms) until its `until` has passed or open is set to 0
 * (from any thread).  open = 0 (the default): it returns once every submitted request has
 * finished. */
int bicadmm_server_set_open(bicadmm_server_t s, int32_t open);
/* Time breakdown.  id >= 0 (a finished request; ERR_STATE before): out[7] = arrival,
 * admission (its create + setup start), setup end, retirement start (objective, polish,
 * copy-out), completion, all seconds on the server's clock, then its iterations and the
 * batched rounds it took part in.  id = -1: out[7] = batch rebuilds (the active set
 * changed), seconds rebuilding, seconds waiting for rounds on the device, seconds admitting
 * (create + setup), seconds retiring, rounds, and the server's clock. */
int bicadmm_server_timing(bicadmm_server_t s, int64_t id, double* out);
/* Result of a finished request: x (n doubles; polished if the server polishes), support
 * (kappa indices), info, and times_out[3] = arrival, admission, completion.  Returns the
 * request's own status when it failed. */
int bicadmm_server_result(bicadmm_server_t s, int64_t id, double* x_host, int64_t len,
                          int64_t* support_out, bicadmm_info* info, double* times_out);
/* counters_out[5]: submitted, finished, rounds, peak estimated device bytes, launches. */
int bicadmm_server_stats(bicadmm_server_t s, int64_t* counters_out);
int bicadmm_server_destroy(bicadmm_server_t s);
const char* bicadmm_server_last_error(bicadmm_server_t s);

/* Free every device buffer of the handle (synchronises its stream).  NULL is accepted. */
int bicadmm_destroy(bicadmm_t h);

/* Text of the last error on this handle ("" if none); valid until the next call on h.
 * With h == NULL returns the last error of a failed bicadmm_create() on the calling host
 * thread. */
const char* bicadmm_last_error(bicadmm_t h);

#ifdef __cplusplus
}
#endif

#endif /* BICADMM_H */
