/*
 * spai.h - C ABI of the GB300 (sm_103a) SPAI-preconditioned CG library.
 *
 * The library solves sparse SPD systems A x = b with conjugate gradients
 * preconditioned by a factorised sparse approximate inverse
 *
 *     M^-1 = G G^T + eps I                         (paper, Eq. 1)
 *
 * where G has the sparsity pattern of A and its values come either from the
 * GNN forward pass of Sec. 3.2.2 (Eqs. 3-5) or from the caller.  Applying M^-1
 * costs two sparse mat-vecs and an axpy (Sec. 3.2.1, Eq. 2); the solver is
 * Algorithm 1 of App. A (standard PCG with the true residual recomputed every
 * 50 iterations).
 *
 * Conventions for every call:
 *  - Pointers documented as "device" must point to memory of the current CUDA
 *    device; "host" pointers to ordinary (or pinned) host memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Work is enqueued on it; a call returns after its results are
 *    complete unless stated otherwise.
 *  - CSR matrices: int32 row pointers (n+1) starting at 0, int32 column
 *    indices with strictly ascending columns in each row, no duplicates, the
 *    diagonal present in every row and a structurally symmetric pattern
 *    (A is SPD).  Values are float64.
 *  - The caller owns every buffer it passes and keeps it alive and unmodified
 *    for the duration of the call (for the server: until the request
 *    completes).  Handles (spai_pattern, spai_precond, spai_system,
 *    spai_server) own their own device memory and free it in *_destroy.
 *  - Return value: SPAI_OK (0) or a negative SPAI_ERR_* code.  No C++
 *    exception crosses this boundary.  spai_last_error() returns a message
 *    for the calling thread's last failure.
 *  - If the CUDA kernels of the library cannot run (no device, wrong
 *    architecture) every compute call fails with SPAI_ERR_CUDA; there is no
 *    CPU fallback.
 */
#ifndef SPAI_H
#define SPAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----- status codes ----- */
#define SPAI_OK                 0
#define SPAI_ERR_INVALID       -1  /* bad argument (null pointer, bad enum, n < 0, ...) */
#define SPAI_ERR_BAD_CSR       -2  /* CSR violates the conventions above */
#define SPAI_ERR_SHAPE         -3  /* sizes of A, G, weights or features disagree */
#define SPAI_ERR_CUDA          -4  /* a CUDA runtime call or kernel launch failed */
#define SPAI_ERR_OOM           -5  /* device allocation failed */
#define SPAI_ERR_BREAKDOWN     -6  /* PCG breakdown: d^T q <= 0 or a non-finite scalar */
#define SPAI_ERR_NOT_CONVERGED -7  /* max_iter reached; x holds the last iterate */
#define SPAI_ERR_TIMEOUT       -8  /* a bounded device-side wait gave up */
#define SPAI_ERR_TOO_LARGE     -9  /* request can never fit under the server's memory cap */
#define SPAI_ERR_NOT_FOUND    -10  /* unknown system id or ticket */

/* ----- value types ----- */
#define SPAI_F64  0
#define SPAI_F32  1
#define SPAI_BF16 2
#define SPAI_F16  3

/* ----- pattern kinds for G (Sec. 3.2.2 keeps A's pattern: FULL) ----- */
#define SPAI_PATTERN_FULL  0  /* pattern of G = pattern of A (learned G) */
#define SPAI_PATTERN_LOWER 1  /* entries with j <= i */
#define SPAI_PATTERN_UPPER 2  /* entries with j >= i (a classical factorised SPAI: G = W^T) */

/* ----- solver options ----- */
#define SPAI_PREC_F64   0  /* everything in float64 */
#define SPAI_PREC_MIXED 1  /* float32 PCG with float64 refinement of x and of the residual */

#define SPAI_CRIT_RESIDUAL 0  /* stop when ||b - A x|| <= rtol ||b|| (tables of Sec. 4.2) */
#define SPAI_CRIT_PRECOND  1  /* Algorithm 1's own test: r^T M^-1 r <= rtol^2 r0^T M^-1 r0 */

#define SPAI_MSG_LATENT 0  /* message MLP reads the latent edge state h_ij (default) */
#define SPAI_MSG_RAW    1  /* message MLP reads the raw edge feature e_ij as Eq. 4 prints it */

typedef struct {
  int64_t n;              /* rows = columns */
  int64_t nnz;            /* stored entries */
  const int32_t* rowptr;  /* device, n+1 */
  const int32_t* colidx;  /* device, nnz */
  const void* val;        /* device, nnz values of type `dtype` */
  int32_t dtype;          /* SPAI_F64 */
} spai_csr;

typedef struct spai_pattern spai_pattern;
typedef struct spai_precond spai_precond;
typedef struct spai_system spai_system;
typedef struct spai_server spai_server;

/* GNN weights (Sec. 3.2.2; sizes of Sec. 4.1).  `blob` is a device array of
 * float32 holding, for every MLP in the order E_n, E_e, (f_m, f_v, f_e) per
 * layer, D, the block [W1 (24 x fan_in, row-major), b1 (24), W2 (fan_out x 24,
 * row-major), b2 (fan_out)].  Every MLP is Linear -> ReLU -> Linear with 24
 * hidden units.  Fan-ins: E_n d_node, E_e b^2, f_m 72 (or 48 + b^2 with
 * SPAI_MSG_RAW), f_v 24, f_e 72, D 24; fan-outs 24 except D (b^2), b the
 * block size (1, or 3 for the paper's 3 x 3 blocks). */
typedef struct {
  const float* blob;   /* device */
  int64_t count;       /* number of floats in blob (checked) */
  int32_t d_node;      /* node feature width, 1..16 */
  int32_t n_layers;    /* message-passing layers L, 0..8 (paper: 4) */
  int32_t msg_edge;    /* SPAI_MSG_LATENT or SPAI_MSG_RAW */
  int32_t block;       /* b: 1 (0 is read as 1) or 3 */
} spai_gnn_weights;

typedef struct {
  double rtol;             /* target ||b - A x|| / ||b|| (paper: 1e-8) */
  int64_t max_iter;        /* iteration cap (all inner iterations); <= 0: min(10 n, 1e6) */
  int32_t replace_period;  /* recompute r = b - A x every this many iterations (50); 0 = never */
  int32_t criterion;       /* SPAI_CRIT_* */
  int32_t precision;       /* SPAI_PREC_* */
  double inner_rtol;       /* mixed only: when the float32 residual has dropped by this factor since the
                              last refinement, fold the float32 correction into the float64 x and
                              replace r by the float64 b - A x (also every replace_period iterations
                              and to confirm convergence); outside (0, 1): 0.1 */
  int32_t max_outer;       /* mixed only: cap on float64 refinements (<= 0: none) */
  int32_t record_history;  /* nonzero: write ||r|| after every iteration into `history` */
  double* history;         /* device, history_len doubles (history[0] = ||r_0||), may be NULL */
  int64_t history_len;
  double* lanczos;         /* device, 2 lanczos_len doubles or NULL: the step length alpha_k of
                              iteration k at [2k] and the ratio beta_k = delta_{k+1} / delta_k that
                              follows it at [2k+1] (the CG / Lanczos coefficients, for
                              spai_ritz_extremes); single-system solves only */
  int64_t lanczos_len;
} spai_pcg_opts;

typedef struct {
  int64_t iters;         /* PCG iterations done (inner iterations for mixed) */
  int32_t outer_iters;   /* float64 refinements of x and r (mixed), else 0 */
  int32_t status;        /* SPAI_OK, SPAI_ERR_NOT_CONVERGED, SPAI_ERR_BREAKDOWN, ... */
  double true_rel_res;   /* ||b - A x|| / ||b|| in float64 at exit, computed on the device */
  double rec_rel_res;    /* recurrence residual at exit relative to ||b|| */
  int64_t history_written; /* entries written to opts->history */
  double engine_ms;      /* device time of the persistent PCG kernel launches (CUDA events on `stream`) */
  int64_t slots;         /* grid-wide phases the persistent kernel executed */
  int32_t launches;      /* persistent kernel launches of this solve */
  int32_t pad;
  int64_t lanczos_written; /* alpha values written to opts->lanczos (betas: one fewer, or as many) */
} spai_pcg_result;

/* ------------------------------------------------------------------------ *
 * Condition-number estimates from a solve's own coefficients (Sec. 4.5
 * measures preconditioners by kappa and Kaporin's condition number of
 * A M^-1).  PCG's step lengths alpha_j and ratios beta_j define the
 * tridiagonal Lanczos matrix T_k of M^-1 A:
 *   T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j][j+1] = sqrt(beta_j)/alpha_j.
 * Host functions (no device work); alpha has k entries, beta k - 1 (host
 * arrays, e.g. copied from opts->lanczos).  SPAI_ERR_INVALID for k < 1 or a
 * non-positive or non-finite coefficient.
 * ------------------------------------------------------------------------ */
/* Smallest and largest eigenvalue of T_k (Ritz values: inside the spectrum
 * of M^-1 A, the extremes converge first), by Sturm-sequence bisection;
 * kappa is estimated by *lam_max / *lam_min. */
int spai_ritz_extremes(const double* alpha, const double* beta, int64_t k, double* lam_min, double* lam_max);

/* Kaporin's condition number estimated by Gauss quadrature with T_m,
 * m = min(k, 400): (sum_i w_i theta_i) / exp(sum_i w_i log theta_i) with
 * Ritz values theta_i and weights w_i the squared first components of T_m's
 * eigenvectors -- the arithmetic over the geometric mean of the spectrum
 * weighted by the solve's normalised starting residual (an unbiased-in-
 * expectation stand-in for the plain means when that residual is random). */
int spai_ritz_kaporin(const double* alpha, const double* beta, int64_t k, double* kaporin);

/* ------------------------------------------------------------------------ *
 * sai_loss - the scale-invariant aligned-identity loss of Sec. 3.3 (Eq. 8)
 * with Hutchinson probes (Eq. 7), the quantity the paper trains G on:
 *   loss[j] = || A (G G^T + eps I) w_j / ||A|| - w_j ||_2^2,  j < k,
 * ||A|| = mean |A_ij| over stored entries.  A: device CSR (F64); M: any
 * preconditioner (its G^T, G and eps); w: device float64, n x k with the
 * probe index fastest (w[i * k + j] = entry i of probe j), 1 <= k <= 32;
 * loss: device float64[k].  Forward value only, float64 arithmetic, fixed
 * summation order.  Errors: SPAI_ERR_INVALID (k, null, dtype),
 * SPAI_ERR_SHAPE (sizes differ).
 * ------------------------------------------------------------------------ */
int spai_sai_loss(const spai_csr* A, const spai_precond* M, const double* w, int32_t k, double* loss, void* stream);

/* Gradient of the SAI loss for training (Sec. 3.3): the loss of every probe
 * as spai_sai_loss writes it, and in grad_g (device float64[nnz of G], the
 * order of G's CSR in the pattern) the gradient of the mean loss over the k
 * probes with respect to G's stored values:
 *   dL/dG_ij = (2/k) sum_p (a_i (G^T w_p)_j + w_pi (G^T a)_j),
 *   a = A (A M^-1 w_p / ||A|| - w_p) / ||A||  (A symmetric, as for every solve).
 * G's values are read in their storage type and the arithmetic is float64.
 * Same arguments and errors as spai_sai_loss. */
int spai_sai_loss_grad(const spai_csr* A, const spai_precond* M, const double* w, int32_t k, double* loss,
                       double* grad_g, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper): runs
 * a kernel whose grid barrier, mbarrier and item-flag wait (the ordering of
 * a fused step's two passes) can never complete, with a limit of limit_us
 * microseconds (1..1e6) each.  *detected = 1 when all three waits gave up,
 * flagged SPAI_ERR_TIMEOUT and returned (the context stays usable). */
int spai_selftest_wait_timeout(int64_t limit_us, int32_t* detected, void* stream);

/* Fills `o` with the defaults (rtol 1e-8, replace_period 50, RESIDUAL, F64). */
void spai_pcg_opts_default(spai_pcg_opts* o);

/* Thread-local message describing the last failed call (never NULL). */
const char* spai_last_error(void);

/* Library version and the CUDA architecture the kernels were built for. */
const char* spai_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads); lets callers count device work per call. */
uint64_t spai_kernel_launches(void);

/* ------------------------------------------------------------------------ *
 * build_pattern - sparsity pattern of G and its explicit transpose.
 * Sec. 3.2.2: G is written on A's pattern (FULL).  LOWER/UPPER restrict it to
 * a triangle for classical factorised inverses.  Validates A (CSR conventions
 * above); a bad CSR returns SPAI_ERR_BAD_CSR and creates nothing.
 * The handle stores G's CSR, G^T's CSR and perm with val_T[perm[e]] = val[e];
 * for FULL the transposed CSR equals G's and perm[e] is the index of (j, i).
 * ------------------------------------------------------------------------ */
int spai_build_pattern(const spai_csr* A, int32_t kind, spai_pattern** out, void* stream);

/* n and nnz of G. */
int spai_pattern_info(const spai_pattern* P, int64_t* n, int64_t* nnz_g);

/* Copies the pattern to caller device buffers (any pointer may be NULL):
 * rowptr/t_rowptr n+1 int32, colidx/t_colidx/perm nnz_g int32. */
int spai_pattern_export(const spai_pattern* P, int32_t* rowptr, int32_t* colidx,
                        int32_t* t_rowptr, int32_t* t_colidx, int32_t* perm, void* stream);

void spai_pattern_destroy(spai_pattern* P);

/* ------------------------------------------------------------------------ *
 * gnn_precond - the GNN forward pass of Sec. 3.2.2 (Eqs. 3-5) writing G.
 * Inputs: A (float64 CSR, device), the pattern P built from A with kind FULL,
 * node features v (device float32, n x d_node row-major) and weights W.
 * Edge features are A_ij / ||A|| with ||A|| = mean |A_ij| (Sec. 3.3).
 * G is stored in `g_dtype` (F64, F32, BF16 or F16) together with G^T, and
 * eps is the shift of Eq. 1.  Returns SPAI_ERR_SHAPE on a d_node / weight /
 * pattern mismatch.
 * Block form (W->block = b = 3, the paper's 3-unknowns-per-node systems):
 * A is the scalar CSR of a matrix made of dense b x b blocks (each block
 * row's b scalar rows list the same blocks in column order, b entries per
 * block; SPAI_ERR_BAD_CSR otherwise).  The GNN runs on the node graph
 * (n / b nodes, node_feat is (n / b) x d_node), every edge feature is the
 * block of A / ||A|| flattened row-major (||A|| over all stored scalar
 * entries) and the decoder writes one b x b block of G per edge, stored
 * in G's scalar CSR (A's pattern).
 * ------------------------------------------------------------------------ */
int spai_gnn_precond(const spai_csr* A, const spai_pattern* P, const float* node_feat,
                     const spai_gnn_weights* W, int32_t g_dtype, double eps,
                     spai_precond** out, void* stream);

/* Reverse pass of the GNN for training (Sec. 3.3 trains the GNN on the SAI
 * loss): the gradient, with respect to every weight of the blob W describes,
 * of sum_e dG[e] G[e], G the forward pass's output on A's full pattern P.
 * dG: device float64[nnz of G] in P's CSR order (e.g. grad_g of
 * spai_sai_loss_grad); dW: device float64[W->count] in the blob's layout.
 * The forward pass is recomputed in float64 from the float32 weights and
 * features and its activations kept ((24 (L + 1) + 265) nnz doubles of
 * scratch); every sum is taken in a fixed order.  W->block 3: the GNN on
 * the node graph of A's dense 3 x 3 blocks, as spai_gnn_precond.  Errors as
 * spai_gnn_precond, SPAI_ERR_OOM. */
int spai_gnn_grad(const spai_csr* A, const spai_pattern* P, const float* node_feat,
                  const spai_gnn_weights* W, const double* dG, double* dW, void* stream);

/* One AdamW step for training the GNN's weights (Sec. 4.1 trains with AdamW
 * and an exponentially decaying learning rate; decoupled weight decay as in
 * Loshchilov & Hutter): with g = grad (scaled to 2-norm max_grad_norm first
 * when it is larger and max_grad_norm > 0),
 *   m = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2,
 *   master -= lr (m / (1 - beta1^step) / (sqrt(v / (1 - beta2^step)) + eps)
 *                 + weight_decay master),
 * and blob = (float) master.  master, m, v, grad: device float64[count]
 * (m and v start at zero, step counts from 1); blob: device float32[count]
 * (the spai_gnn_weights blob).  *grad_norm (host, may be NULL) receives the
 * gradient's 2-norm before clipping; then the call synchronises `stream`.
 * SPAI_ERR_INVALID for a null pointer, count or step < 1 or a parameter out
 * of range. */
typedef struct {
  double lr;             /* learning rate of this step */
  double beta1, beta2;   /* moment decay rates (0.9, 0.999) */
  double eps;            /* denominator guard (1e-8) */
  double weight_decay;   /* decoupled decay rate (0.01) */
  double max_grad_norm;  /* > 0: clip the gradient's 2-norm to this; <= 0: no clipping */
} spai_adamw_cfg;

int spai_adamw_step(double* master, double* m, double* v, const double* grad, float* blob, int64_t count,
                    const spai_adamw_cfg* cfg, int64_t step, double* grad_norm, void* stream);

/* Preconditioner from caller-supplied values of G on P (device array of
 * nnz_g values of type val_dtype, F64 or F32, in P's CSR order), stored in
 * g_dtype.  Used for classical factors (FSAI, Jacobi, identity). */
int spai_precond_from_values(const spai_pattern* P, const void* g_val, int32_t val_dtype,
                             int32_t g_dtype, double eps, spai_precond** out, void* stream);

/* Copies the stored G and G^T values, converted to `dtype` (F64 or F32), to
 * caller device buffers of nnz_g entries (either may be NULL). */
int spai_precond_export(const spai_precond* M, void* g_val, void* gt_val, int32_t dtype, void* stream);

/* ||A|| = mean |A_ij| as computed inside gnn_precond (Sec. 3.3). */
int spai_precond_matrix_norm(const spai_precond* M, double* norm);

void spai_precond_destroy(spai_precond* M);

/* ------------------------------------------------------------------------ *
 * Systems: A prepared for repeated solves (validated, float32 copy, SpMV
 * schedule).  The schedule of the persistent solver's three sparse passes
 * (A, G^T, G; the paper runs library SpMVs and has no counterpart) is:
 *   tile_nnz    entries per row group (rows binned by their first entry),
 *   items_log2  groups per work item = heuristic count * 2^items_log2,
 *   staged      1: groups staged into shared memory by TMA bulk copies
 *               (rows of at most 1024 entries), 0: direct loads,
 *   sell        1: matrices with a SELL-32 copy (slices of 32 rows stored
 *               column-major; built when rows have at most 64 entries and
 *               padding adds at most 25%) are read in that layout, one row
 *               per lane; 0: CSR row groups.  The group size of the SELL
 *               layout scales with tile_nnz.
 *   block       1: a matrix made of dense 3 x 3 blocks (A, and G on its
 *               pattern) is read in the 3 x 3 block layout: slices of 32 block
 *               rows, one column index per block and its 9 values, a lane
 *               per block row (three scalar rows); 0: scalar layouts.
 *   fuse        1: the G^T and G passes of an iteration run in one grid-wide
 *               step, a G work item starting once the G^T items whose rows
 *               it reaches have finished (per-item flags instead of a
 *               grid-wide barrier); 0: one grid-wide step per pass.  The
 *               arithmetic is the same either way.
 *   pair        1: the iteration vectors read at the same column in one pass
 *               are stored as interleaved pairs (s with the search direction
 *               d, read together by the A pass; q = A p with r, read together
 *               by the G^T pass), so each such gather is one 8-byte (float32)
 *               or 16-byte (float64) load instead of two loads at different
 *               addresses; 0: separate vectors.  Default 1 for systems whose
 *               rows were sorted by length (irregular gathers, where every
 *               load is a separate L2 request), else 0.  The arithmetic is
 *               the same either way.
 * Per-row sums are the same in every schedule (entries in stored order);
 * dot products are summed in a schedule-dependent fixed order.
 * The default is the heuristic schedule (sell 1).  `autotune` nonzero makes
 * the first solve of the system (spai_system_solve or spai_pcg_solve_batched)
 * time short runs of every candidate (tile_nnz T0, T0/2, T0/4; items_log2
 * -1, 0, 1; SELL, CSR staged, CSR direct; the heuristic schedule also with
 * fuse 0) with that solve's preconditioner
 * and precision and keep the fastest; it is then fixed, so a system's
 * results are the same alone and in any batch.
 * ------------------------------------------------------------------------ */
int spai_system_create(const spai_csr* A, int32_t autotune, spai_system** out, void* stream);

typedef struct {
  int32_t tile_nnz;    /* entries per row group (CSR) ; 0 in set: the default */
  int32_t items_log2;  /* -4..4 */
  int32_t staged;      /* 0 or 1 */
  int32_t sell;        /* 1: SELL-32 layout for the matrices that have one, 0: CSR row groups */
  int32_t fuse;        /* 1: G^T and G passes in one grid-wide step (default), 0: separate steps */
  int32_t block;       /* 1: the 3 x 3 block layout for A, G and G^T when they are made of dense 3 x 3
                          blocks (default), 0: scalar layouts */
  int32_t pair;        /* 1: paired vectors (default for rows sorted by length), 0: separate vectors */
  int32_t tuned;       /* out: 1 once the autotuner ran or a schedule was set */
} spai_schedule;

/* The system's schedule. */
int spai_system_schedule(const spai_system* S, spai_schedule* out);

/* Fixes the schedule (no autotuning afterwards).  SPAI_ERR_INVALID for a
 * field out of range (tile_nnz above the largest group that fits the
 * staging buffer for this matrix, items_log2 outside -4..4, flags not 0/1).
 * Takes effect for solves started afterwards; a request already submitted to
 * a server keeps the vector layout (`pair`) it was submitted with.  Not to be
 * called while a solve of the system runs on another thread. */
int spai_system_set_schedule(spai_system* S, const spai_schedule* sch);

/* Layout facts of a system (for callers and tests): sizes, the longest row,
 * the SELL-32 copy of A -- slices (0: none, CSR only), stored entries with
 * padding, and whether its rows are ordered by length within windows of
 * 1024 rows (SELL-C-sigma, chosen when rows in their own order would pad
 * more than a quarter) -- and the 3 x 3 block copy (slices of 32 block rows;
 * 0 when A is not made of dense 3 x 3 blocks; stored blocks with padding). */
typedef struct {
  int64_t n, nnz;
  int32_t max_row;
  int32_t sell_slices;
  int64_t sell_total;
  int32_t sell_sorted;
  int32_t block_slices;
  int64_t block_total;
} spai_system_layout;

int spai_system_info(const spai_system* S, spai_system_layout* out);

void spai_system_destroy(spai_system* S);

/* ------------------------------------------------------------------------ *
 * pcg_solve - Algorithm 1 (App. A) with M^-1 = G G^T + eps I (Eq. 1).
 * b and x are device float64 arrays of n entries; x holds x0 on entry and the
 * solution on exit.  With precision MIXED the PCG iterations run in float32
 * (A, G, vectors) with float64 dot products; x is kept in float64 and the
 * float32 residual is periodically replaced by the float64 true residual
 * b - A x (iterative refinement without restarting the Krylov recurrence),
 * so the float64 rtol is reached.  On SPAI_ERR_NOT_CONVERGED or
 * SPAI_ERR_BREAKDOWN x holds the last iterate and `res` is filled.
 * ------------------------------------------------------------------------ */
int spai_pcg_solve(const spai_csr* A, const spai_precond* M, const double* b, double* x,
                   const spai_pcg_opts* opts, spai_pcg_result* res, void* stream);

int spai_system_solve(spai_system* S, const spai_precond* M, const double* b, double* x,
                      const spai_pcg_opts* opts, spai_pcg_result* res, void* stream);

/* Many uneven systems solved together (the batching form; the paper solves
 * one system at a time): systems advance in lockstep in a persistent kernel,
 * each with its own scalars, and leave the work list when they converge.  The
 * whole solve is one CUDA graph launch -- a device-side while loop over
 * persistent launches -- so no host round trip happens until every system is
 * done.  Arrays have nsys entries; res[i] is filled for every system; the
 * return value is SPAI_OK if every system converged, else the first failing
 * status.  One system's failure does not stop the others.  All systems use
 * the same opts (history recording is ignored) and the same G storage type. */
int spai_pcg_solve_batched(int32_t nsys, spai_system* const* S, const spai_precond* const* M,
                           const double* const* b, double* const* x, const spai_pcg_opts* opts,
                           spai_pcg_result* res, void* stream);

/* Same as spai_pcg_solve but b and x are HOST float64 arrays; the copies to
 * and from the device are part of the call. */
int spai_pcg_solve_host(const spai_csr* A, const spai_precond* M, const double* b_host,
                        double* x_host, const spai_pcg_opts* opts, spai_pcg_result* res, void* stream);

/* ------------------------------------------------------------------------ *
 * pcg_solve_noalloc - float64 PCG that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc while they solve, for example code that runs under
 * its own device-memory manager or a fixed memory budget where a library
 * allocation would fail or fragment the pool.  A, G and G^T are raw device
 * CSRs (float64, the conventions above; G^T must be the explicit transpose
 * of G, e.g. from spai_pattern_export / spai_precond_export), b and x are
 * device float64 arrays of n entries (x holds x0 on entry), and
 * M^-1 = G G^T + eps I.  opts->precision must be SPAI_PREC_F64.
 * All working memory (vectors, schedules, reductions) lives in one static
 * device array of 8 MiB that every GPU loading the library holds until the
 * process exits; it limits n to 131072 rows and each matrix to 4194304
 * stored entries (larger inputs return SPAI_ERR_TOO_LARGE, and so does any
 * input whose working set exceeds the array).  The first call on a device
 * looks up the array's device address and keeps it for the rest of the
 * process; make that first call before any stream capture, and do not use
 * this entry point after cudaDeviceReset (the kept address would be stale).
 * Every call validates the CSRs and steps the solver with small
 * device-to-host reads, so it synchronises `stream` before it returns.
 * Every call shares the array and reuses it from the previous call: calls
 * that overlap on the GPU (other streams or threads) race, so the caller
 * must serialise them.  res->engine_ms is not measured (0) since timing
 * events are not created.
 * ------------------------------------------------------------------------ */
int spai_pcg_solve_noalloc(const spai_csr* A, const spai_csr* G, const spai_csr* GT, double eps, const double* b,
                           double* x, const spai_pcg_opts* opts, spai_pcg_result* res, void* stream);

/* ------------------------------------------------------------------------ *
 * serve - continuous batching of solve requests on device-resident systems.
 * Requests (b, x on the host) are queued by submit(), which never blocks;
 * a worker thread admits them into free slots while the HBM footprint stays
 * under hbm_cap_bytes, runs all admitted solves together in persistent
 * launches of `chunk_iters` iterations, retires each system in the iteration
 * it converges and admits waiting requests as slots free up.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t hbm_cap_bytes;   /* cap on the device bytes of admitted requests */
  int32_t max_slots;       /* concurrent requests at most */
  int32_t chunk_iters;     /* iterations per persistent launch between admissions (<= 0: 16) */
  spai_pcg_opts opts;      /* solver options for every request (history ignored) */
} spai_serve_cfg;

typedef struct {
  uint64_t ticket;
  int32_t status;
  int64_t iters;
  int32_t outer_iters;
  double true_rel_res;
  double t_submit_us, t_admit_us, t_done_us;  /* host microseconds since server start */
} spai_completion;

int spai_server_create(const spai_serve_cfg* cfg, spai_server** out);

/* Registers a system with its preconditioner; the server keeps references,
 * so S and M must outlive the server. */
int spai_server_register(spai_server* srv, spai_system* S, const spai_precond* M, int64_t* sys_id);

/* Queues a request: b_host (n doubles) is read and x_host (n doubles) written
 * before the request's completion is reported.  x starts from zero. */
int spai_server_submit(spai_server* srv, int64_t sys_id, const double* b_host, double* x_host,
                       uint64_t* ticket);

/* Copies up to `max` finished requests into `out`; *count receives how many. */
int spai_server_poll(spai_server* srv, spai_completion* out, int32_t max, int32_t* count);

/* Waits up to timeout_ms for the request; SPAI_ERR_TIMEOUT if it did not finish. */
int spai_server_wait(spai_server* srv, uint64_t ticket, int64_t timeout_ms, spai_completion* out);

/* Stops the worker after the admitted requests finish and frees everything. */
int spai_server_destroy(spai_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* SPAI_H */
