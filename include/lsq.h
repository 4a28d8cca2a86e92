/*
 * lsq.h -- C ABI of the GB300 (sm_103a) sparse-sign sketch-and-precondition
 * least-squares library (arXiv 2506.03070).
 *
 * Solves min_x ||b - A x|| for dense, tall A (m x n, m >> n) by Algorithm 1:
 * a sparse sign sketch Y = S [A | b] generated and applied in one pass
 * (Sec. 2.1 definition, Sec. 3.1.2 rejection sampling), a Householder QR of
 * the sketch giving the preconditioner M = R^{-1} and the sketch-and-solve
 * start x0 (Algorithm 1, Sec. 3.2), then preconditioned LSQR (Algorithm 2)
 * in the one-synchronisation arrangement of App. D.5.1.
 *
 * General conventions
 *  - Every call returns an lsq_status: 0 = LSQ_OK, 1 = LSQ_PENDING, < 0 error.
 *    No C++ exception crosses this interface.  lsq_last_error(ctx) gives a
 *    human-readable message for the last error on that context.
 *  - Matrices are row-major with an explicit leading dimension (elements).
 *  - Pointers named "device" must be device memory of the context's GPU,
 *    owned by the caller and valid until the call returns.  Nothing the
 *    caller passes is freed or retained by the library.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered; every call below returns only after its work on
 *    `stream` has completed (it synchronises that stream), so results and
 *    status are final on return.
 *  - Workspace (sketch, R, M, LSQR vectors) is owned by the context and
 *    counted against its HBM budget.  One context must not be used by two
 *    host threads at once.
 *  - There is no CPU fallback: without a usable sm_103a GPU, lsq_create
 *    fails with LSQ_ERR_CUDA.
 */
#ifndef LSQ_H
#define LSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lsq_status;
#define LSQ_OK 0
#define LSQ_PENDING 1
#define LSQ_ERR_ARG (-1)         /* invalid argument (sizes, null pointer, zeta > d, ...) */
#define LSQ_ERR_CUDA (-2)        /* a CUDA runtime call failed; see lsq_last_error */
#define LSQ_ERR_OOM (-3)         /* device allocation failed */
#define LSQ_ERR_BUDGET (-4)      /* workspace would exceed the context's HBM budget */
#define LSQ_ERR_SKETCH (-5)      /* rejection sampling exceeded its round cap */
#define LSQ_ERR_RANK (-6)        /* R has a zero (or negligible) diagonal entry */
#define LSQ_ERR_NOCONV (-7)      /* LSQR hit maxit; x still holds the last iterate */
#define LSQ_ERR_TIMEOUT (-8)     /* a device-side wait gave up; the context stays usable */
#define LSQ_ERR_NONFINITE (-9)   /* A or b holds NaN or Inf */
#define LSQ_ERR_UNSUPPORTED (-10) /* shape/precision combination not built */
#define LSQ_ERR_ACCURACY (-11)   /* the final accuracy pass's backward-error bound exceeds the
                                    gate (lsq_opts.gate); x still holds the solution */

/* Arithmetic of the sketch and of the QR.  In both forms A, b and x stay FP64
 * in memory, the LSQR recurrences (Givens scalars, x, w, v) are FP64, and the
 * final accuracy pass (r = b - A x, A^T r, backward errors) runs in native
 * FP64.  The LSQR passes over A form A v and A^T u in double-float arithmetic
 * on the FP32/integer pipes (each FP64 entry split exactly into two floats
 * holding its top 47 significant bits, products exact, sums as float pairs:
 * relative matvec error about 1e-14 against 1e-16 in FP64), unless
 * LSQ_FLAG_NATIVE_FP64 asks for the FP64 pipe (any n <= 4096; about 2.5x the
 * time at n = 2000, the pass bound by GB300's FP64 rate).  The
 * pair image is taken of A 2^-s, b 2^-t with exact power-of-two shifts s, t
 * chosen from the largest entries, so any finite FP64 data is in range; only
 * entries below 2^-103 of the largest entry of A (or b) are flushed. */
typedef enum {
  LSQ_PREC_FP64 = 0,  /* sketch accumulated and factored in FP64 */
  LSQ_PREC_MIXED = 1  /* every sketch term added in FP32, one chunk of rows at a time (about
                         16 terms per entry per chunk), the chunk sums combined in FP64;
                         lsq_solve factors that sketch in FP64 (tensor-core trailing updates
                         with FP32 accumulation, as the plain form), lsq_precond with FP32 Y
                         factors in FP32.  The solve's ||A||_F (info->anorm_fro, the
                         backward-error bounds' scale) is then summed from the FP32 values
                         of A's entries: relative error about 1e-7 */
} lsq_prec;

typedef enum { LSQ_MEM_DEVICE = 0, LSQ_MEM_HOST = 1 } lsq_mem;

typedef struct lsq_ctx lsq_ctx;

/* One least-squares problem. A: m x n row-major (lda >= n), b: m. With
 * mem = LSQ_MEM_HOST, A, b and the solution x live in host memory and the
 * library moves them to and from the device inside the call: when A and b are
 * pinned or registered (page-locked) and prec = LSQ_PREC_FP64, the sketch
 * pass reads them in place over the host link and writes the device copy in
 * the same pass; otherwise they are copied to the device before the sketch. */
typedef struct {
  const double* A;
  const double* b;
  int64_t m, n, lda;
  int32_t mem; /* lsq_mem */
  int32_t reserved;
} lsq_problem;

/* Solver options (Algorithm 1 parameters d, zeta; Algorithm 2 tolerance). */
typedef struct {
  int64_t d;      /* embedding dimension, n+1 <= d <= 2^31-1; 0 = chosen by lsq_choose_d (lsq_solve) */
  int32_t zeta;   /* nonzeros per sketch column, 1 <= zeta <= min(d, 64) */
  int32_t prec;   /* lsq_prec */
  uint64_t seed;  /* sketch seed (Philox key) */
  double tol;     /* LSQR stopping tolerance (normal-equation test) */
  int64_t maxit;  /* LSQR iteration cap; <= 0 selects 10*ceil(log(tol)/log(sqrt(n/d))) */
  int32_t flags;  /* LSQ_FLAG_* */
  int32_t reserved;
  double gate;    /* accuracy gate: the solve returns LSQ_ERR_ACCURACY when the final accuracy
                     pass finds min(backward_error_ne, backward_error_pre) above it.  0 selects
                     max(1e-10, tol); < 0 disables the gate.  Both bounds are computed in
                     FP64 from r = b - A x (see lsq_info); backward_error_ne is Stewart's
                     rigorous bound, backward_error_pre bounds the Karlson-Walden estimate
                     up to the sketch's distortion.  Not applied with LSQ_FLAG_NO_CHECK. */
} lsq_opts;

#define LSQ_FLAG_TIMING 1      /* record per-phase device times in lsq_info */
#define LSQ_FLAG_NO_CHECK 2    /* skip the final accuracy pass (backward errors not filled) */
#define LSQ_FLAG_NATIVE_FP64 4 /* run the LSQR matvecs on the native FP64 pipe */
#define LSQ_FLAG_NO_IMAGE 8    /* do not keep the 8 B/entry float-pair image of A (saves
                                  m*n*8 bytes of workspace; each pass splits A itself) */
#define LSQ_FLAG_NO_FALLBACK 16 /* mixed form: report LSQ_ERR_NOCONV instead of re-solving
                                   in FP64 when the FP32 preconditioner stalls LSQR */
#define LSQ_FLAG_HBM 64         /* lsq_solve: heavy-ball momentum (Algorithm 6) instead of
                                   LSQR, with eta_hat = sqrt(n/d) (see lsq_hbm) */

typedef struct {
  int32_t status;          /* status of the solve (same as the return value) */
  int32_t stop;            /* 1 normal-equation test, 2 residual test, 3 maxit, 4 breakdown */
  int64_t iters;           /* LSQR iterations */
  double normal_rel_est;   /* LSQR's last ||(AM)^T r|| / (||AM|| ||r||) estimate */
  double backward_error_ne;  /* ||A^T r|| / (||A||_F ||r||), r = b - A x (Stewart's bound) */
  double backward_error_pre; /* ||M^T A^T r|| / (||A||_F ||x||): preconditioned bound */
  double rnorm, arnorm, anorm_fro, xnorm, bnorm;
  int32_t sketch_rounds_max; /* most rejection-sampling redraw rounds any column used */
  int32_t precond_fallback;  /* 1: the mixed form's preconditioner stalled LSQR and the
                                plain form solved the problem again */
  float t_sketch_ms, t_precond_ms, t_lsqr_ms, t_check_ms, t_h2d_ms, t_d2h_ms;
  /* t_lsqr_ms (LSQ_FLAG_TIMING): LSQR and the accuracy pass (one kernel);
   * t_check_ms (always when the pass ran): the accuracy pass alone, from the
   * device clock (%globaltimer) */
  /* lsq_submit / lsq_poll only: host monotonic clock (CLOCK_MONOTONIC) in
   * seconds when the request was submitted, handed to the device, and seen
   * complete; the number of blocks that solved it together and how long its
   * first block waited for the rest of the group (device clock).  For served
   * requests t_sketch_ms, t_precond_ms and t_lsqr_ms (LSQR + accuracy pass)
   * are device-clock durations of the phases. */
  double t_submit_s, t_start_s, t_done_s;
  int32_t group_blocks;
  float t_group_wait_ms;
  int64_t d_used; /* lsq_solve: the embedding dimension used (the chosen one when opts->d == 0) */
} lsq_info;

/* Context on `device` with a workspace budget of hbm_budget_bytes (0 = 90% of
 * the device's free memory at creation).  Device-side waits (grid barriers,
 * bulk-copy completions) of the context's synchronous calls give up after
 * 20 s (LSQ_ERR_TIMEOUT) unless lsq_set_wait_limit sets another limit. */
lsq_status lsq_create(lsq_ctx** out, int device, size_t hbm_budget_bytes);
lsq_status lsq_destroy(lsq_ctx* ctx);
const char* lsq_last_error(const lsq_ctx* ctx);
const char* lsq_status_string(lsq_status s);
/* Bytes of workspace the context holds right now. */
size_t lsq_workspace_bytes(const lsq_ctx* ctx);

/* Sketch indices and signs (test/debug export).  Sec. 3.1.2 steps (i)-(iv)
 * and the signs of Algorithm 3: for columns row0 .. row0+rows-1 of S, the
 * zeta distinct row indices in [0, d), ascending, and their signs (+1/-1; the
 * value is sign/sqrt(zeta)).  The random words come from Philox4x64-10 keyed
 * (seed, 0): index draw (column i, round r, slot j) = counter (i, r, j/4, 0),
 * word j%4, mapped to floor(word*d / 2^64); signs = counter (i, 0, 0, 1),
 * bit k of word 0.  Same device code as lsq_sketch.
 * idx: device int32 [rows x zeta]; sign: device int8 [rows x zeta];
 * rounds: device int32 [rows] or NULL (redraw rounds per column). */
lsq_status lsq_sketch_indices(lsq_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t d, int32_t zeta,
                              int32_t* idx, int8_t* sign, int32_t* rounds, void* stream);

/* Y = S [A | b]  (Algorithm 1 "Form Y = SA"; S never stored).
 * A: device, m x n (lda >= n); b: device m or NULL.
 * Y: device, d x ldy row-major, ldy >= n + (b != NULL); FP64 (prec FP64) or
 * FP32 (prec MIXED: FP32 accumulation in row chunks whose sums are combined in
 * FP64 workspace of d (n + 1) doubles plus d (n + 4) floats, then rounded once
 * to FP32).  Y is overwritten.  Errors: LSQ_ERR_ARG, LSQ_ERR_SKETCH, LSQ_ERR_NONFINITE
 * (A or b not finite). */
lsq_status lsq_sketch(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                      int32_t zeta, uint64_t seed, int32_t prec, void* Y, int64_t ldy, void* stream);

/* Preconditioner from a sketch (Algorithm 1 "QR(Y)", "M = R^{-1}" and
 * "x0 = M Q^T S b"; Sec. 3.2 explicit inverse).  Householder QR of the
 * d x ncol matrix Y (ncol = n + has_b, FP64 or FP32 per prec, ld ldy).
 * Outputs (device, row-major n x n, ld n): R (upper triangular, may be NULL),
 * M = R^{-1} (upper triangular, required); x0 (device n, NULL allowed; only
 * with has_b) = M z, z = first n entries of Q^T (S b).
 * Errors: LSQ_ERR_ARG (d < ncol), LSQ_ERR_RANK (|R_jj| <= n * eps * max|R_ii|). */
lsq_status lsq_precond(lsq_ctx* ctx, const void* Y, int64_t d, int64_t n, int64_t ldy, int32_t has_b, int32_t prec,
                       double* R, double* M, double* x0, void* stream);

/* Which Householder QR lsq_precond and lsq_solve use.  AUTO (the default):
 * the blocked factorisation (compact WY: 64-column panels factored by a
 * cooperative kernel; the Gram matrix and the trailing updates as the
 * library's own tcgen05 tensor-core GEMMs on exact bf16 slices -- 7 slices
 * per row keep FP64 accuracy, 4 keep FP32 accuracy for the mixed form) once
 * the d x (n+1) working copy reaches 32 MiB in its precision, the unblocked one
 * (one grid barrier per column) below.  Both compute the same reflectors. */
/* ---- Embedding dimension (Sec. 4.3 "Selecting the embedding dimension") ----
 * The solve time is modelled as T(d) = T_qr(d) + (t(d) + 2) T_iter(m): the
 * preconditioner grows linearly in d, and the Sec. 4.3 rate estimate
 * (n/d)^{t/2} <= tol gives t(d) = 2 |ln tol| / ln(d/n) LSQR iterations, each
 * linear in m.  Its minimum has a closed form through the Lambert W function
 * (the paper balances the two costs the same way with unit constants):
 * d = n exp(2 W0(sqrt(C)/2)), C = 2 |ln tol| t_iter_per_row m / (t_qr_per_d n).
 * lsq_choose_d measures t_iter_per_row (one LSQR iteration per row of A) and
 * t_qr_per_d (preconditioner time per extra sketch row) on this GPU with
 * synthetic data of width n, once per n and context (tens of ms; not while
 * requests are being served), then clamps d to [max(n+1, 1.25 n), min(m,
 * what fits in an eighth of the budget)].  lsq_solve with opts->d == 0 uses it
 * and reports the choice in info->d_used. */
lsq_status lsq_choose_d(lsq_ctx* ctx, int64_t m, int64_t n, double tol, int64_t* d);
/* The model's minimiser for given constants (no clamping; 0 on bad input). */
int64_t lsq_d_from_model(int64_t m, int64_t n, double tol, double t_iter_per_row, double t_qr_per_d);
/* Principal branch W0 of the Lambert W function on [-1/e, inf) (NaN outside). */
double lsq_lambert_w0(double x);

/* Limit of every device-side wait of this context's later synchronous calls
 * and of serving requests staged after the call (0 < seconds <= 4000; 0
 * restores the built-in 20 s).  A wait that runs out raises LSQ_ERR_TIMEOUT:
 * every block of the launch leaves at its next barrier, bulk copies already
 * issued are waited for, and the context stays usable. */
lsq_status lsq_set_wait_limit(lsq_ctx* ctx, double seconds);
/* Self-test of that mechanism (no counterpart in the paper): kind 0 launches
 * a grid barrier of two co-resident blocks that expects three arrivals, kind 1
 * an mbarrier phase that nothing completes; both must give up after the wait
 * limit.  Returns LSQ_ERR_TIMEOUT when the wait gave up as designed. */
lsq_status lsq_selftest_wait(lsq_ctx* ctx, int32_t kind, void* stream);

#define LSQ_QR_AUTO 0
#define LSQ_QR_UNBLOCKED 1
#define LSQ_QR_BLOCKED 2
lsq_status lsq_set_qr_mode(lsq_ctx* ctx, int32_t mode);

/* Preconditioned LSQR (Algorithm 2) from x0 with preconditioner M (device,
 * n x n row-major upper triangular), in the one-synchronisation order of
 * App. D.5.1.  A, b, x0, x device.  x receives the final iterate.  Stops when
 * ||(AM)^T r|| <= tol ||AM||_est ||r|| (Paige-Saunders test 2 on the
 * preconditioned problem), ||r|| <= tol ||b||, or at maxit (LSQ_ERR_NOCONV).
 * info may be NULL.  Limits: n <= 4096 (LSQ_ERR_UNSUPPORTED beyond), with
 * or without LSQ_FLAG_NATIVE_FP64.  The same limits hold for lsq_solve and
 * lsq_check. */
lsq_status lsq_lsqr(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                    const double* M, const double* x0, double tol, int64_t maxit, int32_t flags, double* x,
                    lsq_info* info, void* stream);

/* Gradient descent with heavy-ball momentum (Algorithm 6, App. C.2) from x0
 * with preconditioner M: x_t = x_{t-1} + alpha M M^T A^T (b - A x_{t-1})
 * + beta (x_{t-1} - x_{t-2}), alpha = (1 - eta_hat^2)^2, beta = eta_hat^2 --
 * the optimal parameters when the singular values of A M lie in
 * [1/(1+eta_hat), 1/(1-eta_hat)], as a sketch with distortion eta_hat leaves
 * them (0 <= eta_hat < 1; sqrt(n/d) estimates it).  One pass over A per
 * iteration (r, A^T r and ||r|| fused, double-float arithmetic as in lsq_lsqr).
 * Stops before an update when ||M^T A^T r|| <= tol ||b|| (which bounds
 * ||A (x - x_*)|| by tol ||b|| / sigma_min(AM), the accuracy target of the
 * paper's Sec. 4.3 experiments), ||r|| <= tol ||b||, or after maxit updates
 * (LSQ_ERR_NOCONV).  Same limits and flags as lsq_lsqr; with a poor eta_hat it
 * converges slowly or diverges, where LSQR needs no parameter. */
lsq_status lsq_hbm(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                   const double* M, const double* x0, double tol, int64_t maxit, double eta_hat, int32_t flags,
                   double* x, lsq_info* info, void* stream);

/* Accuracy of a candidate solution: one pass over A computing r = b - A x,
 * A^T r, ||A||_F and the two backward-error bounds of lsq_info (M may be NULL;
 * then backward_error_pre is 0), all in native FP64 (one warp per row for
 * n <= 512, PW warps sharing a row in column panels above).  All device
 * pointers.  No gate: the bounds are reported, not judged. */
lsq_status lsq_check(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                     const double* x, const double* M, lsq_info* info, void* stream);

/* Allocation-free variant of lsq_check (the paper has no counterpart; this is
 * an interface convenience).  For callers that may not allocate device memory
 * -- code running under another allocator that owns the GPU's memory, or with
 * a memory plan fixed at start-up -- and so cannot create an lsq_ctx: it takes
 * no context and calls no allocator.  Its scratch is one static device array
 * of about 4.1 MB that every GPU loading the library keeps until the process
 * exits.  Limits: n <= 512 (otherwise LSQ_ERR_ARG, nothing launched); a
 * device whose co-resident grid for the pass would exceed the array's 512
 * per-block rows returns LSQ_ERR_UNSUPPORTED.  The first call on a device
 * (and driver context) looks up that array's device address (with the device
 * current); make that first call before any stream capture.  All calls
 * on a device share the array: calls whose GPU work overlaps (other streams,
 * other host threads) race and must be serialised by the caller.  Runs on the
 * current device and `stream`, synchronises `stream`, fills the accuracy
 * fields of info (rnorm, arnorm, anorm_fro, xnorm, bnorm, backward_error_ne,
 * backward_error_pre); same inputs and meaning as lsq_check. */
lsq_status lsq_check_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* x,
                             const double* M, lsq_info* info, void* stream);

/* Algorithm 1 end to end: sketch, precondition, LSQR, accuracy pass.
 * x: n doubles, device memory for LSQ_MEM_DEVICE problems, host memory for
 * LSQ_MEM_HOST problems.  info may be NULL.
 * prec = LSQ_PREC_MIXED adds every sketch term in FP32 (4-wide vector
 * reductions, a third of the FP64 reduction cost per term) in row chunks whose
 * sums are combined in FP64, then factors the sketch as the plain form does:
 * the relative error of the sketch stays near FP32's unit roundoff times the
 * square root of the terms per chunk, which keeps the preconditioner's
 * quality while cond(A) * 1e-7 stays well below one.  The mixed LSQR is capped at
 * twice the iterations the Sec. 4.3 rate estimate predicts
 * (2 ceil(log(tol)/log(sqrt(n/d))) + 5); if it stalls, fails the accuracy
 * gate, or max|A| or max|b| lies outside [2^-60, 2^101) (the FP32 sketch's
 * safe range), the problem is solved again in the plain form
 * (info->precond_fallback = 1) unless LSQ_FLAG_NO_FALLBACK is set. */
lsq_status lsq_solve(lsq_ctx* ctx, const lsq_problem* problem, const lsq_opts* opts, double* x, lsq_info* info,
                     void* stream);

/* ---- Sparse A (CSR) --------------------------------------------------------
 * Algorithm 1 for A given by its nonzeros (the paper's sparse workloads): the
 * sketch touches only the nonzeros (O(zeta nnz); the sketch columns are the
 * dense path's, so S is the same), Householder QR and M = R^{-1} as for dense
 * A, then LSQR (or heavy-ball momentum with LSQ_FLAG_HBM) whose passes run over
 * the nonzeros in FP64.  row_ptr: m+1 int64 offsets (row_ptr[0] = 0,
 * nondecreasing, row_ptr[m] = nnz); col_idx: nnz int32 in [0, n) (any order
 * within a row, duplicates add); values: nnz doubles; b: m doubles; x: n
 * doubles.  All device memory.  opts as for lsq_solve (FP64 form only; d = 0
 * chooses d with the dense model); lsq_info as for lsq_solve.  The structure
 * is checked on the device before any kernel indexes by it (one extra stream
 * synchronisation): malformed offsets or indices give LSQ_ERR_ARG. */
typedef struct {
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* values;
  const double* b;
  int64_t m, n, nnz;
} lsq_csr_problem;

lsq_status lsq_solve_csr(lsq_ctx* ctx, const lsq_csr_problem* problem, const lsq_opts* opts, double* x, lsq_info* info,
                         void* stream);

/* ---- Batched solves -------------------------------------------------------
 * Many independent problems in one persistent launch: every block takes whole
 * problems from a device work counter (largest m*n first) and runs all of
 * Algorithm 1 for each by itself (sketch, Householder QR, M, x0, LSQR with
 * block barriers).  A, b and x of every item are device pointers; x receives
 * the solution.  Limits per item: 1 <= n <= 256, n+1 <= d, 1 <= zeta <= 8
 * (larger problems belong to lsq_solve, which uses the whole GPU).
 * The LSQR pass shape (lsq_batch_shape_set below) is picked per n-range by
 * the context's autotuner (LSQ_FLAG_AUTOTUNE times the candidate shapes on the
 * largest problems of the batch the first time an n-range is seen, and keeps
 * the fastest).  results may be NULL. */
typedef struct {
  const double* A;
  const double* b;
  double* x;
  int64_t m, n, lda;
  int64_t d;
  int32_t zeta;
  int32_t reserved;
  uint64_t seed;
} lsq_batch_item;

typedef struct {
  int32_t status; /* per-problem lsq_status */
  int32_t stop;
  int64_t iters;
  double backward_error_ne, rnorm, anorm_fro, xnorm, bnorm;
} lsq_batch_result;

#define LSQ_FLAG_AUTOTUNE 32 /* lsq_solve_batch: tune the LSQR pass shape for new n-ranges */

lsq_status lsq_solve_batch(lsq_ctx* ctx, const lsq_batch_item* items, int64_t count, double tol, int64_t maxit,
                           int32_t flags, lsq_batch_result* results, void* stream);

/* Pass shape of an n-range of batched and served problems: bucket 0 (n <= 32),
 * 1 (n <= 64), 2 (n <= 128), 3 (n <= 256).  Shape s gives each row L lanes with
 * P column pairs a lane, a warp taking 32/L rows a step: (L, P) = (8,2), (8,4),
 * (16,2), (16,4), (32,2), (32,4) for s = 0..5 (it takes n <= 2 L P).
 * lsq_batch_shape_set pins the shape of a bucket (the value LSQ_FLAG_AUTOTUNE
 * stores after timing the candidates; -1 clears it, and a bucket without a
 * shape takes its default: 0, 1, 3, 5); a shape that cannot take the bucket's
 * largest n, or a bucket outside 0..3, gives LSQ_ERR_ARG.
 * lsq_batch_shape_get writes the pinned shape (-1: none) to *shape.  Neither
 * call may run concurrently with a solve on the same context. */
lsq_status lsq_batch_shape_set(lsq_ctx* ctx, int32_t bucket, int32_t shape);
lsq_status lsq_batch_shape_get(lsq_ctx* ctx, int32_t bucket, int32_t* shape);

/* ---- Serving: asynchronous solves of problems that arrive over time -----
 * lsq_submit queues a problem and returns at once with a ticket; lsq_poll
 * reports LSQ_PENDING until the solve is complete, then its final status
 * (and fills info), after which the ticket is gone.
 *
 * Behind it runs a persistent request loop: one cooperative kernel keeps
 * every block of the GPU resident and takes requests from a ring in device
 * memory (filled by copy-engine copies from the host; completion records are
 * in mapped host memory) as they arrive.  A request is solved by a group of G blocks
 * (G from the problem's size: 1 for small problems, up to the whole grid for
 * the largest), which claim it in arrival order, so requests that arrive
 * while others are on the GPU start as soon as blocks free up and run beside
 * them.  Each group runs Algorithm 1 end to end (sketch, Householder QR,
 * M = R^{-1}, x0, LSQR, accuracy pass) with barriers over its own blocks.
 * Small problems (n <= 256) use the LSQR pass shape the context's autotuner
 * picked for their n-range (see lsq_solve_batch, LSQ_FLAG_AUTOTUNE).
 * A host thread admits queued requests in arrival order while their device
 * memory (sketch, R, M, LSQR vectors, the float-pair image of A, and A, b, x
 * themselves for host problems) fits in the serving arena: the budget is the
 * admission limit, and A, R and the LSQR state stay on the device for the
 * whole solve.  While requests are in flight the server occupies the GPU:
 * synchronous calls on the same device run after it drains.
 *
 * Limits: FP64 form only, 1 <= n <= 1024, n+1 <= d, 1 <= zeta <= 8.
 * A, b (and x) must stay valid until lsq_poll reports completion; for
 * LSQ_MEM_HOST problems they are host memory (pinned memory copies fastest),
 * A and b are copied in when the request is admitted and x is copied out when
 * it completes.  Returns LSQ_ERR_BUDGET only if the problem alone does not
 * fit the arena.  Several host threads may submit and poll concurrently. */
typedef int64_t lsq_ticket;

/* stream: the request starts only after the work enqueued on `stream` before
 * this call has completed (so inputs still being produced, and buffers that
 * pending work reads or writes, e.g. memory a caching allocator recycles, are
 * safe); NULL is the legacy default stream, as everywhere in this header. */
lsq_status lsq_submit(lsq_ctx* ctx, const lsq_problem* problem, const lsq_opts* opts, double* x, lsq_ticket* out,
                      void* stream);
lsq_status lsq_poll(lsq_ctx* ctx, lsq_ticket ticket, lsq_info* info);

/* Serving configuration; takes effect only before the first lsq_submit.
 * arena_bytes: device memory for admitted requests (0 = the context's budget
 * minus the synchronous workspace it holds); cta_bytes: bytes of A per block
 * when sizing a request's group (0 = 64 MiB); max_group: most blocks one
 * request may take (0 = an eighth of the resident blocks).  A request's group
 * is max(A bytes / cta_bytes, QR flops / 2.5e8), clamped to [1, max_group]. */
lsq_status lsq_serve_config(lsq_ctx* ctx, size_t arena_bytes, double cta_bytes, int32_t max_group);

typedef struct {
  int64_t submitted, completed, pending, in_flight;
  int64_t server_launches;  /* launches of the persistent server kernel */
  int64_t grid_blocks;      /* blocks of one launch */
  size_t arena_bytes, arena_peak_bytes;
} lsq_serve_stats;
lsq_status lsq_serve_stats_get(lsq_ctx* ctx, lsq_serve_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* LSQ_H */
