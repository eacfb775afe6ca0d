/*
 * lsrn.h -- C ABI of the GB300 (sm_103a) LSRN solver.
 *
 * LSRN (Meng, Saunders, Mahoney, "LSRN: A Parallel Iterative Solver for
 * Strongly Over- or Under-Determined Systems") computes the min-length
 * solution x* = argmin ||x||_2 subject to x in argmin_z ||A z - b||_2
 * (section 1, eqs. (ls) and (ls_min_length)) of a dense or sparse A that is
 * strongly over- (m >> n) or under-determined (m << n) and possibly
 * rank-deficient, optionally with Tikhonov regularisation W = lambda I
 * (section 5, eqs. (l2_reg), (l2_reg_eq), (l2_reg_eq_under)).
 *
 * A solve runs the steps of Algorithm 1 (m >= n) or Algorithm 2 (m < n):
 *   lsrn_plan        orientation, s = ceil(gamma * min(m, n)), workspace
 *   lsrn_sketch      steps 2-3: A~ = G A (or A G), G Gaussian, drawn on the fly
 *   lsrn_precond     steps 4-5: SVD of A~, rank r, N = V~ Sigma~^-1 (M = U~ Sigma~^-1)
 *   lsrn_solve_lsqr  step 6-7 with LSQR
 *   lsrn_solve_cs    step 6-7 with the Chebyshev semi-iterative method (Algorithm 3)
 *
 * Conventions (apply to every entry point):
 *   - All functions return an lsrn_status; none throws or aborts.  A negative
 *     status means the call failed; the plan (if any) is left in the state it
 *     had before the call unless stated otherwise.
 *   - Pointers to matrix and vector data may be host or device pointers; the
 *     library asks the CUDA runtime which one it is.  Host data is copied to
 *     the device inside the call (so host inputs may be freed on return); device
 *     data must stay valid and unmodified until the call that uses it returns.
 *   - Arithmetic is FP64 unless an option says otherwise.  All work runs on the
 *     CUDA stream given to lsrn_plan, on the device that was current then; a
 *     call that returns results to the caller synchronises that stream.
 *   - A plan is not thread-safe: calls on one plan must not overlap.  Different
 *     plans are independent.
 *   - The library never falls back to CPU arithmetic: without a usable GPU the
 *     calls return LSRN_ERR_CUDA.
 */
#ifndef LSRN_H
#define LSRN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSRN_OK = 0,
  LSRN_PENDING = 1,             /* lsrn_poll: the request is still running */
  LSRN_ERR_INVALID_ARG = -1,    /* bad size, pointer, option or CSR structure */
  LSRN_ERR_OOM = -2,            /* device allocation failed */
  LSRN_ERR_CUDA = -3,           /* CUDA runtime error or no usable device */
  LSRN_ERR_NOT_CONVERGED = -4,  /* LSQR hit max_iter; x holds the last iterate */
  LSRN_ERR_DIVERGED = -5,       /* CS residual grew: the Theorem 4.5 bounds failed */
  LSRN_ERR_TIMEOUT = -6,        /* a bounded device wait gave up */
  LSRN_ERR_QUEUE_FULL = -7,     /* server: no slot or memory budget for the request */
  LSRN_ERR_STATE = -8,          /* calls out of order (e.g. precond before sketch) */
  LSRN_ERR_UNSUPPORTED = -9,    /* valid request this build does not implement */
  LSRN_ERR_COMM = -10           /* the allgather callback of a sharded plan reported failure */
} lsrn_status;

typedef enum {
  LSRN_DENSE_ROWMAJOR = 0,      /* A[i*ld + j], ld >= n */
  LSRN_DENSE_COLMAJOR = 1,      /* A[i + j*ld], ld >= m */
  LSRN_CSR = 2                  /* row_ptr[m+1] (int64), col_idx[nnz] (int32), values[nnz] */
} lsrn_format;

typedef enum { LSRN_F64 = 0, LSRN_F32 = 1 } lsrn_dtype;

typedef enum {
  LSRN_ITER_F64 = 0,            /* every pass over A in FP64 */
  LSRN_ITER_F32 = 1,            /* m >= n: passes stream an FP32 copy of A (FP32 products); the
                                   sweep stops at max(tol, 1e-6) and double-double refinement
                                   against the FP64 A restores full accuracy.  x = N y stays in
                                   range(N) whatever the pass precision.  For m < n the option
                                   is ignored (FP64 passes): there x is iterated in R^n and
                                   FP32 rounding of A would add components in null(A). */
  LSRN_ITER_F32X2 = 2,          /* dense A whose short side q has 512 < q <= 4096 (other
                                   shapes: FP64 passes): the plan keeps A / 2^e as two FP32
                                   planes hi + lo (48 significant bits, 8 bytes per entry, e
                                   the exponent of max |A_ij|) and every pass runs on the FP32
                                   pipe with error-free products and double-float sums folded
                                   into FP64 every 64 rows (relative error of each product and
                                   sum ~2^-48, against 2^-53 in FP64).  Tall and fat; for
                                   m >= n the sweep stops at max(tol, 1e-8); at least two
                                   refinement steps follow (early stop as usual), with the residual
                                   r = b - Ax and A^T r exact to ~2^-65 (three FP32 planes).
                                   Vectors and row coefficients are rescaled by powers of two
                                   inside the pass, so any finite A, b work. */
  LSRN_ITER_AUTO = 3            /* by size: FP64 passes for CSR A and for dense A of less than
                                   1 GiB in FP64 (8 m n bytes; such A is read largely from L2
                                   and the extra refinement passes of the reduced-precision
                                   modes cost more than the passes save); above that
                                   LSRN_ITER_F32X2 where it applies, else LSRN_ITER_F32 for
                                   m >= n, else FP64.  lsrn_info.iter_used reports the choice. */
} lsrn_iter_mode;

typedef enum {
  LSRN_SKETCH_F64 = 0,          /* FP64 FMA arithmetic */
  LSRN_SKETCH_TC_SLICED = 1,    /* tensor cores on exact bf16 slices of G and A,
                                   FP64-accurate (dense A only) */
  LSRN_SKETCH_BF16 = 2,         /* tensor cores on G and A rounded once to bf16, FP32
                                   accumulation per 2048 rows, FP64 beyond (dense A only): a
                                   subspace embedding with ~2^-8 relative error, enough for a
                                   preconditioner of a well-conditioned full-rank A; the
                                   iterations still use the FP64 A */
  LSRN_SKETCH_AUTO = 3          /* dense A: BF16 first; the exact sliced sketch instead as
                                   soon as the BF16 noise floor eta = 2^-8 ||A~||_F / sqrt(n')
                                   exceeds sigma_min(A~) / 16 (seen on the QR's diagonal or
                                   in the final spectrum: rank-deficient or ill-conditioned A).
                                   A kept BF16 preconditioner widens the Chebyshev bounds by
                                   2 eta / sigma_min.  CSR: the FP64 sketch. */
} lsrn_sketch_mode;

typedef enum {
  LSRN_PRECOND_SVD = 0,         /* N = V~ Sigma~^-1 from the SVD of A~ (Algorithm 1/2 steps 4-5) */
  LSRN_PRECOND_QR = 1           /* lambda > 0 only: N = R^-1 from the QR of A~.  The augmented
                                   matrix has full rank, so A R^-1 = (A V~ Sigma~^-1) U_R^T has
                                   the same singular values as A N (Lemma 4.3 unchanged), the
                                   same Theorem 4.5 bounds and CS step count, and LSQR's
                                   iterates up to the orthogonal change of variable U_R; the
                                   one-sided Jacobi sweeps are not needed.  lsrn_plan_get_precond
                                   then reports |R_ii| (descending) in place of sigma~. */
} lsrn_precond_mode;

typedef enum {
  LSRN_SVD_F64 = 0,             /* one-sided Jacobi sweeps in FP64 on R (default) */
  LSRN_SVD_DF = 1               /* 1024 < n' <= 4096: the early sweeps in double-float arithmetic
                                   (pairs of FP32, ~2^-46) on a copy of R, with the rotations
                                   accumulated into P, then Y = P R in FP64 and FP64 sweeps on Y
                                   until no pair rotates (usually one rotating sweep and one
                                   check).  sigma~(Y) is sigma~(R) up to the relative factor
                                   ||P^T P - I|| (~1e-12), and N = W_r Sigma_r^-2 from Y's sweeps
                                   gives R N = P^-1 J, so Lemma 4.3 holds as for FP64 sweeps.
                                   Other sizes: FP64 sweeps.  Correct but not faster on GB300 as
                                   built: a double-float sweep reads and writes the rows of P as
                                   well as W, and with both held in registers two pairs fit on an
                                   SM, so it is bound by latency (about 57 ms a sweep against
                                   41 ms for an FP64 sweep at n' = 2000). */
} lsrn_svd_mode;

/* The matrix A (m x n).  For LSRN_CSR, columns within a row need not be
 * sorted but must be in [0, n) and row_ptr must be non-decreasing with
 * row_ptr[0] = 0 and row_ptr[m] = nnz. */
typedef struct {
  int64_t m, n;
  int64_t ld;                   /* dense leading dimension in elements */
  int64_t nnz;                  /* CSR stored entries */
  int32_t format;               /* lsrn_format */
  int32_t dtype;                /* lsrn_dtype of values (F32 values are widened to FP64) */
  const void* values;
  const int64_t* row_ptr;
  const int32_t* col_idx;
} lsrn_matrix;

typedef struct {
  double gamma;        /* oversampling factor, > 1; s = ceil(gamma*min(m,n)) (default 2.0) */
  double tol;          /* epsilon: LSQR atol = btol, CS tolerance (default 1e-14) */
  double lambda;       /* Tikhonov lambda >= 0, W = lambda I (default 0) */
  double rcond;        /* rank cut: keep sigma_i > rcond*sigma_1; < 0: max(s, n')*2^-53 */
  double cs_alpha;     /* alpha of Theorem 4.5 used for the CS bounds; < 0: 1/sqrt(s) */
  double refine_tol;   /* relative tolerance of each refinement correction (default 1e-3) */
  int32_t max_iter;    /* LSQR iteration cap; < 0: ceil(1.5 * Theorem 4.6 bound) */
  int32_t refine_max;  /* refinement steps after the iteration (default 1; 0 = paper only);
                          steps stop early once one changes x by <= 1e-12 relative */
  uint64_t seed;       /* key of the counter-based generator of G (default 0) */
  int32_t sketch_mode; /* lsrn_sketch_mode (default LSRN_SKETCH_F64) */
  int32_t iter_mode;   /* lsrn_iter_mode (default LSRN_ITER_F64); LSRN_ITER_F32 keeps an
                          FP32 copy of A (4 bytes per entry) and allows at least six
                          refinement steps, stopping once a step changes x by <= 1e-12;
                          correction passes switch from FP32 to FP64 as soon as a step
                          shrinks the change by less than 20x */
  int32_t precond_mode;  /* lsrn_precond_mode (default LSRN_PRECOND_SVD); LSRN_PRECOND_QR
                            needs lambda > 0 (INVALID_ARG otherwise) */
  int32_t svd_mode;      /* lsrn_svd_mode (default LSRN_SVD_F64) */
} lsrn_options;

typedef struct {
  int64_t m, n, s, rank;          /* problem size, sketch size, numerical rank r */
  int32_t iterations;             /* LSQR iterations / CS steps of the main sweep */
  int32_t refine_steps;           /* refinement steps taken */
  int32_t refine_iterations;      /* inner steps spent in refinement */
  int32_t tall;                   /* 1: Algorithm 1, 0: Algorithm 2 */
  int32_t istop;                  /* LSQR: 1 = rule S1, 2 = rule S2, 3 = exact, 0 = cap/none */
  int32_t status;                 /* lsrn_status of the solve */
  double sigma_max_sketch;        /* sigma_1 of A~ */
  double sigma_min_sketch;        /* sigma_r of A~ */
  double sigma_L, sigma_U;        /* CS bounds used (Theorem 4.5), 0 for LSQR */
  double rnorm_est, arnorm_est;   /* LSQR estimates of ||r||, ||(AN)^T r|| at exit */
  double anorm_est;               /* LSQR estimate of ||AN||_F */
  float t_sketch_ms, t_precond_ms, t_iter_ms, t_refine_ms;  /* device time per phase */
  float t_sketch_gemm_ms;         /* tensor-core GEMM kernels inside the sketch (0 otherwise) */
  float t_pass_ms;                /* fused passes over dense A in the solve, main sweep and
                                     refinement corrections (sum of their device times) */
  int32_t n_pass;                 /* those passes that streamed A: passes launched after the
                                     sweep converged return at once and are not counted
                                     (duration below a quarter of the longest pass) */
  float t_qr_ms;                  /* Householder QR of the sketch inside t_precond_ms */
  int32_t jacobi_sweeps;          /* FP64 one-sided Jacobi sweeps of the preconditioner */
  float t_jacobi_ms;              /* the Jacobi sweeps inside t_precond_ms */
  int32_t sketch_used;            /* lsrn_sketch_mode of the sketch the preconditioner used */
  int32_t sketch_escalated;       /* 1: LSRN_SKETCH_AUTO replaced the BF16 sketch by the exact one */
  int32_t jacobi_sweeps_df;       /* double-float sweeps before the FP64 ones (LSRN_SVD_DF) */
  int32_t iter_used;              /* lsrn_iter_mode the passes ran in (LSRN_ITER_AUTO resolved) */
} lsrn_info;

typedef struct lsrn_plan_s* lsrn_plan_t;
typedef struct lsrn_server_s* lsrn_server_t;

/* Human-readable name of a status code (static storage). */
const char* lsrn_status_string(lsrn_status s);

/* Text describing the last CUDA error seen by this thread inside the library
 * (file, line, call, CUDA message); empty if none.  Static thread-local storage. */
const char* lsrn_last_error_message(void);

/* Number of CUDA kernels the library has launched in this process (a
 * diagnostic for profiling and benchmarking; kernels inside CUDA graphs are
 * counted when the graph is launched). */
uint64_t lsrn_kernel_launches(void);

/* Measurement aid with no counterpart in the paper: FP64 fused multiply-add
 * throughput of the current device in TFLOP/s (best of three launches of a
 * register-resident FMA loop, ~0.1 s), the peak against which FP64-arithmetic
 * bound kernels are compared.  Synchronises the device. */
lsrn_status lsrn_probe_fp64_fma(double* tflops);

/* Fill *opt with the defaults listed in lsrn_options.  INVALID_ARG if opt is NULL. */
lsrn_status lsrn_default_options(lsrn_options* opt);

/* Create a plan for A (Algorithm 1 step 1 / Algorithm 2 step 1; section 5's
 * augmentation [A; lambda I] for m >= n or [A/lambda, I_m] for m < n).
 *   A       matrix descriptor; data host or device.  Dense A whose layout is not
 *           the one the iteration streams (row-major for m >= n, column-major for
 *           m < n) and host A are copied into plan-owned device memory; otherwise
 *           the plan keeps the caller's device pointer, which must outlive it.
 *   opt     options, or NULL for defaults.
 *   stream  cudaStream_t to run on (NULL = legacy default stream).
 *   out     receives the plan.  Ownership passes to the caller, who frees it
 *           with lsrn_plan_destroy.
 * INVALID_ARG: m or n < 1, gamma <= 1, lambda < 0, tol <= 0, NULL data, bad ld,
 * CSR indices out of range or row_ptr not monotone (checked on the device).
 * UNSUPPORTED: dense A with min(m, n) > 4096 (the fused pass keeps a whole row
 * of X in registers / one shared-memory stage).  OOM when the workspace does
 * not fit.  Nothing is allocated on failure. */
lsrn_status lsrn_plan(const lsrn_matrix* A, const lsrn_options* opt, void* stream,
                      lsrn_plan_t* out);

/* Algorithm 1 steps 2-3 (A~ = G A, s x n) or Algorithm 2 steps 2-3 (A~ = A G,
 * m x s).  G has i.i.d. N(0,1) entries (rounded to the grid 2^-12) produced by
 * Philox4x32-10 + Box-Muller from (seed, row, column); it is never stored.
 * Asynchronous on the plan's stream. */
lsrn_status lsrn_sketch(lsrn_plan_t p);

/* Sketch reuse across lambda (section 5): a plan created with lambda > 0 keeps
 * the unaugmented part of its sketch (G_1 A for m >= n, A G_1 for m < n), and
 * this call rebuilds A~ for a new lambda > 0 without touching A:
 * A~ = G_1 A + lambda G_2 (m >= n, B = [A; lambda I]) or A G_1 / lambda + G_2
 * (m < n, B = [A / lambda, I_m]).  The preconditioner is then recomputed by the
 * next lsrn_precond / lsrn_solve_*.  INVALID_ARG if the plan was created with
 * lambda = 0 or lambda is not finite and positive.  Before the first sketch it
 * only records lambda.  Asynchronous. */
lsrn_status lsrn_plan_set_lambda(lsrn_plan_t p, double lambda);

/* Algorithm 1 steps 4-5 / Algorithm 2 steps 4-5: SVD of A~ on the device
 * (Householder QR, then one-sided Jacobi), numerical rank r, and N = V~
 * Sigma~^-1 (n x r) or M = U~ Sigma~^-1 (m x r).  Requires lsrn_sketch first
 * (LSRN_ERR_STATE otherwise).  Synchronises; writes r to *rank_out if non-NULL.
 * Returns LSRN_ERR_NOT_CONVERGED if the Jacobi sweeps have not converged after
 * 40 sweeps, and LSRN_ERR_TIMEOUT if a bounded wait of the dataflow sweep
 * (min(m, n) > 1024) gave up. */
lsrn_status lsrn_precond(lsrn_plan_t p, int64_t* rank_out);

/* Algorithm 1 steps 6-7 / Algorithm 2 steps 6-7 with LSQR (Paige and Saunders
 * 1982; stopping rules S1/S2 with atol = btol = tol on the preconditioned
 * problem), followed by opt.refine_max refinement steps.  Runs lsrn_sketch and
 * lsrn_precond first if they have not run.  The plan may be solved for many b.
 *   b     length m (host or device, FP64).
 *   x     length n (host or device, FP64), written with the solution.
 *   info  optional (NULL allowed), filled on return.
 * Returns OK, NOT_CONVERGED (cap reached, x = last iterate) or an error.
 * Rank 0 (A = 0) returns OK with x = 0.  Synchronises. */
lsrn_status lsrn_solve_lsqr(lsrn_plan_t p, const double* b, double* x, lsrn_info* info);

/* As lsrn_solve_lsqr, with Algorithm 3 (Chebyshev semi-iterative method):
 * sigma_L, sigma_U from Theorem 4.5 with alpha = opt.cs_alpha, K + 1 steps with
 * K = ceil((log tol - log 2) / log((sU - sL)/(sU + sL))), no inner products in
 * the loop.  Returns DIVERGED if the final residual exceeds the initial one
 * (the bounds did not hold); x then holds the last iterate.  INVALID_ARG if
 * (1 - alpha) sqrt(s) <= sqrt(r) (no valid upper bound). */
lsrn_status lsrn_solve_cs(lsrn_plan_t p, const double* b, double* x, lsrn_info* info);

/* ---- matrix-free operator (section 1: LSRN touches A only through products) ----
 * A (m x n) given by two callbacks that apply it to blocks of k vectors in
 * device memory, column-major:
 *   matmat(ctx, k, x, y):  y (m x k, ld m) = A x    (x: n x k, ld n)
 *   rmatmat(ctx, k, y, x): x (n x k, ld n) = A^T y  (y: m x k, ld m)
 * each returning 0 on success (nonzero: the call fails with LSRN_ERR_COMM).
 * The library synchronises its stream before a call and reads the output
 * after it, so a callback must finish its work before it returns; it runs on
 * the thread that called into the library.  The sketch is formed from blocks of
 * G's columns: A~ = G A as (A^T G^T)^T with rmatmat for m >= n, A~ = A G with
 * matmat for m < n (about 1 GiB of G per block); each iteration of LSQR or CS
 * costs one matmat and one rmatmat with k = 1.  There is no refinement step
 * (refine_max is taken as 0: the products are the caller's, in the caller's
 * arithmetic), so the accuracy is that of the FP64 iteration.  Ridge
 * (lambda > 0) works as for a stored matrix; iter_mode and sketch_mode are
 * ignored. */
typedef int32_t (*lsrn_matmat_fn)(void* ctx, int64_t k, const double* in, double* out);
typedef struct {
  int64_t m, n;
  lsrn_matmat_fn matmat;      /* out = A in */
  lsrn_matmat_fn rmatmat;     /* out = A^T in */
  void* ctx;
} lsrn_operator;

/* Plan for an operator A (see above).  INVALID_ARG for sizes < 1 or missing
 * callbacks; the rest as lsrn_plan. */
lsrn_status lsrn_plan_operator(const lsrn_operator* op, const lsrn_options* opt, void* stream,
                               lsrn_plan_t* out);

/* ---- choice of the oversampling factor gamma (section 4.3's cost model) ----
 * The paper's operation count of a solve, split into the parts that depend on
 * s = ceil(gamma q) (q = min(m, n)): the sketch (s m randn + 2 s m n) and the QR
 * of the s x q sketch (2 s q^2) grow linearly in s, the SVD of the q x q
 * triangle does not depend on s, and the iteration count falls with s --
 * Theorem 4.6's bound (log eps - log 2) / log sqrt(r/s) for LSQR, Algorithm 3's
 * K + 1 with Theorem 4.5's bounds (alpha = 1/sqrt(s)) for CS.  With per-unit
 * costs measured on this GPU (e.g. from lsrn_info of an earlier solve), the
 * predicted time T(gamma) = (c_sketch + c_qr) s + c_svd + c_iter N(gamma) is
 * minimised over gamma on a grid of step 0.01.  Host arithmetic only. */
typedef struct {
  int64_t m, n;               /* problem size */
  int64_t rank;               /* expected numerical rank r (<= 0: min(m, n)) */
  double tol;                 /* epsilon of the iteration (<= 0: 1e-14) */
  int32_t solver;             /* 0 LSQR, 1 CS */
  double c_sketch;            /* ms per unit of s in the sketch */
  double c_qr;                /* ms per unit of s in the QR of the sketch */
  double c_svd;               /* ms of the SVD of the q x q triangle */
  double c_iter;              /* ms per iteration */
  double gamma_min, gamma_max;  /* search range (<= 0: 1.05 and 8) */
} lsrn_gamma_model;

/* Writes the gamma of least predicted time to *gamma and that time (ms) to
 * *predicted_ms (either may be NULL).  INVALID_ARG for a NULL model, sizes < 1,
 * negative costs or an empty range; UNSUPPORTED if no gamma in the range admits
 * the solver (CS needs (1 - 1/sqrt(s)) sqrt(s) > sqrt(r)). */
lsrn_status lsrn_choose_gamma(const lsrn_gamma_model* model, double* gamma, double* predicted_ms);

/* ---- batched solve: many independent problems, phase by phase ----
 * Solves count independent problems (A[k], b[k]) -> x[k] with the same options
 * and solver (0 = LSQR, 1 = CS), each exactly as lsrn_plan + lsrn_solve_* would
 * (Algorithm 1 or 2 per problem, by its own shape), but phase by phase over the
 * whole batch:
 *   - plans are made from `threads` host threads (0: 8); the sketches are those
 *     of lsrn_sketch_group (the exact tensor-core sketches of small dense
 *     problems grouped into shared launches, the others each on its own
 *     stream, overlapping on the GPU);
 *   - the preconditioners of all problems whose short side is at most 128 and
 *     whose sketch is F64 or TC_SLICED run in ONE persistent launch, one CTA per
 *     problem (Householder QR, one-sided Jacobi, rank, N), largest first; other
 *     problems take the per-problem path (one SM's FP64 rate bounds a problem in
 *     the shared launch, which beats the per-problem path only for small q);
 *   - the iterations run per problem from the host threads, overlapping.
 * A, b, x: arrays of count descriptors / pointers (host or device data, as for
 * lsrn_plan and lsrn_solve_*).  info, status: optional arrays of count entries
 * receiving each problem's info and status.  Returns LSRN_OK if every problem
 * succeeded, else the first failing status (the others are still solved).
 * INVALID_ARG: count < 0, NULL arrays with count > 0, bad threads or solver.
 * Synchronises. */
lsrn_status lsrn_solve_batch(int32_t count, const lsrn_matrix* A, const double* const* b,
                             double* const* x, const lsrn_options* opt, int32_t solver,
                             int32_t threads, lsrn_info* info, int32_t* status);

/* Sketches (Algorithm 1/2 steps 2-3) of count plans at once, each with the
 * result lsrn_sketch would give it, bit for bit.  Dense plans in
 * LSRN_SKETCH_TC_SLICED mode whose long side fits one segment of the sketch's
 * scratch (and that are neither ridge, sharded nor matrix-free) are grouped:
 * their digit planes are prepared one after another on a stream of the call's
 * own, then the output tiles of all of them run in one tensor-core launch (a
 * tile table of (problem, row tile, column tile), the longest problems
 * first), in chunks of at most 8 GiB of planes.  Every other plan is sketched
 * by lsrn_sketch.  Each plan's stream waits for its sketch.  status: optional
 * array of count statuses.  Returns LSRN_OK or the first failing status.
 * INVALID_ARG: count < 0, plans NULL with count > 0, a NULL plan.
 * Synchronises. */
lsrn_status lsrn_sketch_group(int32_t count, lsrn_plan_t* plans, int32_t* status);

/* ---- sharded solve (section 4.4: A partitioned over processes) ----
 * One plan per shard (a GPU, a process or a host thread).  A is split along its
 * long side: for m >= n (Algorithm 1) each shard holds a block of consecutive
 * rows (all n columns); for m < n (Algorithm 2) a block of consecutive columns
 * (all m rows).  The shards exchange data only through the caller's allgather
 * callback:
 *   - the sketch: each shard computes its part of the contraction over the long
 *     side (G_p A_p, or A_p G_p) with G drawn at the block's global long-side
 *     indices (long_offset + i); the s x q partial sketches are gathered once
 *     and summed in rank order, so every shard holds the same A~ and computes
 *     the same N or M (redundantly, no broadcast);
 *   - each fused pass over A: the partial products over the long side (q values,
 *     q = min(m, n)) and the pass's sum of squares (one exchange of q + 1 values
 *     per iteration);
 *   - m >= n: ||b||^2 once per solve; m < n: the LSQR ||x||^2 once per iteration;
 *   - each refinement step's residual product in double-double, and for m < n
 *     the step's relative change of x.
 * Every shard runs identical scalar recurrences.  For m >= n, b is the shard's
 * rows of b and x (n values) is the whole solution on every shard; for m < n,
 * b is the whole b (m values) and x receives the shard's block of the solution
 * (A_local.n values).
 *   allgather(ctx, send, recv, count): send holds `count` doubles in device
 *     memory; the callback must write world * count doubles to recv (device
 *     memory, rank-major: shard p's values at recv[p * count]) before it
 *     returns, and return 0 (nonzero: the solve stops with LSRN_ERR_COMM).  The
 *     library synchronises its stream before the call and reads recv after it.
 *     The callback runs on the thread that called into the library.
 * Ridge (lambda > 0): the rows lambda I (m >= n) or the block I_m (m < n)
 * belong to shard 0. */
typedef int32_t (*lsrn_allgather_fn)(void* ctx, const double* send, double* recv, int64_t count);
typedef struct {
  int32_t rank, world;        /* this shard, number of shards (>= 1) */
  int32_t by_columns;         /* 0: row blocks of a tall A; 1: column blocks of a fat A */
  int64_t long_offset;        /* global index of this shard's first row (column) */
  int64_t long_total;         /* rows (columns) of the whole matrix, >= its short side */
  lsrn_allgather_fn allgather;
  void* ctx;
} lsrn_shard;

/* Plan for one shard: A_local is the shard's block (host or device data, dense
 * or CSR, as for lsrn_plan).  Every shard must pass the same options (seed
 * included) and call lsrn_sketch / lsrn_precond / lsrn_solve_* in the same
 * order: each exchange is a collective over the shards.  INVALID_ARG for
 * inconsistent shard fields, a long side shorter than the short side, or a
 * missing callback with world > 1. */
lsrn_status lsrn_plan_sharded(const lsrn_matrix* A_local, const lsrn_options* opt,
                              const lsrn_shard* shard, void* stream, lsrn_plan_t* out);

/* Release everything the plan owns.  NULL is accepted.  Synchronises. */
lsrn_status lsrn_plan_destroy(lsrn_plan_t p);

/* Copy the sketch to `out` (host or device, FP64): for m >= n A~ (s x n,
 * row-major); for m < n A~^T (s x m, row-major).  *rows and *cols receive the
 * shape.  STATE before lsrn_sketch.  Synchronises. */
lsrn_status lsrn_plan_get_sketch(lsrn_plan_t p, double* out, int64_t* rows, int64_t* cols);

/* Copy the three FP32 planes of a dense plan made with LSRN_ITER_F32X2 (the
 * operand of the double-float passes and of the triple-float residual of the
 * refinement): hi, lo and x3, each rows x ld row-major (rows = the long side,
 * ld = the short side rounded up to a multiple of 4, zero beyond it), with
 * X / scale = hi + lo + x3 exactly, hi = fl32(X / scale), lo = fl32(X / scale
 * - hi), x3 = fl32(X / scale - hi - lo) in round-to-nearest, and scale the
 * power of two that puts max |X| in [1, 2) (1 for a zero or non-finite X).
 * Any of hi, lo, x3, rows, ld, scale may be NULL; hi, lo, x3 are device or
 * host buffers of rows * ld floats owned by the caller.  UNSUPPORTED if the
 * plan has no planes (another iteration mode, CSR A, an operator, or a short
 * side the double-float passes do not take).  Synchronises. */
lsrn_status lsrn_plan_get_planes(lsrn_plan_t p, float* hi, float* lo, float* x3, int64_t* rows,
                                 int64_t* ld, double* scale);

/* Copy the preconditioner N (n' x r, row-major; n' = n for m >= n) or M
 * (m x r) to `out` and the r kept singular values of A~ (descending) to
 * `sigma` (either may be NULL).  STATE before lsrn_precond.  Synchronises. */
lsrn_status lsrn_plan_get_precond(lsrn_plan_t p, double* out, double* sigma, int64_t* rank);

/* Entries G[i0:i0+rows, j0:j0+cols] of the drawing array of the sketching
 * matrix (the draw for long-side index i and sketch index j; section 4.1
 * step 2), row-major, FP64, into device or host memory `g`; optionally the
 * unrounded binary32 normals into `z` (may be NULL).  Used to check the
 * generator bit for bit.  Synchronises. */
lsrn_status lsrn_generate_sketch_block(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0,
                                       int64_t rows, int64_t cols, double* g, float* z,
                                       void* stream);

/* Allocation-free variant of the FP64 sketch (no counterpart in the paper; an
 * interface for callers that cannot allocate device memory -- services that
 * reserve all device memory for their own pool at start-up, code running inside
 * another allocator's callbacks, or paths where cudaMalloc/cudaFree, which can
 * synchronise the device, are not allowed).
 *   A       device pointer, m x n row-major FP64 with leading dimension lda,
 *           m >= n (Algorithm 1's orientation).
 *   gamma   oversampling factor > 1; s = ceil(gamma * n).
 *   seed    key of G, as in lsrn_options.seed.
 *   out     device pointer receiving A~ = G A, s x n row-major (leading dimension
 *           n), equal to what lsrn_sketch computes for the same A, gamma and seed.
 *   stream  cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * The split-K partial sums live in one fixed device array of 32 MiB (4 Mi
 * doubles) that every GPU loading this library holds until process exit;
 * INVALID_ARG if s * n exceeds 4 Mi, if a pointer is not a device pointer, or
 * on bad sizes.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * Every call uses the same array, which keeps the previous call's contents (the
 * kernel writes every partial it reads, so nothing needs clearing); calls whose
 * work overlaps on the GPU (other streams, other threads) race on it.  No device
 * memory is allocated or freed. */
lsrn_status lsrn_sketch_f64_noalloc(const double* A, int64_t m, int64_t n, int64_t lda,
                                    double gamma, uint64_t seed, double* out, void* stream);

/* Test knobs (no counterpart in the paper): process-wide settings that let a
 * test drive a failure path on purpose without faulting the GPU.  Every knob
 * is 0 (off) by default and is read when a preconditioner starts.
 *   LSRN_KNOB_JACOBI_WAIT_NS          > 0: time limit, in nanoseconds of the
 *                                     GPU's global timer, of each dependency
 *                                     wait of the dataflow Jacobi sweep
 *                                     (min(m, n) > 1024); 0: one second.
 *   LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND != 0: the dataflow sweep starts after the
 *                                     first round's pairs, so every later pair
 *                                     waits on rows that are never published
 *                                     and the sweep's bounded wait runs out:
 *                                     lsrn_precond returns LSRN_ERR_TIMEOUT.
 *   LSRN_KNOB_QR_ABSENT_CTA           != 0: one CTA of the cooperative QR
 *                                     leaves before its first grid barrier,
 *                                     so the others' bounded barrier waits
 *                                     run out (limited by
 *                                     LSRN_KNOB_JACOBI_WAIT_NS when that is
 *                                     set, else ten seconds): lsrn_precond
 *                                     returns LSRN_ERR_TIMEOUT.
 * A preconditioner that fails leaves the plan needing a new sketch (the QR
 * overwrites the sketch in place); lsrn_solve_* redoes it by itself.
 * INVALID_ARG for an unknown knob or a negative value. */
typedef enum {
  LSRN_KNOB_JACOBI_WAIT_NS = 0,
  LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND = 1,
  LSRN_KNOB_QR_ABSENT_CTA = 2,
  LSRN_KNOB_COUNT = 3
} lsrn_test_knob;
lsrn_status lsrn_set_test_knob(int32_t knob, int64_t value);

/* ---- serving: a request queue with admission by device-memory budget ----
 * lsrn_submit copies the request (A, b, options) and returns a ticket at once;
 * worker threads plan and solve admitted requests on their own streams while
 * later requests keep arriving; lsrn_poll returns PENDING until the result is
 * ready, then OK/error, copies x (length n) and info, and retires the ticket.
 *   hbm_budget_bytes  device bytes that admitted requests may hold at once.
 *   max_slots         requests that may run concurrently (>= 1).
 *   solver            0 = LSQR, 1 = CS.
 * A request is admitted when a slot is free and its estimated device footprint
 * (the copy of A, the sketch, the factors, the vectors, the tensor-core
 * scratch, the FP32 planes of the mixed iteration modes) fits what the running
 * requests leave of the budget; the oldest
 * queued request that fits goes first.  Each slot has its own worker thread
 * and non-blocking stream on the device current at lsrn_server_create.
 * QUEUE_FULL when a single request alone exceeds the budget; INVALID_ARG for
 * an unknown or already collected ticket.  The server is thread-safe.
 * lsrn_server_destroy waits for running requests and drops queued ones. */
lsrn_status lsrn_server_create(size_t hbm_budget_bytes, int32_t max_slots, lsrn_server_t* out);
lsrn_status lsrn_submit(lsrn_server_t s, const lsrn_matrix* A, const double* b,
                        const lsrn_options* opt, int32_t solver, uint64_t* ticket);
lsrn_status lsrn_poll(lsrn_server_t s, uint64_t ticket, double* x_out, lsrn_info* info);
lsrn_status lsrn_server_destroy(lsrn_server_t s);

/* Continuous batching of the preconditioner phase (beyond the paper, for serving):
 * with max_short_side > 0, a request whose short side is at most that (and at
 * most 128, the batched kernel's limit) and whose preconditioner is the SVD of
 * an F64 or TC_SLICED sketch is sketched by its worker and then handed to the
 * server's batchers (four threads), one of which packs every request waiting
 * at that phase (after a 0.2 ms gathering window) into one launch of the
 * batched preconditioner (one CTA per request, as in lsrn_solve_batch) before
 * the workers continue with their iterations.  0 (the default) turns it off.  Results are those of the batched preconditioner,
 * which agrees with the per-request path to rounding.  INVALID_ARG outside
 * [0, 512]. */
lsrn_status lsrn_server_set_batching(lsrn_server_t s, int32_t max_short_side);
/* Batched preconditioner launches so far and the requests they packed. */
lsrn_status lsrn_server_stats(lsrn_server_t s, uint64_t* batches, uint64_t* batched_requests);

#ifdef __cplusplus
}
#endif

#endif /* LSRN_H */
