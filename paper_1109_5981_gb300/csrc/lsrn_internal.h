// Internal declarations shared by the LSRN translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "lsrn.h"

namespace lsrn {

#define LSRN_CUDA_TRY(expr)                              \
  do {                                                   \
    cudaError_t lsrn_err__ = (expr);                     \
    if (lsrn_err__ != cudaSuccess) {                     \
      record_cuda_error(lsrn_err__, #expr, __FILE__, __LINE__); \
      return lsrn_err__ == cudaErrorMemoryAllocation ? LSRN_ERR_OOM : LSRN_ERR_CUDA; \
    }                                                    \
  } while (0)

#define LSRN_TRY(expr)                 \
  do {                                 \
    lsrn_status lsrn_st__ = (expr);    \
    if (lsrn_st__ != LSRN_OK) return lsrn_st__; \
  } while (0)

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// Current value of a test knob (lsrn_set_test_knob); 0 when unset.
int64_t test_knob(int knob);
int num_sms();
// Stream-ordered allocation from the library's memory pool of the current device.
cudaError_t lsrn_malloc_async(void** ptr, size_t bytes, cudaStream_t st);

// ---- device scalar block (one per plan) -----------------------------------
enum ScalarSlot : int {
  SC_BNORM = 0,   // ||b|| (LSQR: beta_1)
  SC_ALPHA,       // alpha_k
  SC_BETA,        // beta_k
  SC_SU,          // tall: 1/beta (scale of stored u); fat: 1/alpha (scale of stored v)
  SC_CU,          // coefficient handed to the fused pass
  SC_RHOBAR,
  SC_PHIBAR,
  SC_ANORM2,
  SC_RNORM,
  SC_ARNORM,
  SC_ANORM,
  SC_XNORM,
  SC_CX,          // phi/rho   (fat vector update)
  SC_CW,          // theta/rho (fat vector update)
  SC_SS,          // sum of squares from the last pass
  SC_SS0,         // initial sum of squares (CS divergence test)
  SC_ONE,         // constant 1
  SC_ZERO,        // constant 0
  SC_TMP0,
  SC_TMP1,
  SC_ALPHA_NEW,
  SC_SV_NEW,
  SC_COUNT = 32
};

enum IntSlot : int { IC_DONE = 0, IC_ITN, IC_ISTOP, IC_CAP, IC_ROT, IC_TCERR, IC_PASSERR, IC_COUNT = 8 };

// Row modes of the fused pass over the rows of X (see k_iter.cu).
enum RowMode : int {
  RM_ACC_STATE = 0,  // t = st0[i]                                  (no dot)
  RM_LSQR_TALL = 1,  // t = d - c0*st0[i]; st0[i] = t; ss += t^2
  RM_CS_TALL = 2,    // t = st0[i] - c0*d; st0[i] = t; ss += t^2
  RM_APPLY = 3,      // t = d
  RM_FAT_INIT = 4,   // t = sx*d; st0[i] = t; ss += t^2;             acc with sx*t
  RM_FAT_LSQR = 5,   // t = sx*d - c0*st0[i]; st0[i] = t; ss += t^2; acc with sx*t
  RM_FAT_CS = 6,     // t = c0*st0[i] + sx*d; st0[i] = t; st1[i] += c1*t; acc with sx*t
};

struct RowArgs {
  int mode;
  double* st0;
  double* st1;
  const double* coef;   // device pointer to c0, c1 (read at kernel start)
  double sx;            // constant scale of every X row
};

// ---- row sharding (lsrn_plan_sharded) ----------------------------------------
struct Shard {
  int rank = 0, world = 1;
  int64_t lbase = 0;              // global long-side index of this shard's first row
  int64_t long_total = 0;         // long side of the whole matrix
  lsrn_allgather_fn fn = nullptr;
  void* ctx = nullptr;
  double* send = nullptr;         // plan-owned staging: cap doubles
  double* recv = nullptr;         // world * cap doubles
  int64_t cap = 0;
};

// ---- the plan -----------------------------------------------------------
struct Plan {
  int device = 0;
  cudaStream_t stream = nullptr;
  lsrn_options opt{};
  int64_t m = 0, n = 0;
  bool tall = true;
  bool ridge = false;
  double lam = 0.0;
  bool csr = false;

  // X: the matrix the fused passes stream, row-major: A (m >= n) or A^T (m < n)
  const double* X = nullptr;
  int64_t ldx = 0;
  int64_t xrows = 0, xcols = 0;     // rows, columns of X
  double xscale = 1.0;              // 1/lambda for the fat ridge operator [A/lambda, I]
  int64_t extra_rows = 0;           // ridge rows appended to X (coef extra_coef * e_j)
  double extra_coef = 0.0;
  int64_t nstate = 0;               // xrows + extra_rows
  double* owned_X = nullptr;        // plan-owned copy of X, if any
  const float* X32 = nullptr;       // FP32 copy of X (iteration mode LSRN_ITER_F32)
  int64_t ldx32 = 0;
  bool pass_f32 = false;            // fused passes currently stream X32
  const float* X2h = nullptr;       // double-float planes of X / x2scale (LSRN_ITER_F32X2)
  const float* X2l = nullptr;
  const float* X3 = nullptr;        // third plane: X / x2scale = X2h + X2l + X3 exactly
  int64_t ldx2 = 0;
  double x2scale = 1.0;

  // CSR (m >= n: A; m < n: A^T) in both orientations for deterministic passes
  const int64_t* rp = nullptr;  const int32_t* ci = nullptr;  const double* cv = nullptr;   // rows of X
  const int64_t* rpT = nullptr; const int32_t* ciT = nullptr; const double* cvT = nullptr;  // columns of X
  int64_t nnz = 0;
  double* tcsr = nullptr;           // row coefficients between the two sparse passes (xrows)
  std::vector<void*> owned;         // device buffers freed at destroy

  // sketch and preconditioner
  int64_t s = 0;                    // sketch size
  int64_t q = 0;                    // xcols: n (tall) or m (fat)
  double* Xs = nullptr;             // s x q sketch (A~ or A~^T), row-major; QR in place
  double* Wj = nullptr;             // q x q Jacobi workspace (rows = columns of R^T)
  double* tau = nullptr;
  double* sig = nullptr;            // q singular values, sorted descending
  int* perm = nullptr;
  double* Nm = nullptr;             // q x r row-major (N or M)
  double* NT = nullptr;             // r x q row-major
  int64_t rank = 0;
  double sigma_max = 0.0, sigma_min = 0.0;
  int sweeps = 0;                   // FP64 Jacobi sweeps
  int sweeps_df = 0;                // double-float Jacobi sweeps before them
  int state = 0;                    // 0 planned, 1 sketched, 2 preconditioned
  // Replay each Jacobi sweep from a captured CUDA graph.  Off for plans run by
  // the server: there several streams share the GPU and fill one another's
  // launch gaps, and the per-plan capture only adds host work.
  bool graph_sweeps = true;

  // iteration workspace
  double* scal = nullptr;           // SC_COUNT doubles
  int* iscal = nullptr;             // IC_COUNT ints
  double* coefs = nullptr;          // CS coefficient table (2 per step), capacity ncoef
  int64_t ncoef = 0;
  double* st0 = nullptr;            // nstate
  double* st1 = nullptr;            // nstate
  double* vq = nullptr;             // q (g / q vectors, reduced)
  double* vq2 = nullptr;            // q
  double* tmpq = nullptr;           // q
  double* vr[6] = {nullptr};        // r-length vectors
  double* xfull = nullptr;          // nstate (fat) or q (tall x)
  double* bdev = nullptr;           // m (+ ridge) right-hand side staging
  double* pvec = nullptr;           // (nblk + 1) * xcols pass partials
  double* pvec2 = nullptr;          // second partial buffer (double-double low parts)
  double* pscal = nullptr;          // (nblk + 1) scalar partials
  int nblk = 0;                     // CTAs of the fused pass
  cudaEvent_t ev[10] = {nullptr};  // [8]: end of the QR, [9]: end of the Jacobi sweeps
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gemm_events;   // tensor-core GEMM launches
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pass_events;   // fused passes of the main sweep
  bool time_passes = false;
  float t_sketch_ms = 0, t_precond_ms = 0, t_sketch_gemm_ms = 0, t_qr_ms = 0, t_jacobi_ms = 0;
  double* sk_base = nullptr;           // ridge: the unaugmented sketch G_1 A / A G_1 (s x q)
  int sketch_used = LSRN_SKETCH_F64;   // sketch arithmetic that produced Xs
  bool sketch_escalated = false;       // AUTO replaced the BF16 sketch by the exact one
  double bf16_noise = 0.0;             // 2^-8 ||A~||_F / sqrt(q) of a BF16 sketch
  double bound_widen = 0.0;            // relative widening of the Theorem 4.5 bounds
  bool is_op = false;               // A given as an operator (lsrn_plan_operator)
  lsrn_operator op{};
  double* opd = nullptr;            // operator passes: X vin (xrows)
  double* opt_mult = nullptr;       // operator passes: row multipliers (xrows)
  bool sharded = false;             // a shard of a row-partitioned matrix (lsrn_plan_sharded)
  Shard shard;
};

// Sum `count` doubles at `buf` (device) over the shards of a sharded plan:
// allgather through the caller's callback, then a fixed rank-order sum on the
// device, identical on every shard.  No-op for an unsharded plan.
lsrn_status shard_sum(Plan* p, double* buf, int64_t count);
// The same for a double-double vector (hi, lo), summed in double-double.
lsrn_status shard_sum_dd(Plan* p, double* hi, double* lo, int64_t count);

// ---- batched preconditioner (one launch for many problems) -----------------
struct BatchPrecond {
  double* X;      // S x Q sketch (factored in place)
  double* W;      // Q x Q Jacobi workspace
  double* sig;    // Q singular values (descending)
  int* perm;      // Q
  double* N;      // Q x r
  double* NT;     // r x Q
  int64_t S, Q;
  double rcond;
  int* out;       // [rank, sweeps] (sweeps > 40: not converged)
  double* dout;   // [sigma_1, sigma_r]
};
bool batch_precond_applies(int64_t Q);
// A sketched plan whose preconditioner the batched launch can compute.
bool precond_batchable(const Plan* p);
// Preconditioners of sketched, batchable plans in one launch (largest first);
// st[k] receives each plan's status, state 2 on success.
void precond_batch(std::vector<Plan*>& plans, std::vector<lsrn_status>& st);
// N = R^-1 (q x q) and NT from the upper triangle of the factored sketch Xs; T scratch 64 q doubles
lsrn_status launch_trinv(const double* Xs, int64_t q, double* N, double* NT, double* T,
                         double* diag, cudaStream_t st);
lsrn_status launch_batched_precond(const BatchPrecond* dev_probs, int count, int* dev_next,
                                   cudaStream_t st);

// ---- kernels (launchers) -------------------------------------------------
// sketch: C (S x Q, ldc) = xscale * Gamma[lrow0 : lrow0+L]^T X   (X: L x Q row-major)
// lbase: long-side index of X's first row in the whole matrix (G is drawn at
// rows lbase + l; nonzero for a shard of a row-partitioned matrix).
lsrn_status launch_sketch_f64(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                              int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                              double* scratch, size_t scratch_bytes, cudaStream_t st,
                              int64_t lbase = 0);
size_t sketch_f64_scratch_bytes(int64_t L, int64_t Q, int64_t S);
// Same sketch, always through split-K partial sums held in caller-provided
// scratch (scratch_doubles >= nz * S * Q for the split nz it picks, nz >= 1).
lsrn_status launch_sketch_f64_splitk_into(const double* X, int64_t L, int64_t Q, int64_t ldx,
                                          int64_t S, uint64_t seed, uint32_t tag, double* C,
                                          int64_t ldc, double* scratch, size_t scratch_doubles,
                                          cudaStream_t st);
// Tensor-core sketch (exact bf16 digit slices, FP64-accurate), same contract as
// launch_sketch_f64; X is processed in segments of seg_rows rows, each needing
// sketch_tc_scratch_bytes(seg_rows, Q, S) of scratch; *err is set on a timed-out wait.
size_t sketch_tc_scratch_bytes(int64_t Ls, int64_t Q, int64_t S);
int64_t sketch_tc_segment_rows(int64_t L, int64_t Q, int64_t S, size_t budget_bytes);
// Segment length the plan uses: a function of (L, Q, S) and a fixed scratch
// budget only, never of the memory free at the time, so the sketch (whose
// per-column exponents and final roundings are per segment) is reproducible.
constexpr size_t kTcScratchBudget = (size_t)8 << 30;
inline int64_t sketch_tc_plan_segment_rows(int64_t L, int64_t Q, int64_t S) {
  return sketch_tc_segment_rows(L, Q, S, kTcScratchBudget);
}
lsrn_status launch_sketch_tc(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                             int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                             void* scratch, size_t scratch_bytes, int64_t seg_rows, int* err,
                             cudaStream_t st,
                             std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* gemm_events,
                             int64_t lbase = 0);
// Grouped exact sketch: several single-segment problems, their digit planes
// prepared one after another, then all their output tiles in one launch.  Each
// problem's C is bit for bit what launch_sketch_tc gives for it alone.
struct TcGroupItem {
  const double* X;
  int64_t L, Q, ldx;
  double xscale;
  int64_t S;
  uint64_t seed;
  uint32_t tag;
  int64_t lbase;
  double* C;
  int64_t ldc;
  int* err;
};
size_t sketch_tc_group_scratch_bytes(const std::vector<TcGroupItem>& items);
lsrn_status launch_sketch_tc_grouped(const std::vector<TcGroupItem>& items, void* scratch,
                                     size_t scratch_bytes, cudaStream_t st);
// Single-pass BF16 sketch (operands rounded to bf16 once, FP32 accumulation in
// TMEM per 2048 rows, FP64 across chunks and K splits); same contract.
size_t sketch_bf16_scratch_bytes(int64_t Ls, int64_t Q, int64_t S);
int64_t sketch_bf16_segment_rows(int64_t L, int64_t Q, int64_t S, size_t budget_bytes);
lsrn_status launch_sketch_bf16(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                               int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                               void* scratch, size_t scratch_bytes, int64_t seg_rows, int* err,
                               cudaStream_t st,
                               std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* gemm_events,
                               int64_t lbase = 0);
// C[i, j] = scale_c * C[i, j] + coef * Gamma[lrow0 + j, i], i < S, j < Q
lsrn_status launch_sketch_add_gamma(double* C, int64_t ldc, int64_t S, int64_t Q, uint64_t seed,
                                    uint32_t tag, int64_t lrow0, double coef, cudaStream_t st);
// C = scale * base + coef * Gamma[lrow0 + j, i] (ridge sketch from its unaugmented part)
lsrn_status launch_ridge_combine(const double* base, double* C, int64_t ldc, int64_t S, int64_t Q,
                                 double scale, uint64_t seed, uint32_t tag, int64_t lrow0,
                                 double coef, cudaStream_t st);
lsrn_status launch_gamma_block(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0, int64_t rows,
                               int64_t cols, double* g, float* z, cudaStream_t st);
// CSR sketch: C (S x Q) = xscale * Gamma^T X with X given by its columns (CSC of X)
lsrn_status launch_sketch_csr(const int64_t* colptr, const int32_t* rowidx, const double* vals,
                              int64_t L, int64_t Q, double xscale, int64_t S, uint64_t seed,
                              uint32_t tag, double* C, int64_t ldc, cudaStream_t st,
                              int64_t lbase = 0);

// Theorem 4.5 bounds (sigma_L, sigma_U) for the plan's r and s and alpha option
lsrn_status thm45_bounds(const Plan* p, double* sL, double* sU);
bool is_device_pointer(const void* ptr);

// SVD / preconditioner: Xs (S x Q) -> N (Q x r), NT, sig; returns rank.
// With bf16_check the sketch's noise floor p->bf16_noise is measured first, and
// the call returns kPrecondEscalate right after the QR when the smallest
// |R_ii| (an upper bound on sigma_min) is below 16 times it.
constexpr lsrn_status kPrecondEscalate = (lsrn_status)100;   // internal, never returned by the ABI
lsrn_status run_precond(Plan* p, bool bf16_check = false);
// Householder QR of X (S x Q, row-major, in place) in one cooperative launch
// (k_qr_coop.cu); *ran is false when the device cannot hold the grid.
lsrn_status launch_qr_coop(double* X, int64_t S, int64_t Q, double* tau, cudaStream_t st, bool* ran);
// Double-float Jacobi pre-sweeps on R (k_jacobi_df.cu): for 1024 < q <= 4096,
// leaves Y = P R (P the accumulated rotations) in p->Wj for the FP64 sweeps.
bool jacobi_df_applies(int64_t Q);
lsrn_status jacobi_df_phase(Plan* p, int64_t wait_ns_knob, int skip_items, int* sweeps_out);
// Server-owned plans launch the Jacobi rounds directly (see Plan::graph_sweeps).
void plan_disable_sweep_graphs(lsrn_plan_t p);
// The plan behind a handle, and its short side q.
Plan* plan_internal(lsrn_plan_t p);
int64_t plan_short_side(lsrn_plan_t p);

// fused passes
lsrn_status launch_row_pass(const Plan* p, const double* vin, const RowArgs& a, double* pvec,
                            double* pscal, const int* done);
lsrn_status launch_extra_rows(const Plan* p, const double* vin, const RowArgs& a, double* pvec,
                              double* pscal, const int* done);
// The fused pass of an operator plan: d = X vin (callback), row updates as in
// the fused pass, pvec[0:xcols] = X^T multipliers (callback), pscal[0] = sum of squares.
lsrn_status op_row_pass(Plan* p, const double* vin, const RowArgs& a, double* pvec, double* pscal,
                        const int* done);
// Columns k0 .. k0 + kb of the drawing array, column-major: G[c * L + l] = Gamma[lbase + l, k0 + c]
lsrn_status launch_gamma_cols(uint64_t seed, uint32_t tag, int64_t L, int64_t k0, int64_t kb,
                              int64_t S, double* G, cudaStream_t st);
lsrn_status launch_dd_pass(const Plan* p, const double* vin, const double* bvec, double* rout,
                           double* pvec_hi, double* pvec_lo, const int* done);
lsrn_status launch_reduce(const double* pvec, int nslots, int64_t C, double* out,
                          const double* pscal, double* scal_out, const int* done, cudaStream_t st);
lsrn_status launch_reduce_dd(const double* phi, const double* plo, int nslots, int64_t C,
                             double* out_hi, double* out_lo, cudaStream_t st);
// out[i] = c[0]*dot(M_i, v) + c[1]*y[i]; if y2: y2[i] += c[2]*out[i]    (c: device pointer)
lsrn_status launch_gemv(const double* M, int64_t R, int64_t C, const double* v, double* out,
                        const double* y, double* y2, const double* c, const int* done,
                        cudaStream_t st);
// Y (rows x ldy, FP32, zero beyond cols) = X (rows x cols, FP64, ldx)
bool x2_applies(int64_t C);
// LSRN_ITER_AUTO to a concrete pass precision (the rule in lsrn.h); other modes unchanged
inline int32_t resolve_iter_mode(int32_t mode, int64_t m, int64_t n, bool csr) {
  if (mode != LSRN_ITER_AUTO) return mode;
  if (csr || 8.0 * (double)m * (double)n < (double)(1ll << 30)) return LSRN_ITER_F64;
  if (x2_applies(std::min(m, n))) return LSRN_ITER_F32X2;
  return m >= n ? LSRN_ITER_F32 : LSRN_ITER_F64;
}
lsrn_status launch_to_x2(const double* X, int64_t rows, int64_t cols, int64_t ldx, float* Yh,
                         float* Yl, float* Y3, int64_t ldy, unsigned long long* maxbits, double* xs,
                         cudaStream_t st);
lsrn_status launch_to_f32(const double* X, int64_t rows, int64_t cols, int64_t ldx, float* Y,
                          int64_t ldy, cudaStream_t st);
// out[i] = M_i . v accumulated in double-double (warp per row)
lsrn_status launch_gemv_dd(const double* M, int64_t R, int64_t C, const double* v, double* out,
                           cudaStream_t st);
// CSR pass: t = Xrow . vin per row, epilogue as RowArgs; then the transpose product
// Sparse fused pass: out (xcols) = X^T t, t from the row pass (+ ridge rows); ss -> *scal_ss
lsrn_status csr_fused_pass(const Plan* p, const double* vin, const RowArgs& a, double* out,
                           double* tbuf, double* scal_ss, const int* done);

}  // namespace lsrn
