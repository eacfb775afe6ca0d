// C ABI of the LSRN library: plan management and the solve entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

lsrn_status run_lsqr(Plan* p, int* iters, int* istop);
lsrn_status run_cs(Plan* p, int* iters, double* sL, double* sU, bool* diverged);
lsrn_status run_refine(Plan* p, int nsteps, int* inner, int* taken);
lsrn_status finish_x(Plan* p, double* xout);
int pass_blocks(int64_t rows, int64_t C, bool x2);
lsrn_status csr_plan_setup(Plan* p, const lsrn_matrix* A, bool host);

static thread_local char g_last_error[512];
std::atomic<unsigned long long> g_kernel_launches{0};
static std::atomic<long long> g_test_knobs[LSRN_KNOB_COUNT];

int64_t test_knob(int knob) {
  if (knob < 0 || knob >= LSRN_KNOB_COUNT) return 0;
  return (int64_t)g_test_knobs[knob].load(std::memory_order_relaxed);
}

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s:%d: %s -> %s", file, line, what,
           cudaGetErrorString(e));
  if (getenv("LSRN_VERBOSE")) fprintf(stderr, "lsrn: %s\n", g_last_error);
}

// Stream-ordered allocations of the library come from one memory pool per
// device that keeps up to a quarter of the device memory reserved after frees,
// so repeated plans (each holding tens of GB of planes and scratch) reuse
// mapped memory instead of returning it to the driver at every synchronisation.
// The process-wide default pool is left as it is.
cudaError_t lsrn_malloc_async(void** ptr, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(ptr, bytes, st);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (pools[dev] == nullptr) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t p = nullptr;
      if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
        cudaGetLastError();
        return cudaMallocAsync(ptr, bytes, st);
      }
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      uint64_t keep = total_b / 4;
      cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[dev] = p;
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

int num_sms() {
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

bool is_device_pointer(const void* ptr) {
  if (ptr == nullptr) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

namespace {

// out (rows x cols, ld_out, FP64) = transpose or copy of a (FP64/FP32) matrix.
// src element (i, j) of the logical rows_src x cols_src matrix is at
// src[i*ld_row + j*ld_col].
__global__ void gather_matrix_kernel(const void* __restrict__ src, int dtype, int64_t ld_row,
                                     int64_t ld_col, int64_t rows, int64_t cols,
                                     double* __restrict__ out, int64_t ld_out) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  // read with the stride-1 index fastest (coalesced for either source layout)
  const bool src_rows_fast = ld_col == 1;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = src_rows_fast ? r0 + k : r0 + threadIdx.x;
    const int64_t j = src_rows_fast ? c0 + threadIdx.x : c0 + k;
    double v = 0.0;
    if (i < rows && j < cols) {
      const int64_t off = i * ld_row + j * ld_col;
      v = dtype == LSRN_F32 ? (double)((const float*)src)[off] : ((const double*)src)[off];
    }
    if (src_rows_fast) tile[k][threadIdx.x] = v;
    else tile[threadIdx.x][k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = r0 + k, j = c0 + threadIdx.x;
    if (i < rows && j < cols) out[i * ld_out + j] = tile[k][threadIdx.x];
  }
}

}  // namespace

lsrn_status gather_matrix(const void* src, int dtype, int64_t ld_row, int64_t ld_col, int64_t rows,
                          int64_t cols, double* out, int64_t ld_out, cudaStream_t st) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  launch(gather_matrix_kernel, grid, dim3(32, 8), 0, st, src, dtype, ld_row, ld_col, rows, cols, out,
                                                      ld_out);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

static lsrn_status dalloc(Plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = lsrn_malloc_async(ptr, bytes, p->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    record_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    return e == cudaErrorMemoryAllocation ? LSRN_ERR_OOM : LSRN_ERR_CUDA;
  }
  p->owned.push_back(*ptr);
  return LSRN_OK;
}

template <class T>
static lsrn_status dalloc_n(Plan* p, T** ptr, int64_t n) {
  return dalloc(p, (void**)ptr, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
}

static void release(Plan* p) {
  if (p == nullptr) return;
  if (p->stream) {
    for (void* ptr : p->owned) cudaFreeAsync(ptr, p->stream);
    if (p->coefs) cudaFreeAsync(p->coefs, p->stream);
    if (p->sk_base) cudaFreeAsync(p->sk_base, p->stream);
    if (p->shard.send) cudaFreeAsync(p->shard.send, p->stream);
    if (p->shard.recv) cudaFreeAsync(p->shard.recv, p->stream);
    cudaStreamSynchronize(p->stream);
  }
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  for (auto* v : {&p->gemm_events, &p->pass_events})
    for (auto& pr : *v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

static lsrn_status validate_options(const lsrn_options& o) {
  if (!(o.gamma > 1.0) || !std::isfinite(o.gamma)) return LSRN_ERR_INVALID_ARG;
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return LSRN_ERR_INVALID_ARG;
  if (!(o.lambda >= 0.0) || !std::isfinite(o.lambda)) return LSRN_ERR_INVALID_ARG;
  if (o.refine_max < 0 || o.refine_max > 16) return LSRN_ERR_INVALID_ARG;
  if (!(o.refine_tol > 0.0) || !(o.refine_tol < 1.0)) return LSRN_ERR_INVALID_ARG;
  if (o.sketch_mode < LSRN_SKETCH_F64 || o.sketch_mode > LSRN_SKETCH_AUTO) return LSRN_ERR_INVALID_ARG;
  if (o.iter_mode != LSRN_ITER_F64 && o.iter_mode != LSRN_ITER_F32 &&
      o.iter_mode != LSRN_ITER_F32X2 && o.iter_mode != LSRN_ITER_AUTO)
    return LSRN_ERR_INVALID_ARG;
  if (o.precond_mode != LSRN_PRECOND_SVD && o.precond_mode != LSRN_PRECOND_QR)
    return LSRN_ERR_INVALID_ARG;
  if (o.precond_mode == LSRN_PRECOND_QR && !(o.lambda > 0.0)) return LSRN_ERR_INVALID_ARG;
  if (o.svd_mode != LSRN_SVD_F64 && o.svd_mode != LSRN_SVD_DF) return LSRN_ERR_INVALID_ARG;
  return LSRN_OK;
}

static lsrn_status plan_workspace(Plan* p) {
  const int64_t q = p->q, s = p->s;
  // sparse and operator passes write whole vectors
  const bool x2 = p->opt.iter_mode == LSRN_ITER_F32X2 && !p->csr && !p->is_op && x2_applies(p->xcols);
  p->nblk = (p->csr || p->is_op) ? 1 : pass_blocks(p->xrows, p->xcols, x2);
  if (p->nblk <= 0) return LSRN_ERR_UNSUPPORTED;
  LSRN_TRY(dalloc_n(p, &p->Xs, s * q));
  LSRN_TRY(dalloc_n(p, &p->Wj, q * q));
  LSRN_TRY(dalloc_n(p, &p->tau, q));
  LSRN_TRY(dalloc_n(p, &p->sig, q));
  LSRN_TRY(dalloc_n(p, &p->perm, q));
  LSRN_TRY(dalloc_n(p, &p->Nm, q * q));
  LSRN_TRY(dalloc_n(p, &p->NT, q * q));
  LSRN_TRY(dalloc_n(p, &p->scal, (int64_t)SC_COUNT));
  LSRN_TRY(dalloc_n(p, &p->iscal, (int64_t)IC_COUNT));
  // +2: the staged pass copies row state in 16-byte units
  LSRN_TRY(dalloc_n(p, &p->st0, p->nstate + 2));
  LSRN_TRY(dalloc_n(p, &p->st1, p->nstate + 2));
  LSRN_TRY(dalloc_n(p, &p->vq, q + 2));   // + 2: a sharded pass appends its sum of squares
  LSRN_TRY(dalloc_n(p, &p->vq2, q));
  LSRN_TRY(dalloc_n(p, &p->tmpq, q));
  for (auto& v : p->vr) LSRN_TRY(dalloc_n(p, &v, q));
  LSRN_TRY(dalloc_n(p, &p->xfull, std::max(q, p->nstate)));
  LSRN_TRY(dalloc_n(p, &p->bdev, std::max<int64_t>(p->m, 1) + 2));   // + 2: 16-byte bulk copies
  LSRN_TRY(dalloc_n(p, &p->pvec, (int64_t)(p->nblk + 1) * p->xcols));
  LSRN_TRY(dalloc_n(p, &p->pvec2, (int64_t)(p->nblk + 1) * p->xcols));
  LSRN_TRY(dalloc_n(p, &p->pscal, std::max<int64_t>(p->nblk + 1, 8 * (int64_t)num_sms() + 2)));
  if (p->csr) LSRN_TRY(dalloc_n(p, &p->tcsr, p->xrows));
  LSRN_CUDA_TRY(cudaMemsetAsync(p->scal, 0, SC_COUNT * sizeof(double), p->stream));
  LSRN_CUDA_TRY(cudaMemsetAsync(p->iscal, 0, IC_COUNT * sizeof(int), p->stream));
  const double one = 1.0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->scal + SC_ONE, &one, sizeof(double), cudaMemcpyHostToDevice,
                                p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return LSRN_OK;
}

static lsrn_status dense_setup(Plan* p, const lsrn_matrix* A, bool host) {
  const int64_t m = A->m, n = A->n;
  const bool rowmajor = A->format == LSRN_DENSE_ROWMAJOR;
  if (A->ld < (rowmajor ? n : m)) return LSRN_ERR_INVALID_ARG;
  // X = A (row-major) for m >= n, X = A^T (row-major, i.e. A column-major) for m < n.
  const bool layout_ok = (p->tall && rowmajor) || (!p->tall && !rowmajor);
  const bool aligned = ((uintptr_t)A->values % 16 == 0) && (A->ld % 2 == 0);
  if (!host && layout_ok && aligned && A->dtype == LSRN_F64) {
    p->X = (const double*)A->values;
    p->ldx = A->ld;
    return LSRN_OK;
  }
  const int64_t xr = p->xrows, xc = p->xcols;
  const int64_t ldx = xc + (xc & 1);
  double* Xo = nullptr;
  LSRN_TRY(dalloc_n(p, &Xo, xr * ldx));
  if (host && layout_ok && A->dtype == LSRN_F64) {   // straight copy, rows of X are rows of the input
    LSRN_CUDA_TRY(cudaMemcpy2DAsync(Xo, ldx * sizeof(double), A->values, A->ld * sizeof(double),
                                    xc * sizeof(double), xr, cudaMemcpyHostToDevice, p->stream));
    p->X = Xo;
    p->owned_X = Xo;
    p->ldx = ldx;
    return LSRN_OK;
  }
  const void* src = A->values;
  void* staged = nullptr;
  const size_t esz = A->dtype == LSRN_F32 ? 4 : 8;
  const int64_t src_elems = rowmajor ? (m - 1) * A->ld + n : (n - 1) * A->ld + m;
  if (host) {
    LSRN_TRY(dalloc(p, &staged, (size_t)src_elems * esz));
    LSRN_CUDA_TRY(cudaMemcpyAsync(staged, A->values, (size_t)src_elems * esz,
                                  cudaMemcpyHostToDevice, p->stream));
    src = staged;
  }
  // element (i, j) of A sits at i*ld + j (row-major) or i + j*ld (column-major);
  // X(i', j') = A(i', j') for m >= n and A(j', i') for m < n.
  int64_t ld_row, ld_col;
  if (p->tall) {
    ld_row = rowmajor ? A->ld : 1;
    ld_col = rowmajor ? 1 : A->ld;
  } else {
    ld_row = rowmajor ? 1 : A->ld;
    ld_col = rowmajor ? A->ld : 1;
  }
  LSRN_TRY(gather_matrix(src, A->dtype, ld_row, ld_col, xr, xc, Xo, ldx, p->stream));
  if (staged) {
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    cudaFreeAsync(staged, p->stream);
    p->owned.erase(std::find(p->owned.begin(), p->owned.end(), staged));
  }
  p->X = Xo;
  p->owned_X = Xo;
  p->ldx = ldx;
  return LSRN_OK;
}

}  // namespace lsrn

using namespace lsrn;

struct lsrn_plan_s : Plan {};

namespace lsrn {
void plan_disable_sweep_graphs(lsrn_plan_t p) {
  if (p != nullptr) p->graph_sweeps = false;
}
Plan* plan_internal(lsrn_plan_t p) { return p; }
int64_t plan_short_side(lsrn_plan_t p) { return p ? p->q : 0; }
}  // namespace lsrn

extern "C" {

const char* lsrn_status_string(lsrn_status s) {
  switch (s) {
    case LSRN_OK: return "LSRN_OK";
    case LSRN_PENDING: return "LSRN_PENDING";
    case LSRN_ERR_INVALID_ARG: return "LSRN_ERR_INVALID_ARG";
    case LSRN_ERR_OOM: return "LSRN_ERR_OOM";
    case LSRN_ERR_CUDA: return "LSRN_ERR_CUDA";
    case LSRN_ERR_NOT_CONVERGED: return "LSRN_ERR_NOT_CONVERGED";
    case LSRN_ERR_DIVERGED: return "LSRN_ERR_DIVERGED";
    case LSRN_ERR_TIMEOUT: return "LSRN_ERR_TIMEOUT";
    case LSRN_ERR_QUEUE_FULL: return "LSRN_ERR_QUEUE_FULL";
    case LSRN_ERR_STATE: return "LSRN_ERR_STATE";
    case LSRN_ERR_UNSUPPORTED: return "LSRN_ERR_UNSUPPORTED";
    case LSRN_ERR_COMM: return "LSRN_ERR_COMM";
  }
  return "LSRN_UNKNOWN_STATUS";
}

const char* lsrn_last_error_message(void) { return g_last_error; }

uint64_t lsrn_kernel_launches(void) { return (uint64_t)g_kernel_launches.load(); }

lsrn_status lsrn_set_test_knob(int32_t knob, int64_t value) {
  if (knob < 0 || knob >= LSRN_KNOB_COUNT || value < 0) return LSRN_ERR_INVALID_ARG;
  g_test_knobs[knob].store((long long)value, std::memory_order_relaxed);
  return LSRN_OK;
}

lsrn_status lsrn_default_options(lsrn_options* opt) {
  if (opt == nullptr) return LSRN_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->gamma = 2.0;
  opt->tol = 1e-14;
  opt->lambda = 0.0;
  opt->rcond = -1.0;
  opt->cs_alpha = -1.0;
  opt->refine_tol = 1e-3;
  opt->max_iter = -1;
  opt->refine_max = 1;
  opt->seed = 0;
  opt->sketch_mode = LSRN_SKETCH_F64;
  return LSRN_OK;
}

static lsrn_status plan_create(const lsrn_matrix* A, const lsrn_options* opt, void* stream,
                               const lsrn_shard* sh, lsrn_plan_t* out,
                               const lsrn_operator* op = nullptr) {
  if (out == nullptr || (A == nullptr && op == nullptr)) return LSRN_ERR_INVALID_ARG;
  *out = nullptr;
  lsrn_matrix opm{};   // an operator plan's shape, no stored entries
  if (op != nullptr) {
    if (op->m < 1 || op->n < 1 || op->matmat == nullptr || op->rmatmat == nullptr)
      return LSRN_ERR_INVALID_ARG;
    opm.m = op->m;
    opm.n = op->n;
    opm.format = LSRN_DENSE_ROWMAJOR;
    A = &opm;
  }
  if (A->m < 1 || A->n < 1 || (A->values == nullptr && op == nullptr)) return LSRN_ERR_INVALID_ARG;
  if (A->format != LSRN_DENSE_ROWMAJOR && A->format != LSRN_DENSE_COLMAJOR && A->format != LSRN_CSR)
    return LSRN_ERR_INVALID_ARG;
  if (A->dtype != LSRN_F64 && A->dtype != LSRN_F32) return LSRN_ERR_INVALID_ARG;
  lsrn_options o;
  if (opt) o = *opt;
  else lsrn_default_options(&o);
  if (op != nullptr) {   // products are the caller's: FP64 sweeps, no refinement, no stored-A sketch
    o.iter_mode = LSRN_ITER_F64;
    o.sketch_mode = LSRN_SKETCH_F64;
    o.refine_max = 0;
  }
  LSRN_TRY(validate_options(o));
  o.iter_mode = resolve_iter_mode(o.iter_mode, A->m, A->n, A->format == LSRN_CSR);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LSRN_ERR_CUDA;
  }
  lsrn_plan_s* p = new (std::nothrow) lsrn_plan_s();
  if (p == nullptr) return LSRN_ERR_OOM;
  cudaGetDevice(&p->device);
  if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    p->stream = nullptr;
    release(p);
    return LSRN_ERR_CUDA;
  }
  for (auto& e : p->ev) cudaEventCreate(&e);
  if (stream) {  // order after the caller's prior work on its stream
    cudaEventRecord(p->ev[7], (cudaStream_t)stream);
    cudaStreamWaitEvent(p->stream, p->ev[7], 0);
  }
  p->opt = o;
  p->m = A->m;
  p->n = A->n;
  p->tall = A->m >= A->n;
  if (sh != nullptr) {   // a shard: orientation from the partition; exchanges when world > 1
    p->sharded = sh->world > 1;
    p->tall = sh->by_columns == 0;
    p->shard.rank = sh->rank;
    p->shard.world = sh->world;
    p->shard.lbase = sh->long_offset;
    p->shard.long_total = sh->long_total;
    p->shard.fn = sh->allgather;
    p->shard.ctx = sh->ctx;
  }
  p->lam = o.lambda;
  p->ridge = o.lambda > 0.0;
  p->csr = A->format == LSRN_CSR;
  p->xrows = p->tall ? A->m : A->n;
  p->xcols = p->tall ? A->n : A->m;
  p->q = p->xcols;
  p->s = (int64_t)std::ceil(o.gamma * (double)p->q);
  if (p->s <= p->q) p->s = p->q + 1;
  if (p->ridge) {
    // every shard sketches and iterates the same augmented problem (the same
    // A~ from the summed sketch, the same scaling of a fat A); only shard 0
    // holds the appended rows lambda I / I_m in its passes
    p->extra_coef = p->tall ? o.lambda : 1.0;
    p->xscale = p->tall ? 1.0 : 1.0 / o.lambda;
    if (!(p->sharded && p->shard.rank != 0)) p->extra_rows = p->tall ? A->n : A->m;
  }
  p->nstate = p->xrows + p->extra_rows;
  lsrn_status st;
  if (op != nullptr) {
    p->is_op = true;
    p->op = *op;
    st = dalloc_n(p, &p->opd, p->xrows);
    if (st == LSRN_OK) st = dalloc_n(p, &p->opt_mult, p->xrows);
  } else {
    const bool host = !is_device_pointer(A->values);
    if (p->csr) st = csr_plan_setup(p, A, host);
    else st = dense_setup(p, A, host);
  }
  // FP32 passes only for m >= n: there x = N y stays in range(N), which the sketch fixes;
  // for m < n the iterate lives in R^n and FP32 rounding of A would let null(A) in.
  if (st == LSRN_OK && o.iter_mode == LSRN_ITER_F32 && !p->csr && p->tall) {
    p->ldx32 = p->xcols + (p->xcols & 1);
    float* x32 = nullptr;
    st = dalloc_n(p, &x32, p->xrows * p->ldx32);
    if (st == LSRN_OK)
      st = launch_to_f32(p->X, p->xrows, p->xcols, p->ldx, x32, p->ldx32, p->stream);
    p->X32 = x32;
  }
  if (st == LSRN_OK && o.iter_mode == LSRN_ITER_F32X2 && !p->csr && x2_applies(p->xcols)) {
    p->ldx2 = (p->xcols + 3) / 4 * 4;
    float *xh = nullptr, *xl = nullptr, *x3 = nullptr;
    unsigned long long* mb = nullptr;
    st = dalloc_n(p, &xh, p->xrows * p->ldx2);
    if (st == LSRN_OK) st = dalloc_n(p, &xl, p->xrows * p->ldx2);
    if (st == LSRN_OK) st = dalloc_n(p, &x3, p->xrows * p->ldx2);
    if (st == LSRN_OK) st = dalloc_n(p, &mb, 1);
    if (st == LSRN_OK)
      st = launch_to_x2(p->X, p->xrows, p->xcols, p->ldx, xh, xl, x3, p->ldx2, mb, &p->x2scale,
                        p->stream);
    p->X2h = xh;
    p->X2l = xl;
    p->X3 = x3;
  }
  if (st == LSRN_OK) st = plan_workspace(p);
  if (st == LSRN_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LSRN_ERR_CUDA;
  if (st != LSRN_OK) {
    release(p);
    return st;
  }
  *out = p;
  return LSRN_OK;
}

lsrn_status lsrn_plan(const lsrn_matrix* A, const lsrn_options* opt, void* stream,
                      lsrn_plan_t* out) {
  return plan_create(A, opt, stream, nullptr, out);
}

lsrn_status lsrn_plan_operator(const lsrn_operator* op, const lsrn_options* opt, void* stream,
                               lsrn_plan_t* out) {
  if (op == nullptr) return LSRN_ERR_INVALID_ARG;
  return plan_create(nullptr, opt, stream, nullptr, out, op);
}

lsrn_status lsrn_plan_sharded(const lsrn_matrix* A_local, const lsrn_options* opt,
                              const lsrn_shard* shard, void* stream, lsrn_plan_t* out) {
  if (out == nullptr || A_local == nullptr || shard == nullptr) return LSRN_ERR_INVALID_ARG;
  *out = nullptr;
  const lsrn_shard& sh = *shard;
  if (sh.world < 1 || sh.rank < 0 || sh.rank >= sh.world) return LSRN_ERR_INVALID_ARG;
  if (sh.world > 1 && sh.allgather == nullptr) return LSRN_ERR_INVALID_ARG;
  if (sh.by_columns != 0 && sh.by_columns != 1) return LSRN_ERR_INVALID_ARG;
  if (A_local->m < 1 || A_local->n < 1) return LSRN_ERR_INVALID_ARG;
  const int64_t local_long = sh.by_columns ? A_local->n : A_local->m;
  const int64_t short_side = sh.by_columns ? A_local->m : A_local->n;
  if (sh.long_offset < 0 || sh.long_total < sh.long_offset + local_long) return LSRN_ERR_INVALID_ARG;
  if (sh.long_total > (int64_t)0xFFFFFFFFll) return LSRN_ERR_INVALID_ARG;   // G's counter word
  if (sh.long_total < short_side) return LSRN_ERR_INVALID_ARG;              // not the long side
  return plan_create(A_local, opt, stream, &sh, out);
}

// Ridge sketch from the kept unaugmented part: tall, B = [A; lambda I] and
// A~ = G_1 A + lambda G_2; fat, B = [A / lambda, I_m] and A~ = A G_1 / lambda +
// G_2 (section 5), G_2 being G's rows that meet the appended block.
static lsrn_status ridge_sketch(Plan* p) {
  const int64_t lrow0 = p->shard.long_total > 0 ? p->shard.long_total : p->xrows;
  return launch_ridge_combine(p->sk_base, p->Xs, p->q, p->s, p->q, p->xscale, p->opt.seed, 0u,
                              lrow0, p->extra_coef, p->stream);
}

// The sketch Xs with the given arithmetic (dense: F64, TC_SLICED or BF16; CSR
// always FP64), plus the ridge rows and, for a shard, the sum over shards.
static lsrn_status sketch_with(Plan* p, int mode) {
  const uint32_t tag = 0;
  // A ridge plan sketches X unscaled and keeps that part (sk_base), so that a
  // new lambda only recombines it with the rows of G that meet lambda I / I_m.
  const double xs_sk = p->ridge ? 1.0 : p->xscale;
  if (p->is_op) {
    // A~ rows from blocks of G's columns: m >= n: (A^T Gamma_blk)^T, m < n: (A Gamma_blk)^T;
    // the callback's column-major output block is a run of rows of Xs
    mode = LSRN_SKETCH_F64;
    const int64_t L = p->xrows;
    int64_t kb = std::max<int64_t>(4, ((int64_t)1 << 27) / std::max<int64_t>(L, 1) / 4 * 4);
    kb = std::min<int64_t>(kb, (p->s + 3) / 4 * 4);
    double* G = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&G, (size_t)L * kb * sizeof(double), p->stream));
    const lsrn_matmat_fn fn = p->tall ? p->op.rmatmat : p->op.matmat;
    lsrn_status st = LSRN_OK;
    for (int64_t k0 = 0; k0 < p->s && st == LSRN_OK; k0 += kb) {
      const int64_t nb = std::min(kb, p->s - k0);
      st = launch_gamma_cols(p->opt.seed, tag, L, k0, nb, p->s, G, p->stream);
      if (st == LSRN_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LSRN_ERR_CUDA;
      if (st == LSRN_OK && fn(p->op.ctx, nb, G, p->Xs + k0 * p->q) != 0) st = LSRN_ERR_COMM;
    }
    cudaFreeAsync(G, p->stream);
    LSRN_TRY(st);
  } else if (p->csr) {
    mode = LSRN_SKETCH_F64;
    LSRN_TRY(launch_sketch_csr(p->rpT, p->ciT, p->cvT, p->xrows, p->q, xs_sk, p->s,
                               p->opt.seed, tag, p->Xs, p->q, p->stream, p->shard.lbase));
  } else if (mode == LSRN_SKETCH_TC_SLICED || mode == LSRN_SKETCH_BF16) {
    const bool bf = mode == LSRN_SKETCH_BF16;
    int64_t seg = bf ? sketch_bf16_segment_rows(p->xrows, p->q, p->s, kTcScratchBudget)
                     : sketch_tc_plan_segment_rows(p->xrows, p->q, p->s);
    if (const char* env = getenv("LSRN_TC_SEGMENT_ROWS")) {   // testing: force small segments
      const long long v = atoll(env);
      if (v >= 64) seg = std::min<int64_t>(seg, (int64_t)(v / 64 * 64));
    }
    const size_t scratch = bf ? sketch_bf16_scratch_bytes(seg, p->q, p->s)
                              : sketch_tc_scratch_bytes(seg, p->q, p->s);
    void* buf = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async(&buf, scratch, p->stream));
    LSRN_CUDA_TRY(cudaMemsetAsync(p->iscal + IC_TCERR, 0, sizeof(int), p->stream));
    lsrn_status st =
        bf ? launch_sketch_bf16(p->X, p->xrows, p->q, p->ldx, xs_sk, p->s, p->opt.seed, tag,
                                p->Xs, p->q, buf, scratch, seg, p->iscal + IC_TCERR, p->stream,
                                &p->gemm_events, p->shard.lbase)
           : launch_sketch_tc(p->X, p->xrows, p->q, p->ldx, xs_sk, p->s, p->opt.seed, tag,
                              p->Xs, p->q, buf, scratch, seg, p->iscal + IC_TCERR, p->stream,
                              &p->gemm_events, p->shard.lbase);
    cudaFreeAsync(buf, p->stream);
    LSRN_TRY(st);
  } else {
    mode = LSRN_SKETCH_F64;
    const size_t scratch = sketch_f64_scratch_bytes(p->xrows, p->q, p->s);
    double* buf = nullptr;
    if (scratch) LSRN_CUDA_TRY(lsrn_malloc_async((void**)&buf, scratch, p->stream));
    lsrn_status st = launch_sketch_f64(p->X, p->xrows, p->q, p->ldx, xs_sk, p->s, p->opt.seed,
                                       tag, p->Xs, p->q, buf, scratch, p->stream, p->shard.lbase);
    if (buf) cudaFreeAsync(buf, p->stream);
    LSRN_TRY(st);
  }
  LSRN_TRY(shard_sum(p, p->Xs, p->s * p->q));   // A~ = sum over shards of G_p A_p
  p->sketch_used = mode;
  if (p->ridge) {
    if (p->sk_base == nullptr)
      LSRN_CUDA_TRY(lsrn_malloc_async((void**)&p->sk_base, (size_t)p->s * p->q * sizeof(double),
                                      p->stream));
    LSRN_CUDA_TRY(cudaMemcpyAsync(p->sk_base, p->Xs, (size_t)p->s * p->q * sizeof(double),
                                  cudaMemcpyDeviceToDevice, p->stream));
    LSRN_TRY(ridge_sketch(p));
  }
  return LSRN_OK;
}

// A tensor-core sketch's bounded waits: LSRN_ERR_TIMEOUT if one gave up.
static lsrn_status check_tc_error(Plan* p) {
  if (p->sketch_used != LSRN_SKETCH_TC_SLICED && p->sketch_used != LSRN_SKETCH_BF16) return LSRN_OK;
  int tcerr = 0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&tcerr, p->iscal + IC_TCERR, sizeof(int), cudaMemcpyDeviceToHost,
                                p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return tcerr ? LSRN_ERR_TIMEOUT : LSRN_OK;
}

lsrn_status lsrn_sketch(lsrn_plan_t p) {
  if (p == nullptr) return LSRN_ERR_INVALID_ARG;
  cudaSetDevice(p->device);
  cudaEventRecord(p->ev[0], p->stream);
  const int mode = p->opt.sketch_mode == LSRN_SKETCH_AUTO ? LSRN_SKETCH_BF16 : p->opt.sketch_mode;
  for (auto& pr : p->gemm_events) {   // GEMM times of an earlier sketch of this plan
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  p->gemm_events.clear();
  p->sketch_escalated = false;
  p->bound_widen = 0.0;
  LSRN_TRY(sketch_with(p, mode));
  cudaEventRecord(p->ev[1], p->stream);
  p->state = 1;   // a new sketch invalidates an earlier preconditioner
  return LSRN_OK;
}

lsrn_status lsrn_plan_set_lambda(lsrn_plan_t p, double lambda) {
  if (p == nullptr || !(lambda > 0.0) || !std::isfinite(lambda)) return LSRN_ERR_INVALID_ARG;
  if (!p->ridge) return LSRN_ERR_INVALID_ARG;
  cudaSetDevice(p->device);
  p->lam = lambda;
  p->opt.lambda = lambda;
  p->extra_coef = p->tall ? lambda : 1.0;
  p->xscale = p->tall ? 1.0 : 1.0 / lambda;
  if (p->sk_base == nullptr) {   // not sketched yet: the next sketch uses the new lambda
    p->state = 0;
    return LSRN_OK;
  }
  cudaEventRecord(p->ev[0], p->stream);
  LSRN_TRY(ridge_sketch(p));
  cudaEventRecord(p->ev[1], p->stream);
  p->bound_widen = 0.0;
  p->state = 1;   // the preconditioner must be recomputed
  return LSRN_OK;
}

lsrn_status lsrn_precond(lsrn_plan_t p, int64_t* rank_out) {
  if (p == nullptr) return LSRN_ERR_INVALID_ARG;
  if (p->state < 1) return LSRN_ERR_STATE;
  cudaSetDevice(p->device);
  {
    const lsrn_status st = check_tc_error(p);
    if (st != LSRN_OK) {
      p->state = 0;
      return st;
    }
  }
  cudaEventRecord(p->ev[2], p->stream);
  {
    const bool auto_bf16 = p->opt.sketch_mode == LSRN_SKETCH_AUTO && p->sketch_used == LSRN_SKETCH_BF16;
    const bool measure = auto_bf16 || p->sketch_used == LSRN_SKETCH_BF16;
    lsrn_status st = run_precond(p, measure);
    double eta = 1.0;   // BF16 noise floor relative to sigma_min
    if (st == LSRN_OK && measure)
      eta = (p->rank == p->q && p->sigma_min > 0.0) ? p->bf16_noise / p->sigma_min : 1.0;
    if (auto_bf16 && (st == kPrecondEscalate || (st == LSRN_OK && !(eta <= 1.0 / 16.0)))) {
      // the BF16 embedding cannot resolve this spectrum: the exact sketch instead
      st = sketch_with(p, LSRN_SKETCH_TC_SLICED);
      if (st == LSRN_OK) st = check_tc_error(p);
      if (st == LSRN_OK) st = run_precond(p, false);
      p->sketch_escalated = true;
      p->bound_widen = 0.0;
    } else if (st == kPrecondEscalate) {
      st = LSRN_ERR_CUDA;   // cannot happen: only AUTO asks for the early check to return
    } else if (st == LSRN_OK && measure) {
      p->bound_widen = std::min(2.0 * eta, 0.9);
    }
    if (st != LSRN_OK) {
      p->state = 0;   // the QR has overwritten the sketch: a retry must sketch again
      return st;
    }
  }
  cudaEventRecord(p->ev[3], p->stream);
  LSRN_CUDA_TRY(cudaEventSynchronize(p->ev[3]));
  cudaEventElapsedTime(&p->t_sketch_ms, p->ev[0], p->ev[1]);
  cudaEventElapsedTime(&p->t_precond_ms, p->ev[2], p->ev[3]);
  if (cudaEventElapsedTime(&p->t_qr_ms, p->ev[2], p->ev[8]) != cudaSuccess) {
    cudaGetLastError();
    p->t_qr_ms = 0.f;
  }
  if (cudaEventElapsedTime(&p->t_jacobi_ms, p->ev[8], p->ev[9]) != cudaSuccess) {
    cudaGetLastError();
    p->t_jacobi_ms = 0.f;
  }
  p->t_sketch_gemm_ms = 0.f;
  for (auto& pr : p->gemm_events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) p->t_sketch_gemm_ms += ms;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  p->gemm_events.clear();
  p->state = 2;
  if (rank_out) *rank_out = p->rank;
  return LSRN_OK;
}

static lsrn_status solve_common(lsrn_plan_t p, const double* b, double* x, lsrn_info* info,
                                bool use_cs) {
  if (p == nullptr || b == nullptr || x == nullptr) return LSRN_ERR_INVALID_ARG;
  cudaSetDevice(p->device);
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->bdev, b, p->m * sizeof(double), cudaMemcpyDefault, p->stream));
  if (p->state < 1) LSRN_TRY(lsrn_sketch(p));
  if (p->state < 2) LSRN_TRY(lsrn_precond(p, nullptr));
  lsrn_info inf;
  memset(&inf, 0, sizeof(inf));
  // a shard reports the whole problem: the long side is the partitioned one
  const bool long_total = p->shard.long_total > 0;
  inf.m = long_total && p->tall ? p->shard.long_total : p->m;
  inf.n = long_total && !p->tall ? p->shard.long_total : p->n;
  inf.s = p->s;
  inf.rank = p->rank;
  inf.tall = p->tall ? 1 : 0;
  inf.sigma_max_sketch = p->sigma_max;
  inf.sigma_min_sketch = p->sigma_min;
  inf.t_sketch_ms = p->t_sketch_ms;
  inf.t_precond_ms = p->t_precond_ms;
  inf.t_qr_ms = p->t_qr_ms;
  inf.jacobi_sweeps = p->sweeps;
  inf.jacobi_sweeps_df = p->sweeps_df;
  inf.iter_used = p->opt.iter_mode;
  inf.t_jacobi_ms = p->t_jacobi_ms;
  inf.sketch_used = p->sketch_used;
  inf.sketch_escalated = p->sketch_escalated ? 1 : 0;
  inf.t_sketch_gemm_ms = p->t_sketch_gemm_ms;
  lsrn_status result = LSRN_OK;
  const bool xdev = is_device_pointer(x);
  double* xout = xdev ? x : p->xfull;
  if (p->rank == 0) {
    LSRN_TRY(finish_x(p, xout));
  } else {
    cudaEventRecord(p->ev[4], p->stream);
    p->time_passes = true;
    if (use_cs) {
      bool diverged = false;
      LSRN_TRY(run_cs(p, &inf.iterations, &inf.sigma_L, &inf.sigma_U, &diverged));
      if (diverged) result = LSRN_ERR_DIVERGED;
    } else {
      LSRN_TRY(run_lsqr(p, &inf.iterations, &inf.istop));
      if (inf.istop == 0) result = LSRN_ERR_NOT_CONVERGED;
      double sc[SC_COUNT];
      LSRN_CUDA_TRY(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->stream));
      LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
      inf.rnorm_est = sc[SC_RNORM];
      inf.arnorm_est = sc[SC_ARNORM];
      inf.anorm_est = sc[SC_ANORM];
    }
    cudaEventRecord(p->ev[5], p->stream);
    if (result == LSRN_OK) {
      LSRN_TRY(run_refine(p, p->opt.refine_max, &inf.refine_iterations, &inf.refine_steps));
    }
    p->time_passes = false;
    cudaEventRecord(p->ev[6], p->stream);
    LSRN_TRY(finish_x(p, xout));
    LSRN_CUDA_TRY(cudaEventSynchronize(p->ev[6]));
    cudaEventElapsedTime(&inf.t_iter_ms, p->ev[4], p->ev[5]);
    std::vector<float> pass_ms;
    for (auto& pr : p->pass_events) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) pass_ms.push_back(ms);
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    p->pass_events.clear();
    // passes launched after the sweep converged return at once: count only
    // those that streamed A (at least a quarter of the longest pass)
    const float longest = pass_ms.empty() ? 0.f : *std::max_element(pass_ms.begin(), pass_ms.end());
    for (float ms : pass_ms) {
      inf.t_pass_ms += ms;
      if (ms >= 0.25f * longest) inf.n_pass += 1;
    }
    cudaEventElapsedTime(&inf.t_refine_ms, p->ev[5], p->ev[6]);
  }
  if (!xdev)
    LSRN_CUDA_TRY(cudaMemcpyAsync(x, xout, p->n * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  int passerr = 0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&passerr, p->iscal + IC_PASSERR, sizeof(int),
                                cudaMemcpyDeviceToHost, p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  if (passerr) result = LSRN_ERR_TIMEOUT;   // a bounded wait of a staged pass gave up
  inf.status = result;
  if (info) *info = inf;
  return result;
}

lsrn_status lsrn_solve_lsqr(lsrn_plan_t p, const double* b, double* x, lsrn_info* info) {
  return solve_common(p, b, x, info, false);
}

lsrn_status lsrn_solve_cs(lsrn_plan_t p, const double* b, double* x, lsrn_info* info) {
  if (p != nullptr && p->state >= 2 && p->rank > 0) {
    double sL, sU;
    if (thm45_bounds(p, &sL, &sU) != LSRN_OK) return LSRN_ERR_INVALID_ARG;
  }
  return solve_common(p, b, x, info, true);
}

}  // extern "C"

namespace lsrn {

bool precond_batchable(const Plan* p) {
  return (p->sketch_used == LSRN_SKETCH_F64 || p->sketch_used == LSRN_SKETCH_TC_SLICED) &&
         p->opt.sketch_mode != LSRN_SKETCH_AUTO && p->opt.sketch_mode != LSRN_SKETCH_BF16 &&
         p->opt.precond_mode == LSRN_PRECOND_SVD && batch_precond_applies(p->q) && p->state == 1;
}

// Preconditioners of sketched plans (precond_batchable) in one persistent
// launch, largest first.  Waits for each plan's sketch; on return every plan
// whose st[k] is LSRN_OK is preconditioned (state 2).
void precond_batch(std::vector<Plan*>& plans, std::vector<lsrn_status>& st) {
  const int nb = (int)plans.size();
  if (nb == 0) return;
  std::vector<int> order((size_t)nb);
  for (int k = 0; k < nb; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return plans[a]->q > plans[c]->q; });
  cudaStream_t bs = nullptr;
  lsrn_status bst = LSRN_OK;
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    bst = LSRN_ERR_CUDA;
  }
  std::vector<BatchPrecond> hp;
  std::vector<int> live;   // positions in `plans` of the problems launched
  BatchPrecond* dp = nullptr;
  int* dout_i = nullptr;
  double* dout_d = nullptr;
  int* dnext = nullptr;
  if (bst == LSRN_OK) {
    for (int k : order) {   // every sketch must be complete, its bounded waits clean
      Plan* p = plans[k];
      if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
        cudaGetLastError();
        st[k] = LSRN_ERR_CUDA;
      } else if (check_tc_error(p) != LSRN_OK) {
        st[k] = LSRN_ERR_TIMEOUT;
      }
      if (st[k] == LSRN_OK) live.push_back(k);
    }
  }
  const int nl = (int)live.size();
  if (bst == LSRN_OK && nl > 0 &&
      (lsrn_malloc_async((void**)&dp, sizeof(BatchPrecond) * nl, bs) != cudaSuccess ||
       lsrn_malloc_async((void**)&dout_i, sizeof(int) * 2 * nl, bs) != cudaSuccess ||
       lsrn_malloc_async((void**)&dout_d, sizeof(double) * 2 * nl, bs) != cudaSuccess ||
       lsrn_malloc_async((void**)&dnext, sizeof(int), bs) != cudaSuccess)) {
    cudaGetLastError();
    bst = LSRN_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float batch_ms = 0.f;
  std::vector<int> oi((size_t)2 * std::max(nl, 1));
  std::vector<double> od((size_t)2 * std::max(nl, 1));
  if (bst == LSRN_OK && nl > 0) {
    for (int k = 0; k < nl; ++k) {
      Plan* p = plans[live[k]];
      const double rcond = p->opt.rcond >= 0.0 ? p->opt.rcond : (double)std::max(p->s, p->q) * 0x1p-53;
      hp.push_back(BatchPrecond{p->Xs, p->Wj, p->sig, p->perm, p->Nm, p->NT, p->s, p->q, rcond,
                                dout_i + 2 * k, dout_d + 2 * k});
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaMemcpyAsync(dp, hp.data(), sizeof(BatchPrecond) * nl, cudaMemcpyHostToDevice, bs) !=
        cudaSuccess)
      bst = LSRN_ERR_CUDA;
    cudaEventRecord(e0, bs);
    if (bst == LSRN_OK) bst = launch_batched_precond(dp, nl, dnext, bs);
    cudaEventRecord(e1, bs);
    if (bst == LSRN_OK &&
        (cudaMemcpyAsync(oi.data(), dout_i, sizeof(int) * 2 * nl, cudaMemcpyDeviceToHost, bs) !=
             cudaSuccess ||
         cudaMemcpyAsync(od.data(), dout_d, sizeof(double) * 2 * nl, cudaMemcpyDeviceToHost, bs) !=
             cudaSuccess ||
         cudaStreamSynchronize(bs) != cudaSuccess)) {
      cudaGetLastError();
      bst = LSRN_ERR_CUDA;
    }
    if (bst == LSRN_OK) cudaEventElapsedTime(&batch_ms, e0, e1);
  }
  for (int k = 0; k < nl; ++k) {
    const int i = live[k];
    if (bst != LSRN_OK) {
      st[i] = bst;
      continue;
    }
    Plan* p = plans[i];
    p->rank = oi[2 * k];
    p->sweeps = oi[2 * k + 1];
    p->sweeps_df = 0;
    p->sigma_max = od[2 * k];
    p->sigma_min = od[2 * k + 1];
    if (p->sweeps > 40) {
      st[i] = LSRN_ERR_NOT_CONVERGED;
      p->state = 0;   // the QR overwrote the sketch
      continue;
    }
    cudaEventElapsedTime(&p->t_sketch_ms, p->ev[0], p->ev[1]);
    p->t_precond_ms = batch_ms;   // the whole batch's launch
    p->t_qr_ms = 0.f;
    p->t_jacobi_ms = 0.f;
    p->state = 2;
  }
  if (bst != LSRN_OK)
    for (int k : order)
      if (st[k] == LSRN_OK) st[k] = bst;
  if (dp) cudaFreeAsync(dp, bs);
  if (dout_i) cudaFreeAsync(dout_i, bs);
  if (dout_d) cudaFreeAsync(dout_d, bs);
  if (dnext) cudaFreeAsync(dnext, bs);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (bs) {
    cudaStreamSynchronize(bs);
    cudaStreamDestroy(bs);
  }
}

}  // namespace lsrn

namespace {

// Run body(i) for i in [0, n) on `threads` host threads, each bound to `dev`.
template <class F>
void parallel_for(int n, int threads, int dev, F body) {
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) body(i);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

lsrn_status lsrn_choose_gamma(const lsrn_gamma_model* md, double* gamma, double* predicted_ms) {
  if (md == nullptr || md->m < 1 || md->n < 1) return LSRN_ERR_INVALID_ARG;
  if (!(md->c_sketch >= 0.0) || !(md->c_qr >= 0.0) || !(md->c_svd >= 0.0) || !(md->c_iter >= 0.0))
    return LSRN_ERR_INVALID_ARG;
  const double q = (double)std::min(md->m, md->n);
  const double r = md->rank > 0 ? (double)std::min<int64_t>(md->rank, std::min(md->m, md->n)) : q;
  const double eps = md->tol > 0.0 ? md->tol : 1e-14;
  const double g0 = md->gamma_min > 0.0 ? md->gamma_min : 1.05;
  const double g1 = md->gamma_max > 0.0 ? md->gamma_max : 8.0;
  if (!(g1 >= g0) || !(g0 > 1.0)) return LSRN_ERR_INVALID_ARG;
  double best_t = INFINITY, best_g = 0.0;
  const int steps = (int)std::floor((g1 - g0) / 0.01 + 1e-9);
  for (int k = 0; k <= steps; ++k) {
    const double g = g0 + 0.01 * k;
    const double s = std::ceil(g * q);
    if (!(s > r) || !(s > q)) continue;
    double iters;
    if (md->solver == 1) {
      const double a = 1.0 / std::sqrt(s);
      const double lo = (1.0 - a) * std::sqrt(s) - std::sqrt(r);
      if (!(lo > 0.0)) continue;
      const double sU = 1.0 / lo, sL = 1.0 / ((1.0 + a) * std::sqrt(s) + std::sqrt(r));
      const double rho = (sU - sL) / (sU + sL);
      iters = std::ceil((std::log(eps) - std::log(2.0)) / std::log(rho)) + 1.0;
    } else {
      iters = std::ceil((std::log(eps) - std::log(2.0)) / std::log(std::sqrt(r / s)));
    }
    const double t = (md->c_sketch + md->c_qr) * s + md->c_svd + md->c_iter * iters;
    if (t < best_t) {
      best_t = t;
      best_g = g;
    }
  }
  if (!(best_g > 0.0)) return LSRN_ERR_UNSUPPORTED;
  if (gamma) *gamma = best_g;
  if (predicted_ms) *predicted_ms = best_t;
  return LSRN_OK;
}

lsrn_status lsrn_sketch_group(int32_t count, lsrn_plan_t* plans, int32_t* status) {
  if (count < 0 || (count > 0 && plans == nullptr)) return LSRN_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k)
    if (plans[k] == nullptr) return LSRN_ERR_INVALID_ARG;
  std::vector<lsrn_status> st((size_t)count, LSRN_OK);
  std::vector<int> grp, rest;
  const bool forced_segments = getenv("LSRN_TC_SEGMENT_ROWS") != nullptr;
  int dev = -1;
  for (int k = 0; k < count; ++k) {
    Plan* p = plans[k];
    const bool ok = !forced_segments && !p->csr && !p->is_op && !p->sharded && !p->ridge &&
                    p->opt.sketch_mode == LSRN_SKETCH_TC_SLICED && (dev < 0 || p->device == dev) &&
                    sketch_tc_plan_segment_rows(p->xrows, p->q, p->s) >= p->xrows;
    if (ok) {
      grp.push_back(k);
      dev = p->device;
    } else {
      rest.push_back(k);
    }
  }
  if (!rest.empty()) {
    int cur = 0;
    cudaGetDevice(&cur);
    parallel_for((int)rest.size(), std::min<int>(8, (int)rest.size()), cur,
                 [&](int i) { st[rest[i]] = lsrn_sketch(plans[rest[i]]); });
  }
  if (!grp.empty()) {
    cudaSetDevice(dev);
    cudaStream_t gs = nullptr;
    lsrn_status gst = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) == cudaSuccess ? LSRN_OK
                                                                                            : LSRN_ERR_CUDA;
    size_t k0 = 0;
    while (gst == LSRN_OK && k0 < grp.size()) {
      // a chunk of plans whose digit planes fit 8 GiB (at least one plan)
      std::vector<TcGroupItem> items;
      std::vector<Plan*> ps;
      size_t k1 = k0;
      for (; k1 < grp.size(); ++k1) {
        Plan* p = plans[grp[k1]];
        std::vector<TcGroupItem> trial = items;
        trial.push_back(TcGroupItem{p->X, p->xrows, p->q, p->ldx, p->xscale, p->s, p->opt.seed, 0u,
                                    p->shard.lbase, p->Xs, p->q, p->iscal + IC_TCERR});
        if (!items.empty() && sketch_tc_group_scratch_bytes(trial) > kTcScratchBudget) break;
        items.swap(trial);
        ps.push_back(p);
      }
      for (Plan* p : ps) {   // the plan's own earlier work (A's layout) comes first
        cudaEventRecord(p->ev[0], p->stream);
        cudaStreamWaitEvent(gs, p->ev[0], 0);
        for (auto& pr : p->gemm_events) {
          cudaEventDestroy(pr.first);
          cudaEventDestroy(pr.second);
        }
        p->gemm_events.clear();
        p->sketch_escalated = false;
        p->bound_widen = 0.0;
        cudaMemsetAsync(p->iscal + IC_TCERR, 0, sizeof(int), gs);
      }
      const size_t bytes = sketch_tc_group_scratch_bytes(items);
      void* buf = nullptr;
      if (lsrn_malloc_async(&buf, bytes, gs) != cudaSuccess) {
        cudaGetLastError();
        gst = LSRN_ERR_OOM;
        break;
      }
      gst = launch_sketch_tc_grouped(items, buf, bytes, gs);
      cudaFreeAsync(buf, gs);
      for (Plan* p : ps) {
        cudaEventRecord(p->ev[1], gs);
        cudaStreamWaitEvent(p->stream, p->ev[1], 0);
        if (gst == LSRN_OK) {
          p->sketch_used = LSRN_SKETCH_TC_SLICED;
          p->state = 1;
        }
      }
      for (size_t k = k0; k < k1; ++k) st[grp[k]] = gst;
      k0 = k1;
    }
    for (size_t k = k0; k < grp.size(); ++k) st[grp[k]] = gst;   // after a failure
    if (gs) cudaStreamDestroy(gs);
  }
  lsrn_status first = LSRN_OK;
  for (int k = 0; k < count; ++k) {
    if (status) status[k] = st[k];
    if (first == LSRN_OK && st[k] != LSRN_OK) first = st[k];
  }
  return first;
}

lsrn_status lsrn_solve_batch(int32_t count, const lsrn_matrix* A, const double* const* b,
                             double* const* x, const lsrn_options* opt, int32_t solver,
                             int32_t threads, lsrn_info* info, int32_t* status) {
  if (count < 0 || threads < 0 || (solver != 0 && solver != 1)) return LSRN_ERR_INVALID_ARG;
  if (count == 0) return LSRN_OK;
  if (A == nullptr || b == nullptr || x == nullptr) return LSRN_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LSRN_ERR_CUDA;
  }
  const int nth = std::max(1, std::min<int>(threads > 0 ? threads : 8, count));
  std::vector<lsrn_plan_t> plans((size_t)count, nullptr);
  std::vector<lsrn_status> st((size_t)count, LSRN_OK);
  // 1. plans on the host threads, then the sketches: the exact tensor-core
  // sketches of small dense problems grouped into shared launches
  parallel_for(count, nth, dev, [&](int i) { st[i] = lsrn_plan(&A[i], opt, nullptr, &plans[i]); });
  {
    std::vector<lsrn_plan_t> ok;
    std::vector<int> idx;
    for (int i = 0; i < count; ++i)
      if (st[i] == LSRN_OK) {
        ok.push_back(plans[i]);
        idx.push_back(i);
      }
    std::vector<int32_t> gst(ok.size(), LSRN_OK);
    lsrn_sketch_group((int32_t)ok.size(), ok.data(), gst.data());
    for (size_t k = 0; k < idx.size(); ++k) st[idx[k]] = (lsrn_status)gst[k];
  }
  // 2. preconditioners: one launch for the small dense-sketch problems, largest first
  {
    std::vector<Plan*> ps;
    std::vector<int> idx;
    for (int i = 0; i < count; ++i)
      if (st[i] == LSRN_OK && precond_batchable(plans[i])) {
        ps.push_back(plans[i]);
        idx.push_back(i);
      }
    std::vector<lsrn_status> bst(ps.size(), LSRN_OK);
    precond_batch(ps, bst);
    for (size_t k = 0; k < idx.size(); ++k) st[idx[k]] = bst[k];
  }
  // 3. the other preconditioners and all iterations, overlapping across problems
  parallel_for(count, nth, dev, [&](int i) {
    if (st[i] == LSRN_OK) {
      lsrn_info inf;
      st[i] = solver == 1 ? lsrn_solve_cs(plans[i], b[i], x[i], &inf)
                          : lsrn_solve_lsqr(plans[i], b[i], x[i], &inf);
      if (info) info[i] = inf;
    } else if (info) {
      memset(&info[i], 0, sizeof(lsrn_info));
      info[i].status = st[i];
    }
    if (plans[i]) lsrn_plan_destroy(plans[i]);
  });
  lsrn_status first = LSRN_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (first == LSRN_OK && st[i] != LSRN_OK) first = st[i];
  }
  return first;
}

lsrn_status lsrn_plan_destroy(lsrn_plan_t p) {
  if (p == nullptr) return LSRN_OK;
  cudaSetDevice(p->device);
  release(p);
  return LSRN_OK;
}

lsrn_status lsrn_plan_get_sketch(lsrn_plan_t p, double* out, int64_t* rows, int64_t* cols) {
  if (p == nullptr) return LSRN_ERR_INVALID_ARG;
  if (p->state < 1) return LSRN_ERR_STATE;
  if (rows) *rows = p->s;
  if (cols) *cols = p->q;
  if (out) {
    LSRN_CUDA_TRY(cudaMemcpyAsync(out, p->Xs, p->s * p->q * sizeof(double), cudaMemcpyDefault,
                                  p->stream));
  }
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return LSRN_OK;
}

lsrn_status lsrn_plan_get_planes(lsrn_plan_t p, float* hi, float* lo, float* x3, int64_t* rows,
                                 int64_t* ld, double* scale) {
  if (p == nullptr) return LSRN_ERR_INVALID_ARG;
  if (p->X2h == nullptr || p->X2l == nullptr || p->X3 == nullptr) return LSRN_ERR_UNSUPPORTED;
  if (rows) *rows = p->xrows;
  if (ld) *ld = p->ldx2;
  if (scale) *scale = p->x2scale;
  const size_t bytes = (size_t)(p->xrows * p->ldx2) * sizeof(float);
  const float* src[3] = {p->X2h, p->X2l, p->X3};
  float* dst[3] = {hi, lo, x3};
  for (int k = 0; k < 3; ++k)
    if (dst[k]) LSRN_CUDA_TRY(cudaMemcpyAsync(dst[k], src[k], bytes, cudaMemcpyDefault, p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return LSRN_OK;
}

lsrn_status lsrn_plan_get_precond(lsrn_plan_t p, double* out, double* sigma, int64_t* rank) {
  if (p == nullptr) return LSRN_ERR_INVALID_ARG;
  if (p->state < 2) return LSRN_ERR_STATE;
  if (rank) *rank = p->rank;
  if (out && p->rank > 0)
    LSRN_CUDA_TRY(cudaMemcpyAsync(out, p->Nm, p->q * p->rank * sizeof(double), cudaMemcpyDefault,
                                  p->stream));
  if (sigma && p->rank > 0)
    LSRN_CUDA_TRY(cudaMemcpyAsync(sigma, p->sig, p->rank * sizeof(double), cudaMemcpyDefault,
                                  p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return LSRN_OK;
}

lsrn_status lsrn_generate_sketch_block(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0,
                                       int64_t rows, int64_t cols, double* g, float* z,
                                       void* stream) {
  if (rows < 0 || cols < 0 || i0 < 0 || j0 < 0) return LSRN_ERR_INVALID_ARG;
  if (i0 + rows > (int64_t)0xFFFFFFFFll) return LSRN_ERR_INVALID_ARG;
  if (rows * cols == 0) return LSRN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool gdev = g == nullptr || is_device_pointer(g);
  const bool zdev = z == nullptr || is_device_pointer(z);
  double* gd = g;
  float* zd = z;
  const size_t tot = (size_t)(rows * cols);
  if (g && !gdev) LSRN_CUDA_TRY(lsrn_malloc_async((void**)&gd, tot * sizeof(double), st));
  if (z && !zdev) LSRN_CUDA_TRY(lsrn_malloc_async((void**)&zd, tot * sizeof(float), st));
  lsrn_status res = launch_gamma_block(seed, tag, i0, j0, rows, cols, gd, zd, st);
  if (g && !gdev) {
    cudaMemcpyAsync(g, gd, tot * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(gd, st);
  }
  if (z && !zdev) {
    cudaMemcpyAsync(z, zd, tot * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(zd, st);
  }
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  return res;
}

}  // extern "C"
