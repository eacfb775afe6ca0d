// Sparse (CSR) operator: plan-time setup and the two passes that replace the
// dense fused pass (section 6.5: LSRN only uses A through products, so sparse
// A costs O(nnz) per product).
//
// X is the operator the passes stream (A for m >= n, A^T for m < n).  The plan
// keeps X by rows (rp/ci/cv) and by columns (rpT/ciT/cvT, i.e. the CSR of X^T);
// the column copy is built with a stable radix sort by column, so entries of a
// column are in row order and every sum below has a fixed order (results do not
// depend on scheduling).  One iteration's "fused pass" becomes
//   row pass:    d_i = X_i . vin, t_i = row coefficient (LSQR/CS state update)
//   column pass: out_c = sum_{i in column c} X[i, c] * t_i
// and the sketch C = Gamma^T X is formed column by column (k_sketch.cu).
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <vector>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

lsrn_status launch_row_coef_extra(const Plan* p, const double* vin, const RowArgs& a, double* out,
                                  double* pscal_slot, const int* done);

namespace {

// ---- setup --------------------------------------------------------------------
__global__ void csr_validate_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    int64_t m, int64_t n, int64_t nnz, int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || rp[m] != nnz)) atomicExch(bad, 1);
  if (i < m) {
    const int64_t a = rp[i], b = rp[i + 1];
    if (b < a || a < 0 || b > nnz) {
      atomicExch(bad, 1);
      return;
    }
    for (int64_t e = a; e < b; ++e)
      if (ci[e] < 0 || (int64_t)ci[e] >= n) {
        atomicExch(bad, 1);
        return;
      }
  }
}

__global__ void widen_kernel(const float* __restrict__ src, int64_t n, double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

__global__ void expand_rows_kernel(const int64_t* __restrict__ rp, int64_t m, int32_t* __restrict__ row,
                                   int32_t* __restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
    row[e] = (int32_t)i;
    idx[e] = (int32_t)e;
  }
}

// rpT[c] = first position k with key[k] >= c (keys sorted), rpT[ncol] = nnz
__global__ void col_ptr_kernel(const int32_t* __restrict__ keys, int64_t nnz, int64_t ncol,
                               int64_t* __restrict__ rpT) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > nnz) return;
  const int64_t prev = (k == 0) ? -1 : (int64_t)keys[k - 1];
  const int64_t cur = (k == nnz) ? ncol : (int64_t)keys[k];
  for (int64_t c = prev + 1; c <= cur; ++c) rpT[c] = k;
}

__global__ void gather_transpose_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ row,
                                        const double* __restrict__ val, int64_t nnz,
                                        int32_t* __restrict__ ciT, double* __restrict__ cvT) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int32_t e = perm[k];
  ciT[k] = row[e];
  cvT[k] = val[e];
}

// ---- passes ---------------------------------------------------------------------
template <int LANES>
__device__ __forceinline__ double lane_sum(double v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int LANES>
__device__ __forceinline__ void lane_sum_dd(double& h, double& l) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    const double oh = __shfl_xor_sync(0xffffffffu, h, o);
    const double ol = __shfl_xor_sync(0xffffffffu, l, o);
    dd_add(h, l, oh, ol);
  }
}

// Row pass over X's rows: d_i = X_i . vin, coefficient via the row mode; tout[i]
// receives the multiplier of X_i; per-block sum of squares into pscal.
template <int LANES>
__global__ void __launch_bounds__(256) csr_rowdot_kernel(const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci,
                                                         const double* __restrict__ cv, int64_t rows,
                                                         const double* __restrict__ vin, RowArgs args,
                                                         double* __restrict__ tout,
                                                         double* __restrict__ pscal,
                                                         const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ double sred[8];
  const int tid = threadIdx.x, lane = tid % LANES;
  constexpr int GPW = 32 / LANES;   // groups per warp; loops below are uniform per warp
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + tid) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) / 32;
  const bool need_dot = args.mode != RM_ACC_STATE;
  double c0 = 0.0, c1 = 0.0;
  if (args.coef) {
    c0 = args.coef[0];
    c1 = args.coef[1];
  }
  double ss = 0.0;
  for (int64_t wb = gw * GPW; wb < rows; wb += nw * GPW) {
    const int64_t i = wb + (tid & 31) / LANES;
    double d = 0.0;
    const bool live = i < rows;
    if (live && need_dot)
      for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += LANES) d = fma(cv[e], vin[ci[e]], d);
    d = lane_sum<LANES>(d);
    if (live && lane == 0) {
      double s0 = 0.0, s1 = 0.0;
      if (args.st0 != nullptr && args.mode != RM_APPLY) s0 = args.st0[i];
      if (args.mode == RM_FAT_CS) s1 = args.st1[i];
      double t = 0.0;
      switch (args.mode) {
        case RM_ACC_STATE: t = s0; break;
        case RM_LSQR_TALL: t = d - c0 * s0; args.st0[i] = t; ss = fma(t, t, ss); break;
        case RM_CS_TALL: t = s0 - c0 * d; args.st0[i] = t; ss = fma(t, t, ss); break;
        case RM_APPLY: t = d; break;
        case RM_FAT_INIT: t = args.sx * d; args.st0[i] = t; ss = fma(t, t, ss); t *= args.sx; break;
        case RM_FAT_LSQR:
          t = args.sx * d - c0 * s0; args.st0[i] = t; ss = fma(t, t, ss); t *= args.sx; break;
        case RM_FAT_CS:
          t = c0 * s0 + args.sx * d; args.st0[i] = t; args.st1[i] = fma(c1, t, s1); t *= args.sx;
          break;
      }
      tout[i] = t;
    }
  }
  ss = lane_sum<32>(ss);
  if ((tid & 31) == 0) sred[tid >> 5] = ss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sred[q];
    pscal[blockIdx.x] = t;
  }
}

// Column pass: out[c] = sum over column c of X of X[i, c] * t[i]  (fixed order).
template <int LANES>
__global__ void __launch_bounds__(256) csr_coldot_kernel(const int64_t* __restrict__ rpT,
                                                         const int32_t* __restrict__ ciT,
                                                         const double* __restrict__ cvT, int64_t cols,
                                                         const double* __restrict__ t,
                                                         double* __restrict__ out,
                                                         const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int tid = threadIdx.x, lane = tid % LANES;
  constexpr int GPW = 32 / LANES;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + tid) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) / 32;
  for (int64_t wb = gw * GPW; wb < cols; wb += nw * GPW) {
    const int64_t c = wb + (tid & 31) / LANES;
    double acc = 0.0;
    if (c < cols)
      for (int64_t e = rpT[c] + lane; e < rpT[c + 1]; e += LANES) acc = fma(cvT[e], t[ciT[e]], acc);
    acc = lane_sum<LANES>(acc);
    if (c < cols && lane == 0) out[c] = acc;
  }
}

// Double-double row pass (m >= n): r_i = b_i - X_i . x, rout[i] = r_i.
template <int LANES>
__global__ void __launch_bounds__(256) csr_rowdot_dd_kernel(const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const double* __restrict__ cv,
                                                            int64_t rows, const double* __restrict__ x,
                                                            const double* __restrict__ b,
                                                            double* __restrict__ rout) {
  const int tid = threadIdx.x, lane = tid % LANES;
  constexpr int GPW = 32 / LANES;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + tid) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) / 32;
  for (int64_t wb = gw * GPW; wb < rows; wb += nw * GPW) {
    const int64_t i = wb + (tid & 31) / LANES;
    double h = 0.0, l = 0.0;
    if (i < rows)
      for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += LANES) dd_add_prod(h, l, -cv[e], x[ci[e]]);
    lane_sum_dd<LANES>(h, l);
    if (i < rows && lane == 0) {
      dd_add(h, l, b[i], 0.0);
      rout[i] = h + l;
    }
  }
}

// Double-double column pass: (oh, ol)[c] = sum over column c of X[i, c] * (sc * t[i]).
template <int LANES>
__global__ void __launch_bounds__(256) csr_coldot_dd_kernel(const int64_t* __restrict__ rpT,
                                                            const int32_t* __restrict__ ciT,
                                                            const double* __restrict__ cvT,
                                                            int64_t cols, const double* __restrict__ t,
                                                            double sc, double* __restrict__ oh,
                                                            double* __restrict__ ol) {
  const int tid = threadIdx.x, lane = tid % LANES;
  constexpr int GPW = 32 / LANES;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + tid) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) / 32;
  for (int64_t wb = gw * GPW; wb < cols; wb += nw * GPW) {
    const int64_t c = wb + (tid & 31) / LANES;
    double h = 0.0, l = 0.0;
    if (c < cols)
      for (int64_t e = rpT[c] + lane; e < rpT[c + 1]; e += LANES) dd_add_prod(h, l, cvT[e], sc * t[ciT[e]]);
    lane_sum_dd<LANES>(h, l);
    if (c < cols && lane == 0) {
      oh[c] = h;
      ol[c] = l;
    }
  }
}

__global__ void sum_to_kernel(const double* __restrict__ part, int n, double* __restrict__ out,
                              const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

__global__ void fill_zero_kernel(double* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 0.0;
}

int lanes_for(int64_t nnz, int64_t rows) {
  const double avg = rows > 0 ? (double)nnz / (double)rows : 0.0;
  if (avg >= 24) return 32;
  if (avg >= 12) return 16;
  if (avg >= 6) return 8;
  return 4;
}

unsigned blocks_for(int64_t rows, int lanes) {
  const int64_t groups = 256 / lanes;
  const int64_t want = std::max<int64_t>(1, (rows + groups - 1) / groups);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 8 * (int64_t)num_sms()));
}

template <class F>
lsrn_status dispatch_lanes(int lanes, F f) {
  switch (lanes) {
    case 32: return f(std::integral_constant<int, 32>());
    case 16: return f(std::integral_constant<int, 16>());
    case 8: return f(std::integral_constant<int, 8>());
    default: return f(std::integral_constant<int, 4>());
  }
}

}  // namespace

// Build device copies of A (rows) and its transpose (columns), validate, and
// point the plan's X-by-rows / X-by-columns arrays at them.
lsrn_status csr_plan_setup(Plan* p, const lsrn_matrix* A, bool host) {
  if (A->row_ptr == nullptr || A->col_idx == nullptr || A->nnz < 0) return LSRN_ERR_INVALID_ARG;
  if (A->nnz > (int64_t)0x7FFFFFFF || A->m > (int64_t)0x7FFFFFFF || A->n > (int64_t)0x7FFFFFFF)
    return LSRN_ERR_UNSUPPORTED;
  cudaStream_t st = p->stream;
  const int64_t m = A->m, n = A->n, nnz = A->nnz;
  auto alloc = [&](void** ptr, size_t bytes) -> lsrn_status {
    *ptr = nullptr;
    cudaError_t e = lsrn_malloc_async(ptr, std::max<size_t>(bytes, 16), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? LSRN_ERR_OOM : LSRN_ERR_CUDA;
    }
    p->owned.push_back(*ptr);
    return LSRN_OK;
  };
  int64_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* cv = nullptr;
  LSRN_TRY(alloc((void**)&rp, (m + 1) * sizeof(int64_t)));
  LSRN_TRY(alloc((void**)&ci, nnz * sizeof(int32_t)));
  LSRN_TRY(alloc((void**)&cv, nnz * sizeof(double)));
  LSRN_CUDA_TRY(cudaMemcpyAsync(rp, A->row_ptr, (m + 1) * sizeof(int64_t), cudaMemcpyDefault, st));
  if (nnz) LSRN_CUDA_TRY(cudaMemcpyAsync(ci, A->col_idx, nnz * sizeof(int32_t), cudaMemcpyDefault, st));
  if (A->dtype == LSRN_F64) {
    if (nnz) LSRN_CUDA_TRY(cudaMemcpyAsync(cv, A->values, nnz * sizeof(double), cudaMemcpyDefault, st));
  } else if (nnz) {
    float* tmp = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&tmp, nnz * sizeof(float), st));
    LSRN_CUDA_TRY(cudaMemcpyAsync(tmp, A->values, nnz * sizeof(float), cudaMemcpyDefault, st));
    launch(widen_kernel, dim3((unsigned)((nnz + 255) / 256)), dim3(256), 0, st, (const float*)tmp, nnz, cv);
    cudaFreeAsync(tmp, st);
  }
  (void)host;
  // validate structure
  int* bad = nullptr;
  LSRN_CUDA_TRY(lsrn_malloc_async((void**)&bad, sizeof(int), st));
  LSRN_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
  launch(csr_validate_kernel, dim3((unsigned)((m + 255) / 256)), dim3(256), 0, st,
         (const int64_t*)rp, (const int32_t*)ci, m, n, nnz, bad);
  int hbad = 0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(bad, st);
  if (hbad) return LSRN_ERR_INVALID_ARG;
  // transpose: stable sort of entry indices by column
  int64_t* rpT = nullptr;
  int32_t* ciT = nullptr;
  double* cvT = nullptr;
  LSRN_TRY(alloc((void**)&rpT, (n + 1) * sizeof(int64_t)));
  LSRN_TRY(alloc((void**)&ciT, nnz * sizeof(int32_t)));
  LSRN_TRY(alloc((void**)&cvT, nnz * sizeof(double)));
  if (nnz > 0) {
    int32_t *row = nullptr, *idx = nullptr, *keys_out = nullptr, *perm = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&row, nnz * sizeof(int32_t), st));
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&idx, nnz * sizeof(int32_t), st));
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&keys_out, nnz * sizeof(int32_t), st));
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&perm, nnz * sizeof(int32_t), st));
    launch(expand_rows_kernel, dim3((unsigned)((m + 255) / 256)), dim3(256), 0, st,
           (const int64_t*)rp, m, row, idx);
    int end_bit = 1;
    while (end_bit < 32 && ((int64_t)1 << end_bit) <= n) ++end_bit;
    size_t temp = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, temp, (const int32_t*)ci, keys_out, (const int32_t*)idx,
                                    perm, (int)nnz, 0, end_bit, st);
    void* tbuf = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async(&tbuf, std::max<size_t>(temp, 16), st));
    LSRN_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tbuf, temp, (const int32_t*)ci, keys_out,
                                                  (const int32_t*)idx, perm, (int)nnz, 0, end_bit,
                                                  st));
    launch(col_ptr_kernel, dim3((unsigned)((nnz + 1 + 255) / 256)), dim3(256), 0, st,
           (const int32_t*)keys_out, nnz, n, rpT);
    launch(gather_transpose_kernel, dim3((unsigned)((nnz + 255) / 256)), dim3(256), 0, st,
           (const int32_t*)perm, (const int32_t*)row, (const double*)cv, nnz, ciT, cvT);
    cudaFreeAsync(tbuf, st);
    cudaFreeAsync(row, st);
    cudaFreeAsync(idx, st);
    cudaFreeAsync(keys_out, st);
    cudaFreeAsync(perm, st);
  } else {
    LSRN_CUDA_TRY(cudaMemsetAsync(rpT, 0, (n + 1) * sizeof(int64_t), st));
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  p->nnz = nnz;
  if (p->tall) {   // X = A
    p->rp = rp; p->ci = ci; p->cv = cv;
    p->rpT = rpT; p->ciT = ciT; p->cvT = cvT;
  } else {         // X = A^T: rows of X are columns of A
    p->rp = rpT; p->ci = ciT; p->cv = cvT;
    p->rpT = rp; p->ciT = ci; p->cvT = cv;
  }
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  return LSRN_OK;
}

// CSR version of the fused pass: out (xcols) = X^T t with t from the row pass,
// plus the ridge rows; sum of squares into scal_ss.
lsrn_status csr_fused_pass(const Plan* p, const double* vin, const RowArgs& a, double* out,
                           double* tbuf, double* scal_ss, const int* done) {
  const int lr = lanes_for(p->nnz, p->xrows);
  const unsigned br = blocks_for(p->xrows, lr);
  LSRN_TRY(dispatch_lanes(lr, [&](auto L) -> lsrn_status {
    launch(csr_rowdot_kernel<decltype(L)::value>, dim3(br), dim3(256), 0, p->stream, p->rp, p->ci,
           p->cv, p->xrows, vin, a, tbuf, p->pscal, done);
    return LSRN_OK;
  }));
  const int lc = lanes_for(p->nnz, p->xcols);
  const unsigned bc = blocks_for(p->xcols, lc);
  LSRN_TRY(dispatch_lanes(lc, [&](auto L) -> lsrn_status {
    launch(csr_coldot_kernel<decltype(L)::value>, dim3(bc), dim3(256), 0, p->stream, p->rpT, p->ciT,
           p->cvT, p->xcols, (const double*)tbuf, out, done);
    return LSRN_OK;
  }));
  int nparts = (int)br;
  if (p->extra_rows > 0) {
    LSRN_TRY(launch_row_coef_extra(p, vin, a, out, p->pscal + br, done));
    nparts += 1;
  }
  launch(sum_to_kernel, dim3(1), dim3(32), 0, p->stream, (const double*)p->pscal, nparts, scal_ss, done);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

// CSR version of the double-double pass, written into partial slot 0 of
// (phi, plo) with the other slots up to nblk zeroed (slot nblk: ridge rows).
lsrn_status csr_dd_pass(const Plan* p, const double* vin, const double* bvec, double* rout,
                        double* phi, double* plo, double* tbuf) {
  const int64_t C = p->xcols;
  launch(fill_zero_kernel, dim3(256), dim3(256), 0, p->stream, phi, (int64_t)p->nblk * C);
  launch(fill_zero_kernel, dim3(256), dim3(256), 0, p->stream, plo, (int64_t)p->nblk * C);
  const int lc = lanes_for(p->nnz, p->xcols);
  const unsigned bc = blocks_for(p->xcols, lc);
  if (bvec != nullptr) {   // m >= n: r = b - X x, then X^T r
    const int lr = lanes_for(p->nnz, p->xrows);
    const unsigned br = blocks_for(p->xrows, lr);
    LSRN_TRY(dispatch_lanes(lr, [&](auto L) -> lsrn_status {
      launch(csr_rowdot_dd_kernel<decltype(L)::value>, dim3(br), dim3(256), 0, p->stream, p->rp,
             p->ci, p->cv, p->xrows, vin, bvec, rout);
      return LSRN_OK;
    }));
    LSRN_TRY(dispatch_lanes(lc, [&](auto L) -> lsrn_status {
      launch(csr_coldot_dd_kernel<decltype(L)::value>, dim3(bc), dim3(256), 0, p->stream, p->rpT,
             p->ciT, p->cvT, p->xcols, (const double*)rout, 1.0, phi, plo);
      return LSRN_OK;
    }));
  } else {                 // m < n: B x = sum_j (sx x_j) X_j
    (void)tbuf;
    LSRN_TRY(dispatch_lanes(lc, [&](auto L) -> lsrn_status {
      launch(csr_coldot_dd_kernel<decltype(L)::value>, dim3(bc), dim3(256), 0, p->stream, p->rpT,
             p->ciT, p->cvT, p->xcols, vin, p->xscale, phi, plo);
      return LSRN_OK;
    }));
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
