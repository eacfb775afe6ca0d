// LSQR (Paige and Saunders 1982) and Chebyshev semi-iteration (Algorithm 3)
// on the preconditioned operator, driven from the host with all scalars kept on
// the device (no host round trip inside an iteration), plus the refinement
// step that follows them.
//
//   m >= n (Algorithm 1): operator B N on R^r, B = A or [A; lambda I]; the
//     iterate is y and x = N y (step 7).
//   m <  n (Algorithm 2): operator M^T B on R^{n'}, B = A or [A/lambda, I];
//     the iterate is x itself (x = z / lambda with ridge).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int kCtl = 1024;   // threads of the single-CTA control kernels

__device__ double block_sum_1024(double v, double* sh) {
  v = group_sum<32>(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kCtl / 32; ++w) t += sh[w];
  return t;
}

__global__ void sumsq_kernel(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(v[i], v[i], acc);
  acc = group_sum<32>(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

__global__ void fill_kernel(double* __restrict__ v, int64_t n, double val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = val;
}

__global__ void scale_copy_kernel(const double* __restrict__ src, int64_t n, double a,
                                  double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = a * src[i];
}

// v = c0*h + c1*v; z += c2*v      (c: device pointer)
__global__ void cheb_vec_kernel(const double* __restrict__ h, double* __restrict__ v,
                                double* __restrict__ z, int64_t n, const double* __restrict__ c) {
  const double c0 = c[0], c1 = c[1], c2 = c[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = fma(c0, h[i], c1 * v[i]);
    v[i] = vi;
    z[i] = fma(c2, vi, z[i]);
  }
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// ---- LSQR, m >= n -----------------------------------------------------------
// scal[SC_SS] = ||b||^2 on entry; tmpr = N^T B^T b.
__global__ void __launch_bounds__(kCtl) lsqr_tall_init_kernel(double* scal, int* isc,
                                                              const double* __restrict__ tmpr,
                                                              double* __restrict__ v,
                                                              double* __restrict__ w,
                                                              double* __restrict__ y, int64_t r) {
  __shared__ double sh[32];
  const double beta = sqrt(scal[SC_SS]);
  const double su = beta > 0.0 ? 1.0 / beta : 0.0;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) {
    const double vh = su * tmpr[k];
    acc = fma(vh, vh, acc);
  }
  const double alpha = sqrt(block_sum_1024(acc, sh));
  const double inv = alpha > 0.0 ? 1.0 / alpha : 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) {
    const double vk = su * tmpr[k] * inv;
    v[k] = vk;
    w[k] = vk;
    y[k] = 0.0;
  }
  if (threadIdx.x == 0) {
    scal[SC_BNORM] = beta;
    scal[SC_BETA] = beta;
    scal[SC_ALPHA] = alpha;
    scal[SC_SU] = su;
    scal[SC_CU] = alpha * su;
    scal[SC_PHIBAR] = beta;
    scal[SC_RHOBAR] = alpha;
    scal[SC_ANORM2] = 0.0;
    scal[SC_RNORM] = beta;
    scal[SC_ARNORM] = alpha * beta;
    isc[IC_ITN] = 0;
    const int exact = (alpha == 0.0 || beta == 0.0) ? 1 : 0;   // x = 0 is the solution
    isc[IC_ISTOP] = exact ? 3 : 0;
    isc[IC_DONE] = exact;
  }
}

// One LSQR step after the fused pass (t = B N v - alpha u, g = B^T t reduced,
// scal[SC_SS] = ||t||^2) and tmpr = N^T g.
__global__ void __launch_bounds__(kCtl) lsqr_tall_update_kernel(double* scal, int* isc,
                                                                const double* __restrict__ tmpr,
                                                                double* __restrict__ v,
                                                                double* __restrict__ w,
                                                                double* __restrict__ y, int64_t r,
                                                                double atol, double btol) {
  if (isc[IC_DONE]) return;
  __shared__ double sh[32];
  const double alpha = scal[SC_ALPHA];
  const double beta = sqrt(scal[SC_SS]);
  const double su = beta > 0.0 ? 1.0 / beta : 0.0;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) {
    const double vh = fma(su, tmpr[k], -beta * v[k]);
    acc = fma(vh, vh, acc);
  }
  const double alpha_new = sqrt(block_sum_1024(acc, sh));
  const double inv = alpha_new > 0.0 ? 1.0 / alpha_new : 0.0;
  const double rhobar = scal[SC_RHOBAR], phibar = scal[SC_PHIBAR];
  const double rho = hypot(rhobar, beta);
  const double c = rhobar / rho, s = beta / rho;
  const double theta = s * alpha_new;
  const double phi = c * phibar;
  const double cy = phi / rho, cw = theta / rho;
  double yacc = 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) {
    const double vk = fma(su, tmpr[k], -beta * v[k]) * inv;
    v[k] = vk;
    const double yk = fma(cy, w[k], y[k]);
    y[k] = yk;
    w[k] = fma(-cw, w[k], vk);
    yacc = fma(yk, yk, yacc);
  }
  const double ynorm = sqrt(block_sum_1024(yacc, sh));
  if (threadIdx.x == 0) {
    const double anorm2 = scal[SC_ANORM2] + alpha * alpha + beta * beta;
    const double phibar_new = s * phibar;
    const double rnorm = phibar_new;
    const double arnorm = phibar_new * alpha_new * fabs(c);
    const double anorm = sqrt(anorm2);
    const double bnorm = scal[SC_BNORM];
    scal[SC_ANORM2] = anorm2;
    scal[SC_RHOBAR] = -c * alpha_new;
    scal[SC_PHIBAR] = phibar_new;
    scal[SC_ALPHA] = alpha_new;
    scal[SC_BETA] = beta;
    scal[SC_SU] = su;
    scal[SC_CU] = alpha_new * su;
    scal[SC_RNORM] = rnorm;
    scal[SC_ARNORM] = arnorm;
    scal[SC_ANORM] = anorm;
    scal[SC_XNORM] = ynorm;
    const int itn = isc[IC_ITN] + 1;
    isc[IC_ITN] = itn;
    const double test1 = rnorm / bnorm;
    const double test2 = (anorm * rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
    const double rtol = btol + atol * anorm * ynorm / bnorm;
    int istop = 0;
    if (test1 <= rtol) istop = 1;
    else if (test2 <= atol) istop = 2;
    else if (alpha_new == 0.0 || beta == 0.0) istop = 3;
    isc[IC_ISTOP] = istop;
    if (istop != 0 || itn >= isc[IC_CAP]) isc[IC_DONE] = 1;
  }
}

// ---- LSQR, m < n ------------------------------------------------------------
// tmpr = M^T b: beta_1 = ||tmpr||, u = tmpr / beta_1.
__global__ void __launch_bounds__(kCtl) lsqr_fat_init_u_kernel(double* scal, int* isc,
                                                               const double* __restrict__ tmpr,
                                                               double* __restrict__ u, int64_t r) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) acc = fma(tmpr[k], tmpr[k], acc);
  const double beta = sqrt(block_sum_1024(acc, sh));
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) u[k] = tmpr[k] * inv;
  if (threadIdx.x == 0) {
    scal[SC_BNORM] = beta;
    scal[SC_BETA] = beta;
    scal[SC_PHIBAR] = beta;
    scal[SC_ANORM2] = 0.0;
    scal[SC_RNORM] = beta;
    isc[IC_ITN] = 0;
    isc[IC_ISTOP] = beta == 0.0 ? 3 : 0;
    isc[IC_DONE] = beta == 0.0 ? 1 : 0;
  }
}

// After the first pass: scal[SC_SS] = ||vhat||^2 -> alpha_1, sv = 1/alpha_1.
__global__ void lsqr_fat_init_alpha_kernel(double* scal, int* isc) {
  if (threadIdx.x != 0) return;
  const double alpha = sqrt(scal[SC_SS]);
  scal[SC_ALPHA] = alpha;
  scal[SC_SU] = alpha > 0.0 ? 1.0 / alpha : 0.0;
  scal[SC_RHOBAR] = alpha;
  scal[SC_ARNORM] = alpha * scal[SC_BETA];
  if (alpha == 0.0 && !isc[IC_DONE]) {
    isc[IC_DONE] = 1;
    isc[IC_ISTOP] = 3;
  }
}

// uhat = sv * tmpr - alpha u; beta = ||uhat||; u = uhat / beta; coefficient
// for the pass c0 = beta * sv.
__global__ void __launch_bounds__(kCtl) lsqr_fat_u_kernel(double* scal, int* isc,
                                                          const double* __restrict__ tmpr,
                                                          double* __restrict__ u, int64_t r) {
  if (isc[IC_DONE]) return;
  __shared__ double sh[32];
  const double alpha = scal[SC_ALPHA], sv = scal[SC_SU];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) {
    const double uh = fma(sv, tmpr[k], -alpha * u[k]);
    acc = fma(uh, uh, acc);
  }
  const double beta = sqrt(block_sum_1024(acc, sh));
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int64_t k = threadIdx.x; k < r; k += kCtl) u[k] = fma(sv, tmpr[k], -alpha * u[k]) * inv;
  if (threadIdx.x == 0) {
    scal[SC_BETA] = beta;
    scal[SC_ANORM2] += alpha * alpha + beta * beta;
    scal[SC_CU] = beta * sv;
  }
}

// Scalar part of the step after the second pass (scal[SC_SS] = ||vhat||^2).
__global__ void lsqr_fat_scalar_kernel(double* scal, const int* isc) {
  if (isc[IC_DONE] || threadIdx.x != 0) return;
  const double beta = scal[SC_BETA];
  const double alpha_new = sqrt(scal[SC_SS]);
  const double rhobar = scal[SC_RHOBAR], phibar = scal[SC_PHIBAR];
  const double rho = hypot(rhobar, beta);
  const double c = rhobar / rho, s = beta / rho;
  const double theta = s * alpha_new;
  const double phi = c * phibar;
  scal[SC_CX] = phi / rho;
  scal[SC_CW] = theta / rho;
  scal[SC_RHOBAR] = -c * alpha_new;
  scal[SC_PHIBAR] = s * phibar;
  scal[SC_RNORM] = s * phibar;
  scal[SC_ARNORM] = s * phibar * alpha_new * fabs(c);
  scal[SC_ANORM] = sqrt(scal[SC_ANORM2]);
  scal[SC_ALPHA_NEW] = alpha_new;
  scal[SC_SV_NEW] = alpha_new > 0.0 ? 1.0 / alpha_new : 0.0;
}

// x += cx w; w = vhat * sv_new - cw w; partial ||x||^2.
__global__ void __launch_bounds__(256) lsqr_fat_vec_kernel(const double* scal, const int* isc,
                                                           double* __restrict__ x,
                                                           double* __restrict__ w,
                                                           const double* __restrict__ vhat,
                                                           int64_t n, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  if (!isc[IC_DONE]) {
    const double cx = scal[SC_CX], cw = scal[SC_CW], sv = scal[SC_SV_NEW];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double xi = fma(cx, w[i], x[i]);
      x[i] = xi;
      w[i] = fma(-cw, w[i], vhat[i] * sv);
      acc = fma(xi, xi, acc);
    }
  }
  acc = group_sum<32>(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    part[blockIdx.x] = t;
  }
}

__global__ void lsqr_fat_test_kernel(double* scal, int* isc, const double* __restrict__ part,
                                     int nparts, double atol, double btol) {
  if (isc[IC_DONE] || threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nparts; ++i) t += part[i];
  const double xnorm = sqrt(t);
  const double rnorm = scal[SC_RNORM], arnorm = scal[SC_ARNORM], anorm = scal[SC_ANORM];
  const double bnorm = scal[SC_BNORM];
  const double alpha_new = scal[SC_ALPHA_NEW], beta = scal[SC_BETA];
  scal[SC_XNORM] = xnorm;
  scal[SC_ALPHA] = alpha_new;
  scal[SC_SU] = scal[SC_SV_NEW];
  const int itn = isc[IC_ITN] + 1;
  isc[IC_ITN] = itn;
  const double test1 = rnorm / bnorm;
  const double test2 = (anorm * rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
  const double rtol = btol + atol * anorm * xnorm / bnorm;
  int istop = 0;
  if (test1 <= rtol) istop = 1;
  else if (test2 <= atol) istop = 2;
  else if (alpha_new == 0.0 || beta == 0.0) istop = 3;
  isc[IC_ISTOP] = istop;
  if (istop != 0 || itn >= isc[IC_CAP]) isc[IC_DONE] = 1;
}

// r = b - (qh + ql) in double-double, rounded.
__global__ void resid_dd_kernel(const double* __restrict__ b, const double* __restrict__ qh,
                                const double* __restrict__ ql, int64_t m, double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    double h = b[i], l = 0.0;
    dd_add(h, l, -qh[i], -ql[i]);
    r[i] = h + l;
  }
}

inline unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * num_sms()));
}

}  // namespace

// partial sums of ||a - b||^2 (part[2k]) and ||b||^2 (part[2k+1])
__global__ void diffnorm_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                double* __restrict__ part) {
  __shared__ double s1[8], s2[8];
  double d2 = 0.0, b2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = a[i] - b[i];
    d2 = fma(d, d, d2);
    b2 = fma(b[i], b[i], b2);
  }
  d2 = group_sum<32>(d2);
  b2 = group_sum<32>(b2);
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = d2;
    s2[threadIdx.x >> 5] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      t1 += s1[w];
      t2 += s2[w];
    }
    part[2 * blockIdx.x] = t1;
    part[2 * blockIdx.x + 1] = t2;
  }
}

// ---- helpers used by the host drivers --------------------------------------
// ||a - b|| / ||b|| (synchronises)
// ||a - b|| / ||b||; with long_side set, a and b are a shard's block of a
// vector over the long side and the sums run over all shards.
static lsrn_status rel_change(Plan* p, const double* a, const double* b, int64_t n, double* out,
                              bool long_side = false) {
  const int parts = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 64);
  launch(diffnorm_kernel, dim3(parts), dim3(256), 0, p->stream, a, b, n, p->pscal);
  double host[128];
  LSRN_CUDA_TRY(cudaMemcpyAsync(host, p->pscal, 2 * parts * sizeof(double), cudaMemcpyDeviceToHost,
                                p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  double d[2] = {0.0, 0.0};
  for (int i = 0; i < parts; ++i) {
    d[0] += host[2 * i];
    d[1] += host[2 * i + 1];
  }
  if (long_side && p->sharded) {
    LSRN_CUDA_TRY(cudaMemcpyAsync(p->pscal, d, sizeof(d), cudaMemcpyHostToDevice, p->stream));
    LSRN_TRY(shard_sum(p, p->pscal, 2));
    LSRN_CUDA_TRY(cudaMemcpyAsync(d, p->pscal, sizeof(d), cudaMemcpyDeviceToHost, p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  }
  const double d2 = d[0], b2 = d[1];
  *out = b2 > 0.0 ? std::sqrt(d2 / b2) : (d2 > 0.0 ? 1.0 : 0.0);
  return LSRN_OK;
}
static lsrn_status sumsq(Plan* p, const double* v, int64_t n, double* out) {
  const int parts = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 2 * num_sms());
  launch(sumsq_kernel, parts, 256, 0, p->stream, v, n, p->pscal);
  launch(sum_parts_kernel, 1, 32, 0, p->stream, p->pscal, parts, out);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

static lsrn_status fill(Plan* p, double* v, int64_t n, double val) {
  if (n <= 0) return LSRN_OK;
  launch(fill_kernel, grid_for(n), 256, 0, p->stream, v, n, val);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

// One fused pass (+ ridge rows) and its reduction into out (C) and scal[SC_SS].
static lsrn_status fused_pass_local(Plan* p, const double* vin, const RowArgs& a, double* out,
                                    const int* done) {
  if (p->csr) return csr_fused_pass(p, vin, a, out, p->tcsr, p->scal + SC_SS, done);
  if (p->is_op) {
    LSRN_TRY(op_row_pass(p, vin, a, p->pvec, p->pscal, done));
    LSRN_TRY(launch_extra_rows(p, vin, a, p->pvec, p->pscal, done));
    const int nslots = p->nblk + (p->extra_rows > 0 ? 1 : 0);
    return launch_reduce(p->pvec, nslots, p->xcols, out, p->pscal, p->scal + SC_SS, done, p->stream);
  }
  if (p->time_passes) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, p->stream);
    LSRN_TRY(launch_row_pass(p, vin, a, p->pvec, p->pscal, done));
    cudaEventRecord(e1, p->stream);
    p->pass_events.emplace_back(e0, e1);
  } else {
    LSRN_TRY(launch_row_pass(p, vin, a, p->pvec, p->pscal, done));
  }
  LSRN_TRY(launch_extra_rows(p, vin, a, p->pvec, p->pscal, done));
  const int nslots = p->nblk + (p->extra_rows > 0 ? 1 : 0);
  return launch_reduce(p->pvec, nslots, p->xcols, out, p->pscal, p->scal + SC_SS, done, p->stream);
}

// The pass, and for a shard the sum over shards of its column vector and its
// sum of squares (one exchange of q + 1 values; out has room for q + 2).
static lsrn_status fused_pass(Plan* p, const double* vin, const RowArgs& a, double* out,
                              const int* done) {
  LSRN_TRY(fused_pass_local(p, vin, a, out, done));
  if (!p->sharded) return LSRN_OK;
  if (done != nullptr) {   // after convergence the pass wrote nothing: nothing to exchange
    int d = 0;             // (the flag is the same on every shard: identical recurrences)
    LSRN_CUDA_TRY(cudaMemcpyAsync(&d, done, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (d != 0) return LSRN_OK;
  }
  const int64_t C = p->xcols;
  LSRN_CUDA_TRY(cudaMemcpyAsync(out + C, p->scal + SC_SS, sizeof(double), cudaMemcpyDeviceToDevice,
                                p->stream));
  LSRN_TRY(shard_sum(p, out, C + 1));
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->scal + SC_SS, out + C, sizeof(double), cudaMemcpyDeviceToDevice,
                                p->stream));
  return LSRN_OK;
}

// shard_sum, skipped once the device `done` flag is set (the same on every shard)
static lsrn_status shard_sum_unless_done(Plan* p, double* buf, int64_t count, const int* done) {
  if (!p->sharded) return LSRN_OK;
  if (done != nullptr) {
    int d = 0;
    LSRN_CUDA_TRY(cudaMemcpyAsync(&d, done, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (d != 0) return LSRN_OK;
  }
  return shard_sum(p, buf, count);
}

// ||v||^2 of a vector over the long side (b): summed over the shards.
static lsrn_status sumsq_long(Plan* p, const double* v, int64_t n, double* out) {
  LSRN_TRY(sumsq(p, v, n, out));
  return shard_sum(p, out, 1);
}

static const double* c100(Plan* p) { return p->scal + SC_ONE; }   // (1, 0, 0)

// Run `body` for each iteration until the device done flag is set or `cap`
// steps have been issued; the flag is read back every `batch` steps.
// Small problems (at most kGraphIterElems entries of X) replay the batch of
// `batch` steps from a CUDA graph captured once: the same kernels with the same
// device-resident arguments every batch, one launch instead of ~5 per step
// (launch throughput, not the GPU, bounds such problems).  Their passes are then
// not timed one by one.  Sharded and operator plans call back to the host
// inside a step and are never captured.
constexpr int64_t kGraphIterElems = (int64_t)1 << 25;

static bool capture_iterations(const Plan* p) {
  return !p->sharded && !p->is_op && p->xrows * p->xcols <= kGraphIterElems;
}

template <class F>
static lsrn_status iterate(Plan* p, int cap, F body) {
  const int batch = 8;
  int issued = 0;
  int done = 0;
  cudaGraphExec_t g = nullptr;
  unsigned long long nodes = 0;
  if (capture_iterations(p) && cap >= batch) {
    p->time_passes = false;
    lsrn_status cst = LSRN_OK;
    g = capture_graph(p->stream, [&]() {
      for (int i = 0; i < batch && cst == LSRN_OK; ++i) cst = body();
    }, &nodes);
    if (cst != LSRN_OK && g != nullptr) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  }
  while (issued < cap && !done) {
    const int nb = std::min(batch, cap - issued);
    if (g != nullptr && nb == batch) {
      LSRN_CUDA_TRY(cudaGraphLaunch(g, p->stream));
      g_kernel_launches.fetch_add(nodes, std::memory_order_relaxed);
    } else {
      for (int i = 0; i < nb; ++i) LSRN_TRY(body());
    }
    issued += nb;
    LSRN_CUDA_TRY(cudaMemcpyAsync(&done, p->iscal + IC_DONE, sizeof(int), cudaMemcpyDeviceToHost,
                                  p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  }
  if (g != nullptr) cudaGraphExecDestroy(g);
  return LSRN_OK;
}

// Tolerance of the main sweep: the option, or a looser one when refinement
// (at least two steps, each contracting the error by ~refine_tol) follows
// anyway: the FP32 floor in FP32 mode, 1e-8 in double-float mode for m >= n.
// (For m < n the correction by CS on M^T B contracts less per step, so the
// sweep keeps tol.)
static double sweep_tol(const Plan* p) {
  if (p->X32 != nullptr) return std::max(p->opt.tol, 1e-6);
  if (p->X2h != nullptr && p->tall && p->opt.refine_max > 0) return std::max(p->opt.tol, 1e-8);
  return p->opt.tol;
}

static int lsqr_cap(const Plan* p) {
  if (p->opt.max_iter >= 0) return std::max(1, p->opt.max_iter);
  const double rs = (double)p->rank / (double)p->s;
  const double bound = (std::log(sweep_tol(p)) - std::log(2.0)) / std::log(std::sqrt(rs));
  return std::max(1, (int)std::ceil(1.5 * bound));
}

// Chebyshev coefficient blocks (8 doubles per step):
//   [1, beta, alpha, beta, alpha, -alpha, 1, 0]
static std::vector<double> cheb_table(double sL, double sU, double tol, int* steps) {
  const double d = 0.5 * (sU * sU + sL * sL);
  const double c = 0.5 * (sU * sU - sL * sL);
  const double rho = (sU - sL) / (sU + sL);
  int K = 0;
  if (rho > 0.0) K = (int)std::ceil((std::log(tol) - std::log(2.0)) / std::log(rho));
  K = std::max(K, 0);
  std::vector<double> t((size_t)(K + 1) * 8);
  double alpha = 0.0;
  for (int k = 0; k <= K; ++k) {
    double beta;
    if (k == 0) {
      beta = 0.0;
      alpha = 1.0 / d;
    } else if (k == 1) {
      beta = 0.5 * (c / d) * (c / d);
      alpha = 1.0 / (d - c * c / (2.0 * d));
    } else {
      beta = (alpha * c / 2.0) * (alpha * c / 2.0);
      alpha = 1.0 / (d - alpha * c * c / 4.0);
    }
    double* e = &t[(size_t)k * 8];
    e[0] = 1.0; e[1] = beta; e[2] = alpha; e[3] = beta; e[4] = alpha; e[5] = -alpha; e[6] = 1.0; e[7] = 0.0;
  }
  *steps = K + 1;
  return t;
}

lsrn_status thm45_bounds(const Plan* p, double* sL, double* sU) {
  const double s = (double)p->s, r = (double)p->rank;
  const double a = p->opt.cs_alpha >= 0.0 ? p->opt.cs_alpha : 1.0 / std::sqrt(s);
  const double lo = (1.0 - a) * std::sqrt(s) - std::sqrt(r);
  if (!(lo > 0.0)) return LSRN_ERR_INVALID_ARG;
  *sU = 1.0 / lo;
  *sL = 1.0 / ((1.0 + a) * std::sqrt(s) + std::sqrt(r));
  // a BF16 preconditioner: sigma(AN) may leave the bounds by its noise floor
  *sU *= 1.0 + p->bound_widen;
  *sL *= 1.0 - p->bound_widen;
  return LSRN_OK;
}

static lsrn_status upload_coefs(Plan* p, const std::vector<double>& t) {
  if ((int64_t)t.size() > p->ncoef) {
    if (p->coefs) cudaFreeAsync(p->coefs, p->stream);
    p->coefs = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&p->coefs, t.size() * sizeof(double), p->stream));
    p->ncoef = (int64_t)t.size();
  }
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->coefs, t.data(), t.size() * sizeof(double),
                                cudaMemcpyHostToDevice, p->stream));
  // the table must outlive this call: wait for the copy
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return LSRN_OK;
}

// ---- drivers ---------------------------------------------------------------
// Vectors: vr[0] v, vr[1] w, vr[2] y, vr[3] tmpr/h, vr[4] z, vr[5] u (fat) / rho.

lsrn_status run_lsqr(Plan* p, int* iters, int* istop) {
  const int64_t r = p->rank, q = p->q;
  const double tol = sweep_tol(p);
  p->pass_f32 = p->X32 != nullptr;
  double* v = p->vr[0];
  double* w = p->vr[1];
  double* y = p->vr[2];
  double* tmpr = p->vr[3];
  int cap = lsqr_cap(p);
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->iscal + IC_CAP, &cap, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  const int* done = p->iscal + IC_DONE;
  if (p->tall) {
    // u state = b (rows m) and zeros for the ridge rows; ||b||^2.
    LSRN_CUDA_TRY(cudaMemcpyAsync(p->st0, p->bdev, p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    LSRN_TRY(fill(p, p->st0 + p->m, p->nstate - p->m, 0.0));
    RowArgs a0{RM_ACC_STATE, p->st0, nullptr, nullptr, 1.0};
    LSRN_TRY(fused_pass(p, nullptr, a0, p->vq, nullptr));
    LSRN_TRY(sumsq_long(p, p->bdev, p->m, p->scal + SC_SS));   // the pass overwrote SC_SS
    LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, tmpr, nullptr, nullptr, c100(p), nullptr, p->stream));
    launch(lsqr_tall_init_kernel, 1, kCtl, 0, p->stream, p->scal, p->iscal, tmpr, v, w, y, r);
    LSRN_CUDA_TRY(cudaGetLastError());
    RowArgs a{RM_LSQR_TALL, p->st0, nullptr, p->scal + SC_CU, 1.0};
    LSRN_TRY(iterate(p, cap, [&]() -> lsrn_status {
      LSRN_TRY(launch_gemv(p->Nm, q, r, v, p->tmpq, nullptr, nullptr, c100(p), done, p->stream));
      LSRN_TRY(fused_pass(p, p->tmpq, a, p->vq, done));
      LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, tmpr, nullptr, nullptr, c100(p), done, p->stream));
      launch(lsqr_tall_update_kernel, 1, kCtl, 0, p->stream, p->scal, p->iscal, tmpr, v, w, y, r, tol, tol);
      LSRN_CUDA_TRY(cudaGetLastError());
      return LSRN_OK;
    }));
  } else {
    double* u = p->vr[5];
    double* vhat = p->st0;
    double* x = p->st1;
    double* wv = p->xfull;
    const int64_t ns = p->nstate;
    LSRN_TRY(launch_gemv(p->NT, r, q, p->bdev, tmpr, nullptr, nullptr, c100(p), nullptr, p->stream));
    launch(lsqr_fat_init_u_kernel, 1, kCtl, 0, p->stream, p->scal, p->iscal, tmpr, u, r);
    LSRN_TRY(launch_gemv(p->Nm, q, r, u, p->vq2, nullptr, nullptr, c100(p), nullptr, p->stream));
    RowArgs a0{RM_FAT_INIT, vhat, nullptr, nullptr, p->xscale};
    LSRN_TRY(fused_pass(p, p->vq2, a0, p->vq, nullptr));
    launch(lsqr_fat_init_alpha_kernel, 1, 32, 0, p->stream, p->scal, p->iscal);
    LSRN_TRY(fill(p, x, ns, 0.0));
    // w = vhat * sv
    double sv_host = 0.0;
    LSRN_CUDA_TRY(cudaMemcpyAsync(&sv_host, p->scal + SC_SU, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    launch(scale_copy_kernel, grid_for(ns), 256, 0, p->stream, vhat, ns, sv_host, wv);
    LSRN_CUDA_TRY(cudaGetLastError());
    const int nparts = (int)grid_for(ns);
    RowArgs a{RM_FAT_LSQR, vhat, nullptr, p->scal + SC_CU, p->xscale};
    LSRN_TRY(iterate(p, cap, [&]() -> lsrn_status {
      LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, tmpr, nullptr, nullptr, c100(p), done, p->stream));
      launch(lsqr_fat_u_kernel, 1, kCtl, 0, p->stream, p->scal, p->iscal, tmpr, u, r);
      LSRN_TRY(launch_gemv(p->Nm, q, r, u, p->vq2, nullptr, nullptr, c100(p), done, p->stream));
      LSRN_TRY(fused_pass(p, p->vq2, a, p->vq, done));
      launch(lsqr_fat_scalar_kernel, 1, 32, 0, p->stream, p->scal, p->iscal);
      launch(lsqr_fat_vec_kernel, nparts, 256, 0, p->stream, p->scal, p->iscal, x, wv, vhat, ns, p->pscal);
      if (p->sharded) {   // ||x||^2 over all shards' blocks of x
        launch(sum_parts_kernel, 1, 32, 0, p->stream, (const double*)p->pscal, nparts,
               p->pscal + nparts);
        LSRN_TRY(shard_sum_unless_done(p, p->pscal + nparts, 1, done));
        launch(lsqr_fat_test_kernel, 1, 32, 0, p->stream, p->scal, p->iscal,
               (const double*)(p->pscal + nparts), 1, tol, tol);
      } else {
        launch(lsqr_fat_test_kernel, 1, 32, 0, p->stream, p->scal, p->iscal, p->pscal, nparts, tol, tol);
      }
      LSRN_CUDA_TRY(cudaGetLastError());
      return LSRN_OK;
    }));
  }
  int isc[IC_COUNT];
  LSRN_CUDA_TRY(cudaMemcpyAsync(isc, p->iscal, sizeof(isc), cudaMemcpyDeviceToHost, p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  *iters = isc[IC_ITN];
  *istop = isc[IC_ISTOP];
  return LSRN_OK;
}

lsrn_status run_cs(Plan* p, int* iters, double* sL_out, double* sU_out, bool* diverged) {
  const int64_t r = p->rank, q = p->q;
  double sL, sU;
  LSRN_TRY(thm45_bounds(p, &sL, &sU));
  *sL_out = sL;
  *sU_out = sU;
  int steps = 0;
  LSRN_TRY(upload_coefs(p, cheb_table(sL, sU, sweep_tol(p), &steps)));
  *iters = steps;
  p->pass_f32 = p->X32 != nullptr;
  double ss0 = 0.0, ss1 = 0.0;
  if (p->tall) {
    double* v = p->vr[0];
    double* y = p->vr[2];
    LSRN_CUDA_TRY(cudaMemcpyAsync(p->st0, p->bdev, p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    LSRN_TRY(fill(p, p->st0 + p->m, p->nstate - p->m, 0.0));
    LSRN_TRY(sumsq_long(p, p->bdev, p->m, p->scal + SC_SS0));
    RowArgs a0{RM_ACC_STATE, p->st0, nullptr, nullptr, 1.0};
    LSRN_TRY(fused_pass(p, nullptr, a0, p->vq, nullptr));
    LSRN_TRY(fill(p, v, r, 0.0));
    LSRN_TRY(fill(p, y, r, 0.0));
    for (int k = 0; k < steps; ++k) {
      const double* blk = p->coefs + (int64_t)k * 8;
      LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, v, v, y, blk + 0, nullptr, p->stream));
      LSRN_TRY(launch_gemv(p->Nm, q, r, v, p->tmpq, nullptr, nullptr, c100(p), nullptr, p->stream));
      RowArgs a{RM_CS_TALL, p->st0, nullptr, blk + 2, 1.0};
      LSRN_TRY(fused_pass(p, p->tmpq, a, p->vq, nullptr));
    }
  } else {
    double* rho = p->vr[5];
    double* v = p->st0;
    double* x = p->st1;
    LSRN_TRY(launch_gemv(p->NT, r, q, p->bdev, rho, nullptr, nullptr, c100(p), nullptr, p->stream));
    LSRN_TRY(sumsq(p, rho, r, p->scal + SC_SS0));
    LSRN_TRY(fill(p, v, p->nstate, 0.0));
    LSRN_TRY(fill(p, x, p->nstate, 0.0));
    for (int k = 0; k < steps; ++k) {
      const double* blk = p->coefs + (int64_t)k * 8;
      LSRN_TRY(launch_gemv(p->Nm, q, r, rho, p->vq2, nullptr, nullptr, c100(p), nullptr, p->stream));
      RowArgs a{RM_FAT_CS, v, x, blk + 3, p->xscale};
      LSRN_TRY(fused_pass(p, p->vq2, a, p->vq, nullptr));
      LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, rho, rho, nullptr, blk + 5, nullptr, p->stream));
    }
    LSRN_TRY(sumsq(p, rho, r, p->scal + SC_SS));
  }
  LSRN_CUDA_TRY(cudaMemcpyAsync(&ss0, p->scal + SC_SS0, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  LSRN_CUDA_TRY(cudaMemcpyAsync(&ss1, p->scal + SC_SS, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  *diverged = !(ss1 <= ss0 * (1.0 + 1e-9)) || !std::isfinite(ss1);
  return LSRN_OK;
}

// Refinement after the iteration (see lsrn.h).  m >= n: x = N y is formed,
// r = b - B x and g = B^T r in double-double, then K z = N^T g with
// K = N^T B^T B N by Algorithm 3's recurrence, y += z.  m < n: r = b - B x in
// double-double, then Algorithm 3 on min ||M^T B d - M^T r||, x += d.
lsrn_status run_refine(Plan* p, int nsteps, int* inner, int* taken) {
  *inner = 0;
  *taken = 0;
  // With an FP32 copy of A, correction passes start in FP32 and switch to FP64
  // for the remaining steps once a step contracts the change by less than 20x
  // (FP32 rounding of A perturbs the preconditioned operator by ~u32 kappa(A)).
  if (p->X32 != nullptr) nsteps = std::max(nsteps, 6);
  // Double-float passes perturb A by ~2^-46 relative, so with a nonzero
  // residual a step contracts by ~kappa^2 2^-46 |r| / (|A||x|): two steps at least.
  if (p->X2h != nullptr && nsteps > 0) nsteps = std::max(nsteps, 2);
  if (nsteps <= 0 || p->rank == 0 || p->is_op) return LSRN_OK;   // operator plans: no refinement
  p->pass_f32 = p->X32 != nullptr;
  double prev_change = 1.0;
  const int64_t r = p->rank, q = p->q;
  double sL, sU;
  if (thm45_bounds(p, &sL, &sU) != LSRN_OK) return LSRN_OK;   // no bounds: skip refinement
  int steps = 0;
  LSRN_TRY(upload_coefs(p, cheb_table(sL, sU, p->opt.refine_tol, &steps)));
  const int nslots = p->nblk + (p->extra_rows ? 1 : 0);
  // The device work of one step (everything but the host read of the change),
  // the same kernels with the same arguments every step: small problems replay
  // it from a CUDA graph, captured again only when the pass precision switches.
  auto step_kernels = [&]() -> lsrn_status {
    if (p->tall) {
      double* y = p->vr[2];
      double* h = p->vr[3];
      double* z = p->vr[4];
      double* v = p->vr[0];
      double* x = p->xfull;
      LSRN_TRY(launch_gemv_dd(p->Nm, q, r, y, x, p->stream));
      LSRN_TRY(launch_dd_pass(p, x, p->bdev, p->st1, p->pvec, p->pvec2, nullptr));
      LSRN_TRY(launch_reduce_dd(p->pvec, p->pvec2, nslots, q, p->vq, p->vq2, p->stream));
      LSRN_TRY(shard_sum_dd(p, p->vq, p->vq2, q));
      // g = hi + lo
      launch(axpy_kernel, grid_for(q), 256, 0, p->stream, p->vq, p->vq2, q, 1.0);
      LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, h, nullptr, nullptr, c100(p), nullptr, p->stream));
      LSRN_TRY(fill(p, v, r, 0.0));
      LSRN_TRY(fill(p, z, r, 0.0));
      RowArgs a{RM_APPLY, nullptr, nullptr, nullptr, 1.0};
      for (int k = 0; k < steps; ++k) {
        const double* blk = p->coefs + (int64_t)k * 8;
        launch(cheb_vec_kernel, grid_for(r), 256, 0, p->stream, h, v, z, r, blk + 0);
        LSRN_TRY(launch_gemv(p->Nm, q, r, v, p->tmpq, nullptr, nullptr, c100(p), nullptr, p->stream));
        LSRN_TRY(fused_pass(p, p->tmpq, a, p->vq, nullptr));
        LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, h, h, nullptr, blk + 5, nullptr, p->stream));
      }
      launch(axpy_kernel, grid_for(r), 256, 0, p->stream, y, z, r, 1.0);
      // x = N y after the step, compared with x before it
      LSRN_TRY(launch_gemv_dd(p->Nm, q, r, y, p->tmpq, p->stream));
    } else {
      double* rho = p->vr[5];
      double* v = p->st0;
      double* x = p->st1;
      LSRN_TRY(launch_dd_pass(p, x, nullptr, nullptr, p->pvec, p->pvec2, nullptr));
      LSRN_TRY(launch_reduce_dd(p->pvec, p->pvec2, nslots, q, p->vq, p->vq2, p->stream));
      LSRN_TRY(shard_sum_dd(p, p->vq, p->vq2, q));
      launch(resid_dd_kernel, grid_for(q), 256, 0, p->stream, p->bdev, p->vq, p->vq2, q, p->tmpq);
      LSRN_TRY(launch_gemv(p->NT, r, q, p->tmpq, rho, nullptr, nullptr, c100(p), nullptr, p->stream));
      LSRN_TRY(fill(p, v, p->nstate, 0.0));
      LSRN_CUDA_TRY(cudaMemcpyAsync(p->xfull, x, p->nstate * sizeof(double),
                                    cudaMemcpyDeviceToDevice, p->stream));
      for (int k = 0; k < steps; ++k) {
        const double* blk = p->coefs + (int64_t)k * 8;
        LSRN_TRY(launch_gemv(p->Nm, q, r, rho, p->vq2, nullptr, nullptr, c100(p), nullptr, p->stream));
        RowArgs a{RM_FAT_CS, v, x, blk + 3, p->xscale};
        LSRN_TRY(fused_pass(p, p->vq2, a, p->vq, nullptr));
        LSRN_TRY(launch_gemv(p->NT, r, q, p->vq, rho, rho, nullptr, blk + 5, nullptr, p->stream));
      }
    }
    LSRN_CUDA_TRY(cudaGetLastError());
    return LSRN_OK;
  };
  const bool use_graph = capture_iterations(p) && nsteps > 1;
  cudaGraphExec_t g = nullptr;
  bool g_f32 = false;
  unsigned long long nodes = 0;
  for (int it = 0; it < nsteps; ++it) {
    double change = 0.0;
    if (use_graph && (g == nullptr || g_f32 != p->pass_f32)) {
      if (g != nullptr) cudaGraphExecDestroy(g);
      p->time_passes = false;
      lsrn_status cst = LSRN_OK;
      g = capture_graph(p->stream, [&]() { cst = step_kernels(); }, &nodes);
      if (cst != LSRN_OK && g != nullptr) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
      g_f32 = p->pass_f32;
    }
    if (g != nullptr) {
      LSRN_CUDA_TRY(cudaGraphLaunch(g, p->stream));
      g_kernel_launches.fetch_add(nodes, std::memory_order_relaxed);
    } else {
      LSRN_TRY(step_kernels());
    }
    if (p->tall) LSRN_TRY(rel_change(p, p->xfull, p->tmpq, q, &change));
    else LSRN_TRY(rel_change(p, p->xfull, p->st1, p->nstate, &change, true));
    *inner += steps;
    *taken += 1;
    if (change <= 1e-12) break;
    if (p->pass_f32 && change > prev_change / 20.0) p->pass_f32 = false;
    prev_change = change;
  }
  if (g != nullptr) cudaGraphExecDestroy(g);
  p->pass_f32 = false;
  return LSRN_OK;
}

// Final x (length n) into `xout` (device): m >= n: x = N y; m < n: x = x[:n] (/lambda).
lsrn_status finish_x(Plan* p, double* xout) {
  const int64_t r = p->rank, q = p->q;
  if (r == 0) return fill(p, xout, p->n, 0.0);
  if (p->tall) return launch_gemv_dd(p->Nm, q, r, p->vr[2], xout, p->stream);
  const double sc = p->ridge ? 1.0 / p->lam : 1.0;
  launch(scale_copy_kernel, grid_for(p->n), 256, 0, p->stream, p->st1, p->n, sc, xout);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
