// Inverse of the upper triangular R (q x q) of the sketch's QR factorisation,
// for the preconditioner N = R^-1 of a full-rank problem (preconditioner mode
// LSRN_PRECOND_QR).  With A~ = Q R and R = U_R Sigma V^T, R^-1 = V Sigma^-1 U_R^T:
// A R^-1 = (A V Sigma^-1) U_R^T has the singular values of the SVD
// preconditioner's A N (Lemma 4.3 applies unchanged), so Theorem 4.5's bounds,
// Algorithm 3's step count and LSQR's iterates (up to the orthogonal change of
// variable U_R) are those of N = V Sigma^-1.
//
// Blocked by 64: the diagonal blocks are inverted by back substitution, one
// CTA per block; then block rows from the bottom up,
//   X[i, j] = -R[i, i]^-1 sum_{k = i+1 .. j} R[i, k] X[k, j]   (j > i),
// as one tiled FP64 product T = R[i, i+1:] X[i+1:, i+1:] (X is upper
// triangular, so the sum stops at k = j) and one 64 x 64 by 64 x n product.
#include <algorithm>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int TB = 64;

// Inverse of the diagonal block b of R (rows/cols [64 b, 64 b + nb)): thread c
// solves R_b x = e_c by back substitution; X[b, b] = the inverse (upper triangular).
__global__ void __launch_bounds__(TB) trinv_diag_kernel(const double* __restrict__ R, int64_t ldr,
                                                        int64_t q, double* __restrict__ X,
                                                        int64_t ldx) {
  extern __shared__ double dsm[];                       // two 64 x 65 blocks (66.5 KB)
  double (*Rb)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(dsm);
  double (*Xb)[TB + 1] = reinterpret_cast<double (*)[TB + 1]>(dsm + TB * (TB + 1));
  const int64_t o = (int64_t)blockIdx.x * TB;
  const int nb = (int)min((int64_t)TB, q - o);
  const int c = threadIdx.x;
  for (int i = 0; i < TB; ++i) Rb[i][c] = (i < nb && c < nb && c >= i) ? R[(o + i) * ldr + o + c] : 0.0;
  __syncthreads();
  if (c < nb) {
    for (int i = nb - 1; i >= 0; --i) {
      double acc = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) acc = fma(-Rb[i][k], Xb[k][c], acc);
      Xb[i][c] = (i <= c) ? acc / Rb[i][i] : 0.0;
    }
  }
  __syncthreads();
  for (int i = 0; i < nb; ++i)
    if (c < nb) X[(o + i) * ldx + o + c] = Xb[i][c];
}

// T[0:nb_i, c] = sum_{k = k0 .. min(c, q-1)} R[r0 + ., k] X[k, c] for columns c >= c0,
// a 64 x 64 output tile per CTA (4 x 4 per thread), K in steps of 32.
__global__ void __launch_bounds__(256) trinv_rowprod_kernel(const double* __restrict__ R, int64_t ldr,
                                                            const double* __restrict__ X, int64_t ldx,
                                                            int64_t q, int64_t r0, int nbi, int64_t k0,
                                                            double* __restrict__ T, int64_t ldt) {
  __shared__ double sr[TB][33];
  __shared__ double sx[32][TB + 1];
  const int tid = threadIdx.x;
  const int64_t cb = k0 + (int64_t)blockIdx.x * TB;   // first column of this tile
  const int tr = tid >> 4, tc = tid & 15;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int64_t kend = min(q, cb + TB);   // X[k, c] = 0 for k > c
  for (int64_t ks = k0; ks < kend; ks += 32) {
    for (int t = tid; t < TB * 32; t += 256) {
      const int rr = t / 32, kk = t % 32;
      const int64_t k = ks + kk;
      sr[rr][kk] = (rr < nbi && k < q) ? R[(r0 + rr) * ldr + k] : 0.0;
    }
    for (int t = tid; t < 32 * TB; t += 256) {
      const int kk = t / TB, cc = t % TB;
      const int64_t k = ks + kk, c = cb + cc;
      sx[kk][cc] = (k < q && c < q && k <= c) ? X[k * ldx + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      double ra[4], xb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ra[a] = sr[tr + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) xb[b] = sx[kk][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(ra[a], xb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = tr + 16 * a;
    if (r >= nbi) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = cb + tc + 16 * b;
      if (c < q) T[(int64_t)r * ldt + (c - k0)] = acc[a][b];
    }
  }
}

// X[r0 + i, c] = - sum_k Dinv[i, k] T[k, c - k0]   (Dinv = X[r0.., r0..], the inverted diagonal block)
__global__ void __launch_bounds__(256) trinv_apply_kernel(double* __restrict__ X, int64_t ldx,
                                                          int64_t q, int64_t r0, int nbi, int64_t k0,
                                                          const double* __restrict__ T, int64_t ldt) {
  __shared__ double sd[TB][TB + 1];
  const int tid = threadIdx.x;
  for (int t = tid; t < TB * TB; t += 256) {
    const int i = t / TB, k = t % TB;
    sd[i][k] = (i < nbi && k < nbi) ? X[(r0 + i) * ldx + r0 + k] : 0.0;
  }
  __syncthreads();
  const int64_t c = k0 + (int64_t)blockIdx.x * 256 + tid;
  if (c >= q) return;
  double t[TB];
#pragma unroll
  for (int k = 0; k < TB; ++k) t[k] = k < nbi ? T[(int64_t)k * ldt + (c - k0)] : 0.0;
  for (int i = 0; i < nbi; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < TB; ++k) acc = fma(sd[i][k], t[k], acc);
    X[(r0 + i) * ldx + c] = -acc;
  }
}

// NT[k][i] = N[i][k]
__global__ void transpose_kernel(const double* __restrict__ N, int64_t q, double* __restrict__ NT) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < q && c < q) ? N[r * q + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = c0 + k, c = r0 + threadIdx.x;
    if (r < q && c < q) NT[r * q + c] = tile[threadIdx.x][k];
  }
}

// sig[i] = |R_ii| in the order of descending magnitude (estimates reported in
// lsrn_info for this mode), and the extremes
__global__ void diag_abs_kernel(const double* __restrict__ R, int64_t q, double* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < q) d[i] = fabs(R[i * q + i]);
}

}  // namespace

// N (q x q, row-major) = R^-1 of the upper triangle of Xs (ld q); NT its
// transpose.  T is scratch of 64 x q doubles.
lsrn_status launch_trinv(const double* Xs, int64_t q, double* N, double* NT, double* T,
                         double* diag, cudaStream_t st) {
  const int64_t nbk = (q + TB - 1) / TB;
  LSRN_CUDA_TRY(cudaMemsetAsync(N, 0, (size_t)q * q * sizeof(double), st));
  const size_t dsmem = 2 * TB * (TB + 1) * sizeof(double);
  LSRN_CUDA_TRY(cudaFuncSetAttribute(trinv_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dsmem));
  launch(trinv_diag_kernel, (unsigned)nbk, TB, dsmem, st, Xs, q, q, N, q);
  for (int64_t bi = nbk - 2; bi >= 0; --bi) {
    const int64_t r0 = bi * TB;
    const int nbi = (int)std::min<int64_t>(TB, q - r0);
    const int64_t k0 = r0 + nbi;   // first column right of the diagonal block
    const int64_t ncol = q - k0;
    launch(trinv_rowprod_kernel, (unsigned)((ncol + TB - 1) / TB), 256, 0, st, Xs, q,
           (const double*)N, q, q, r0, nbi, k0, T, q);
    launch(trinv_apply_kernel, (unsigned)((ncol + 255) / 256), 256, 0, st, N, q, q, r0, nbi, k0,
           (const double*)T, q);
  }
  launch(transpose_kernel, dim3((unsigned)((q + 31) / 32), (unsigned)((q + 31) / 32)), dim3(32, 8), 0,
         st, (const double*)N, q, NT);
  launch(diag_abs_kernel, (unsigned)((q + 255) / 256), 256, 0, st, Xs, q, diag);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
