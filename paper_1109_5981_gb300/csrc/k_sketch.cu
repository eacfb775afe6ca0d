// Sketch kernels: A~ = G A (Algorithm 1, step 3) and A~ = A G (Algorithm 2,
// step 3) with G drawn on the fly (step 2), never stored.
//
// Both orientations are computed as C = Gamma^T X with X row-major (L x Q):
//   m >= n:  X = A   (L = m, Q = n), C = A~      (s x n), G = Gamma^T
//   m <  n:  X = A^T (L = n, Q = m), C = A~^T    (s x m), G = Gamma
// Gamma[l, i] (l < L, i < s) is the quantised normal of row l, column i of the
// drawing array, so one Philox call serves four consecutive sketch indices.
#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int SK_BM = 64;   // sketch rows (i) per CTA
constexpr int SK_BN = 64;   // columns of X (j) per CTA
constexpr int SK_BK = 16;   // rows of X (l) per step
constexpr int SK_CHUNK = 512;  // rows of X summed in plain FP64 before the double-double fold

// FP64 FMA sketch tile: C[i0:i0+64, j0:j0+64] += xscale * sum_l Gamma[l, i] X[l, j]
// over l in [lbeg, lend).  256 threads, 4x4 outputs each.  The Gamma tile is
// generated into shared memory once per l-step and shared by the 64 columns.
__global__ void __launch_bounds__(256) sketch_f64_kernel(const double* __restrict__ X, int64_t L,
                                                         int64_t Q, int64_t ldx, double xscale,
                                                         int64_t S, uint64_t seed, uint32_t tag,
                                                         int64_t lchunk, double* __restrict__ out,
                                                         int64_t ldo, int64_t out_stride_z,
                                                         int64_t lbase) {
  __shared__ double Gs[SK_BK][SK_BM];
  __shared__ double Xs[SK_BK][SK_BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t j0 = (int64_t)blockIdx.x * SK_BN;
  const int64_t i0 = (int64_t)blockIdx.y * SK_BM;
  const int64_t lbeg = (int64_t)blockIdx.z * lchunk;
  const int64_t lend = min(L, lbeg + lchunk);
  // Two-level accumulation: acc sums one chunk of SK_CHUNK rows of X, the
  // chunk sums are folded into a double-double total (hi, lo), so rounding
  // grows with sqrt(chunk) instead of with the length of the contraction.
  double acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = hi[a][b] = lo[a][b] = 0.0;

  int steps_in_chunk = 0;
  for (int64_t l0 = lbeg; l0 < lend; l0 += SK_BK) {
    {  // Gamma tile: thread -> (row lr, group of four sketch indices)
      const int lr = tid / 16, g4 = tid % 16;
      const int64_t l = l0 + lr;
      const int64_t i = i0 + 4 * g4;
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (l < lend && i < S) z = normal4(seed, tag, (uint64_t)(lbase + l), (uint64_t)(i >> 2));
      Gs[lr][4 * g4 + 0] = (l < lend && i + 0 < S) ? (double)quantize_g(z.x) : 0.0;
      Gs[lr][4 * g4 + 1] = (l < lend && i + 1 < S) ? (double)quantize_g(z.y) : 0.0;
      Gs[lr][4 * g4 + 2] = (l < lend && i + 2 < S) ? (double)quantize_g(z.z) : 0.0;
      Gs[lr][4 * g4 + 3] = (l < lend && i + 3 < S) ? (double)quantize_g(z.w) : 0.0;
    }
    {  // X tile
      const int lr = tid / 16, c4 = (tid % 16) * 4;
      const int64_t l = l0 + lr;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t j = j0 + c4 + k;
        Xs[lr][c4 + k] = (l < lend && j < Q) ? X[l * ldx + j] * xscale : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK_BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Gs[kk][ty * 4 + u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Xs[kk][tx * 4 + u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
    if (++steps_in_chunk == SK_CHUNK / SK_BK) {
      steps_in_chunk = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          dd_add(hi[u][v], lo[u][v], acc[u][v], 0.0);
          acc[u][v] = 0.0;
        }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dd_add(hi[u][v], lo[u][v], acc[u][v], 0.0);
      acc[u][v] = hi[u][v] + lo[u][v];
    }
  double* o = out + (int64_t)blockIdx.z * out_stride_z;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty * 4 + u;
    if (i >= S) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t j = j0 + tx * 4 + v;
      if (j < Q) o[i * ldo + j] = acc[u][v];
    }
  }
}

// C[i, j] = sum_z P[z][i, j]   (fixed order: deterministic)
__global__ void splitk_reduce_kernel(const double* __restrict__ P, int nz, int64_t S, int64_t Q,
                                     double* __restrict__ C, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * Q) return;
  const int64_t i = idx / Q, j = idx % Q;
  double acc = 0.0;
  for (int z = 0; z < nz; ++z) acc += P[(int64_t)z * S * Q + idx];
  C[i * ldc + j] = acc;
}

// C[i, j] = C[i, j] + coef * Gamma[lrow0 + j, i]
__global__ void sketch_add_gamma_kernel(double* __restrict__ C, int64_t ldc, int64_t S, int64_t Q,
                                        uint64_t seed, uint32_t tag, int64_t lrow0, double coef) {
  const int64_t ng = (S + 3) / 4;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ng * Q) return;
  const int64_t j = idx / ng, g = idx % ng;
  const float4 z = normal4(seed, tag, (uint64_t)(lrow0 + j), (uint64_t)g);
  const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = 4 * g + k;
    if (i < S) C[i * ldc + j] += coef * (double)quantize_g(zz[k]);
  }
}

// C[i, j] = scale * base[i, j] + coef * Gamma[lrow0 + j, i]   (the sketch of a ridge
// problem from its unaugmented part: G_1 A + lambda G_2, or A G_1 / lambda + G_2)
__global__ void ridge_combine_kernel(const double* __restrict__ base, double* __restrict__ C,
                                     int64_t ldc, int64_t S, int64_t Q, double scale,
                                     uint64_t seed, uint32_t tag, int64_t lrow0, double coef) {
  const int64_t ng = (S + 3) / 4;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ng * Q) return;
  const int64_t j = idx / ng, g = idx % ng;
  const float4 z = normal4(seed, tag, (uint64_t)(lrow0 + j), (uint64_t)g);
  const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = 4 * g + k;
    if (i < S) C[i * ldc + j] = fma(coef, (double)quantize_g(zz[k]), scale * base[i * ldc + j]);
  }
}

__global__ void gamma_block_kernel(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0, int64_t rows,
                                   int64_t cols, double* __restrict__ g, float* __restrict__ z) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t r = idx / cols, c = idx % cols;
  const uint64_t j = (uint64_t)(j0 + c);
  const float4 v = normal4(seed, tag, (uint64_t)(i0 + r), j >> 2);
  const float vv[4] = {v.x, v.y, v.z, v.w};
  const float zz = vv[j & 3];
  if (g) g[idx] = (double)quantize_g(zz);
  if (z) z[idx] = zz;
}

// CSR sketch: C[i, j] = xscale * sum_{l in column j of X} X[l, j] Gamma[l, i].
// One CTA per (column j, block of 256 sketch indices); the column's entries are
// walked in stored order (deterministic).
__global__ void __launch_bounds__(256) sketch_csr_kernel(const int64_t* __restrict__ colptr,
                                                         const int32_t* __restrict__ rowidx,
                                                         const double* __restrict__ vals,
                                                         int64_t Q, double xscale, int64_t S,
                                                         uint64_t seed, uint32_t tag,
                                                         double* __restrict__ C, int64_t ldc,
                                                         int64_t lbase) {
  const int64_t j = blockIdx.x;
  const int64_t ib = (int64_t)blockIdx.y * 1024;
  const int tid = threadIdx.x;
  const int64_t i = ib + 4 * tid;     // four sketch indices per thread
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t e0 = colptr[j], e1 = colptr[j + 1];
  for (int64_t e = e0; e < e1; ++e) {
    const int64_t l = rowidx[e];
    const double a = vals[e] * xscale;
    if (i < S) {
      const float4 z = normal4(seed, tag, (uint64_t)(lbase + l), (uint64_t)(i >> 2));
      acc[0] = fma(a, (double)quantize_g(z.x), acc[0]);
      acc[1] = fma(a, (double)quantize_g(z.y), acc[1]);
      acc[2] = fma(a, (double)quantize_g(z.z), acc[2]);
      acc[3] = fma(a, (double)quantize_g(z.w), acc[3]);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (i + k < S) C[(i + k) * ldc + j] = acc[k];
}

int64_t splitk_factor(int64_t L, int64_t Q, int64_t S) {
  const int64_t tiles = ((Q + SK_BN - 1) / SK_BN) * ((S + SK_BM - 1) / SK_BM);
  const int64_t want = (2 * (int64_t)num_sms() + tiles - 1) / tiles;
  const int64_t maxz = std::max<int64_t>(1, L / (SK_BK * 8));
  return std::max<int64_t>(1, std::min(want, maxz));
}

}  // namespace

size_t sketch_f64_scratch_bytes(int64_t L, int64_t Q, int64_t S) {
  const int64_t z = splitk_factor(L, Q, S);
  return z > 1 ? (size_t)z * S * Q * sizeof(double) : 0;
}

lsrn_status launch_sketch_f64(const double* X, int64_t L, int64_t Q, int64_t ldx, double xscale,
                              int64_t S, uint64_t seed, uint32_t tag, double* C, int64_t ldc,
                              double* scratch, size_t scratch_bytes, cudaStream_t st,
                              int64_t lbase) {
  const int64_t z = splitk_factor(L, Q, S);
  const int64_t lchunk = ((L + z - 1) / z + SK_BK - 1) / SK_BK * SK_BK;
  const int64_t nz = (L + lchunk - 1) / lchunk;
  dim3 grid((unsigned)((Q + SK_BN - 1) / SK_BN), (unsigned)((S + SK_BM - 1) / SK_BM), (unsigned)nz);
  if (nz == 1) {
    launch(sketch_f64_kernel, grid, 256, 0, st, X, L, Q, ldx, xscale, S, seed, tag, lchunk, C, ldc,
           (int64_t)0, lbase);
  } else {
    if (scratch == nullptr || scratch_bytes < (size_t)nz * S * Q * sizeof(double))
      return LSRN_ERR_INVALID_ARG;
    launch(sketch_f64_kernel, grid, 256, 0, st, X, L, Q, ldx, xscale, S, seed, tag, lchunk, scratch, Q,
           S * Q, lbase);
    const int64_t tot = S * Q;
    launch(splitk_reduce_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, scratch, (int)nz, S, Q, C,
                                                                          ldc);
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_sketch_f64_splitk_into(const double* X, int64_t L, int64_t Q, int64_t ldx,
                                          int64_t S, uint64_t seed, uint32_t tag, double* C,
                                          int64_t ldc, double* scratch, size_t scratch_doubles,
                                          cudaStream_t st) {
  // split factor as in launch_sketch_f64, capped by the scratch, at least one slice
  int64_t z = splitk_factor(L, Q, S);
  z = std::max<int64_t>(1, std::min<int64_t>(z, (int64_t)(scratch_doubles / (size_t)(S * Q))));
  const int64_t lchunk = ((L + z - 1) / z + SK_BK - 1) / SK_BK * SK_BK;
  const int64_t nz = (L + lchunk - 1) / lchunk;
  if ((size_t)(nz * S * Q) > scratch_doubles) return LSRN_ERR_INVALID_ARG;
  dim3 grid((unsigned)((Q + SK_BN - 1) / SK_BN), (unsigned)((S + SK_BM - 1) / SK_BM), (unsigned)nz);
  launch(sketch_f64_kernel, grid, dim3(256), 0, st, X, L, Q, ldx, 1.0, S, seed, tag, lchunk,
         scratch, Q, S * Q, (int64_t)0);
  const int64_t tot = S * Q;
  launch(splitk_reduce_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st,
         (const double*)scratch, (int)nz, S, Q, C, ldc);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_sketch_add_gamma(double* C, int64_t ldc, int64_t S, int64_t Q, uint64_t seed,
                                    uint32_t tag, int64_t lrow0, double coef, cudaStream_t st) {
  const int64_t tot = ((S + 3) / 4) * Q;
  if (tot == 0) return LSRN_OK;
  launch(sketch_add_gamma_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, C, ldc, S, Q, seed, tag,
                                                                          lrow0, coef);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

// G[c * L + l] = Gamma[l, k0 + c] for l < L, c < kb (zero past column S)
__global__ void gamma_cols_kernel(uint64_t seed, uint32_t tag, int64_t L, int64_t k0, int64_t kb,
                                  int64_t S, double* __restrict__ G) {
  const int64_t ng = (kb + 3) / 4;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ng * L) return;
  const int64_t l = idx % L, g = idx / L;
  const int64_t c0 = 4 * g;                    // k0 is a multiple of 4
  const float4 z = normal4(seed, tag, (uint64_t)l, (uint64_t)((k0 + c0) >> 2));
  const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t c = c0 + k;
    if (c < kb) G[c * L + l] = (k0 + c < S) ? (double)quantize_g(zz[k]) : 0.0;
  }
}

lsrn_status launch_gamma_cols(uint64_t seed, uint32_t tag, int64_t L, int64_t k0, int64_t kb,
                              int64_t S, double* G, cudaStream_t st) {
  if (k0 % 4 != 0) return LSRN_ERR_INVALID_ARG;
  const int64_t tot = ((kb + 3) / 4) * L;
  if (tot == 0) return LSRN_OK;
  launch(gamma_cols_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, seed, tag, L, k0, kb, S, G);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_ridge_combine(const double* base, double* C, int64_t ldc, int64_t S, int64_t Q,
                                 double scale, uint64_t seed, uint32_t tag, int64_t lrow0,
                                 double coef, cudaStream_t st) {
  const int64_t tot = ((S + 3) / 4) * Q;
  if (tot == 0) return LSRN_OK;
  launch(ridge_combine_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, base, C, ldc, S, Q, scale,
         seed, tag, lrow0, coef);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_gamma_block(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0, int64_t rows,
                               int64_t cols, double* g, float* z, cudaStream_t st) {
  const int64_t tot = rows * cols;
  if (tot == 0) return LSRN_OK;
  launch(gamma_block_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, seed, tag, i0, j0, rows, cols,
                                                                      g, z);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_sketch_csr(const int64_t* colptr, const int32_t* rowidx, const double* vals,
                              int64_t L, int64_t Q, double xscale, int64_t S, uint64_t seed,
                              uint32_t tag, double* C, int64_t ldc, cudaStream_t st,
                              int64_t lbase) {
  (void)L;
  if (Q == 0 || S == 0) return LSRN_OK;
  dim3 grid((unsigned)Q, (unsigned)((S + 1023) / 1024));
  launch(sketch_csr_kernel, grid, 256, 0, st, colptr, rowidx, vals, Q, xscale, S, seed, tag, C, ldc,
         lbase);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
