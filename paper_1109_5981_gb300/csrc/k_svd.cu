// Preconditioner (Algorithm 1 steps 4-5, Algorithm 2 steps 4-5) on the device.
//
// Input: the sketch Xs (S x Q, row-major, S > Q): A~ for m >= n, A~^T for m < n.
// 1. Householder QR of Xs -> R (Q x Q upper triangular); Q is not formed.  All
//    columns in one cooperative launch (k_qr_coop.cu) wherever the device
//    holds its grid and the sketch's rows fit its shared memory; otherwise one
//    column at a time up to 3000 columns, blocked in panels of 32 columns
//    with the compact WY form beyond.
// 2. One-sided (Hestenes) Jacobi on Y = R^T: rotate pairs of columns of Y
//    (= rows of R, contiguous in memory) until all pairs are orthogonal to
//    |y_a . y_b| <= tol ||y_a|| ||y_b||; parallel round-robin ordering.  For
//    q > 1024 one persistent kernel per sweep runs the rounds as a dataflow
//    (each pair waits for its two rows); otherwise one kernel per round.  With Y J = W (orthogonal columns, norms sigma_j),
//    R = J Sigma U_W^T, so the right singular vectors of Xs are W Sigma^-1.
// 3. sigma sorted descending, rank r = #{sigma_j > rcond * sigma_1},
//    N = V~ Sigma~^-1 = W_r Sigma_r^-2 (Q x r), also stored transposed.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

// Reflector for column k: H = I - tau v v^T, v_k = 1, annihilates X[k+1:, k].
__global__ void __launch_bounds__(256) hh_reflector_kernel(double* __restrict__ X, int64_t S,
                                                           int64_t Q, int64_t k,
                                                           double* __restrict__ tau) {
  __shared__ double red[8];
  __shared__ double s_scal;
  const int tid = threadIdx.x;
  double ss = 0.0;
  for (int64_t i = k + 1 + tid; i < S; i += 256) {
    const double x = X[i * Q + k];
    ss = fma(x, x, ss);
  }
  ss = group_sum<32>(ss);
  if ((tid & 31) == 0) red[tid >> 5] = ss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    const double alpha = X[k * Q + k];
    double tk = 0.0, scal = 0.0;
    if (t > 0.0) {
      const double nrm = sqrt(alpha * alpha + t);
      const double beta = alpha >= 0.0 ? -nrm : nrm;
      tk = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
      X[k * Q + k] = beta;
    }
    tau[k] = tk;
    s_scal = scal;
  }
  __syncthreads();
  const double scal = s_scal;
  if (scal != 0.0)
    for (int64_t i = k + 1 + tid; i < S; i += 256) X[i * Q + k] *= scal;
}

// wpart[rb][c] = sum_{i in row block rb, i >= k} v_i X[i, c] for c in (k, Q)
__global__ void __launch_bounds__(128) hh_w_kernel(const double* __restrict__ X, int64_t S,
                                                   int64_t Q, int64_t k, int64_t rpb,
                                                   double* __restrict__ wpart,
                                                   const double* __restrict__ tau) {
  if (tau[k] == 0.0) return;
  const int64_t c = k + 1 + (int64_t)blockIdx.x * 128 + threadIdx.x;
  const int64_t r0 = k + (int64_t)blockIdx.y * rpb;
  const int64_t r1 = min(S, r0 + rpb);
  double acc = 0.0;
  if (c < Q) {
    for (int64_t i = r0; i < r1; ++i) {
      const double v = (i == k) ? 1.0 : X[i * Q + k];
      acc = fma(v, X[i * Q + c], acc);
    }
    wpart[(int64_t)blockIdx.y * Q + c] = acc;
  }
}

// X[i, c] -= tau v_i w_c with w_c = sum_rb wpart[rb][c]
__global__ void __launch_bounds__(128) hh_update_kernel(double* __restrict__ X, int64_t S, int64_t Q,
                                                        int64_t k, int64_t rpb, int nrb,
                                                        const double* __restrict__ wpart,
                                                        const double* __restrict__ tau) {
  const double tk = tau[k];
  if (tk == 0.0) return;
  const int64_t c = k + 1 + (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= Q) return;
  double w = 0.0;
  for (int b = 0; b < nrb; ++b) w += wpart[(int64_t)b * Q + c];
  const double t = tk * w;
  const int64_t r0 = k + (int64_t)blockIdx.y * rpb;
  const int64_t r1 = min(S, r0 + rpb);
  for (int64_t i = r0; i < r1; ++i) {
    const double v = (i == k) ? 1.0 : X[i * Q + k];
    X[i * Q + c] = fma(-v, t, X[i * Q + c]);
  }
}

// ---- blocked Householder QR --------------------------------------------------
// Panels of kQrNb columns: one CTA factors the panel in place (reflectors below
// the diagonal with an implicit unit, R on and above it) and forms T of the
// compact WY form H_k0 ... H_k0+nb-1 = I - V T V^T (T upper triangular).  The
// trailing columns C = X[k0:S, k0+nb:Q] then get C <- C - V T^T (V^T C):
// W = V^T C as per-chunk partial sums (row chunks of kQrChunk, summed in a
// fixed order, so the result does not depend on scheduling), W2 = T^T W, and
// the rank-nb update C -= V W2 tile by tile.
constexpr int kQrNb = 32;
constexpr int kQrPanelThreads = 512;
constexpr int kQrChunk = 256;
constexpr int64_t kQrBlockedMin = 3000;   // columns from which the blocked QR is faster

// V[r][i] of panel k0 (rows r >= k0 of X, i < nb): 1 on the diagonal, 0 above.
__device__ __forceinline__ double qr_v(const double* X, int64_t Q, int64_t k0, int64_t r, int i) {
  const int64_t k = k0 + i;
  if (r < k) return 0.0;
  if (r == k) return 1.0;
  return X[r * Q + k];
}

__global__ void __launch_bounds__(kQrPanelThreads) qr_panel_kernel(double* __restrict__ X, int64_t S,
                                                                    int64_t Q, int64_t k0, int nb,
                                                                    double* __restrict__ tau,
                                                                    double* __restrict__ T) {
  __shared__ double red[kQrPanelThreads / 32][kQrNb];
  __shared__ double vals[kQrNb];
  __shared__ double Ts[kQrNb][kQrNb];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  for (int q = tid; q < kQrNb * kQrNb; q += kQrPanelThreads) Ts[q / kQrNb][q % kQrNb] = 0.0;
  for (int j = 0; j < nb; ++j) {
    const int64_t k = k0 + j;
    // 1. reflector for column k
    double ss = 0.0;
    for (int64_t r = k + 1 + tid; r < S; r += kQrPanelThreads) {
      const double x = X[r * Q + k];
      ss = fma(x, x, ss);
    }
    ss = group_sum<32>(ss);
    if (lane == 0) red[wp][0] = ss;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kQrPanelThreads / 32; ++w) t += red[w][0];
      const double alpha = X[k * Q + k];
      double tk = 0.0, scal = 0.0;
      if (t > 0.0) {
        const double nrm = sqrt(alpha * alpha + t);
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        tk = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
        X[k * Q + k] = beta;
      }
      tau[k] = tk;
      vals[0] = tk;
      vals[1] = scal;
    }
    __syncthreads();
    const double tk = vals[0], scal = vals[1];
    if (scal != 0.0)
      for (int64_t r = k + 1 + tid; r < S; r += kQrPanelThreads) X[r * Q + k] *= scal;
    __syncthreads();
    // 2. apply H_k to the panel columns k+1 .. k0+nb-1
    const int ncol = nb - j - 1;
    if (ncol > 0 && tk != 0.0) {
      double part[kQrNb];
#pragma unroll
      for (int c = 0; c < kQrNb; ++c) part[c] = 0.0;
      for (int64_t r = k + tid; r < S; r += kQrPanelThreads) {
        const double v = (r == k) ? 1.0 : X[r * Q + k];
#pragma unroll
        for (int c = 0; c < kQrNb; ++c)
          if (c < ncol) part[c] = fma(v, X[r * Q + k + 1 + c], part[c]);
      }
#pragma unroll
      for (int c = 0; c < kQrNb; ++c) {
        if (c < ncol) {
          const double t = group_sum<32>(part[c]);
          if (lane == 0) red[wp][c] = t;
        }
      }
      __syncthreads();
      if (tid < ncol) {
        double t = 0.0;
        for (int w = 0; w < kQrPanelThreads / 32; ++w) t += red[w][tid];
        vals[tid] = tk * t;
      }
      __syncthreads();
      for (int64_t r = k + tid; r < S; r += kQrPanelThreads) {
        const double v = (r == k) ? 1.0 : X[r * Q + k];
        for (int c = 0; c < ncol; ++c) X[r * Q + k + 1 + c] = fma(-v, vals[c], X[r * Q + k + 1 + c]);
      }
      __syncthreads();
    }
  }
  // 3. T: T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j)
  for (int j = 0; j < nb; ++j) {
    double part[kQrNb];
#pragma unroll
    for (int c = 0; c < kQrNb; ++c) part[c] = 0.0;
    for (int64_t r = k0 + j + tid; r < S; r += kQrPanelThreads) {
      const double vj = qr_v(X, Q, k0, r, j);
#pragma unroll
      for (int c = 0; c < kQrNb; ++c)
        if (c < j) part[c] = fma(qr_v(X, Q, k0, r, c), vj, part[c]);
    }
#pragma unroll
    for (int c = 0; c < kQrNb; ++c) {
      if (c < j) {
        const double t = group_sum<32>(part[c]);
        if (lane == 0) red[wp][c] = t;
      }
    }
    __syncthreads();
    if (tid < j) {
      double t = 0.0;
      for (int w = 0; w < kQrPanelThreads / 32; ++w) t += red[w][tid];
      vals[tid] = t;
    }
    __syncthreads();
    if (tid == 0) {
      const double tj = tau[k0 + j];
      for (int i = 0; i < j; ++i) {
        double acc = 0.0;
        for (int l = i; l < j; ++l) acc = fma(Ts[i][l], vals[l], acc);
        Ts[i][j] = -tj * acc;
      }
      Ts[j][j] = tj;
      for (int i = j + 1; i < kQrNb; ++i) Ts[i][j] = 0.0;
    }
    __syncthreads();
  }
  for (int q = tid; q < kQrNb * kQrNb; q += kQrPanelThreads) T[q] = Ts[q / kQrNb][q % kQrNb];
}

// Wpart[ch][i][c] = sum over rows r of chunk ch of V[r][i] C[r][c], c = trailing column
// index (0 .. Q - k0 - nb), 64 columns per CTA, rows [k0 + ch kQrChunk, ...).
__global__ void __launch_bounds__(256) qr_vtc_kernel(const double* __restrict__ X, int64_t S,
                                                     int64_t Q, int64_t k0, int nb,
                                                     double* __restrict__ Wpart) {
  __shared__ double sv[32][kQrNb + 1];
  __shared__ double sc[32][64 + 1];
  const int tid = threadIdx.x;
  const int c = tid & 63, ib = tid >> 6;   // 4 blocks of 8 reflectors
  const int64_t cbase = k0 + nb + (int64_t)blockIdx.x * 64;
  const int64_t ncol_tr = Q - k0 - nb;
  const int64_t r0 = k0 + (int64_t)blockIdx.y * kQrChunk;
  const int64_t r1 = min(S, r0 + kQrChunk);
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (int64_t rs = r0; rs < r1; rs += 32) {
    for (int q = tid; q < 32 * kQrNb; q += 256) {
      const int rr = q / kQrNb, i = q % kQrNb;
      const int64_t r = rs + rr;
      sv[rr][i] = (r < r1 && i < nb) ? qr_v(X, Q, k0, r, i) : 0.0;
    }
    for (int q = tid; q < 32 * 64; q += 256) {
      const int rr = q / 64, cc = q % 64;
      const int64_t r = rs + rr, col = cbase + cc;
      sc[rr][cc] = (r < r1 && col < Q) ? X[r * Q + col] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const double x = sc[rr][c];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(sv[rr][ib * 8 + q], x, acc[q]);
    }
    __syncthreads();
  }
  const int64_t col = (int64_t)blockIdx.x * 64 + c;
  if (col < ncol_tr) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = ib * 8 + q;
      Wpart[((int64_t)blockIdx.y * kQrNb + i) * ncol_tr + col] = acc[q];
    }
  }
}

// W2[:, c] = T^T (sum over chunks of Wpart[ch][:, c]), one thread per trailing column.
__global__ void qr_w2_kernel(const double* __restrict__ Wpart, int nchunk, int64_t ncol_tr, int nb,
                             const double* __restrict__ T, double* __restrict__ W2) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol_tr) return;
  double w[kQrNb];
#pragma unroll
  for (int i = 0; i < kQrNb; ++i) w[i] = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) {
#pragma unroll
    for (int i = 0; i < kQrNb; ++i)
      if (i < nb) w[i] += Wpart[((int64_t)ch * kQrNb + i) * ncol_tr + c];
  }
#pragma unroll
  for (int j = 0; j < kQrNb; ++j) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i <= j; ++i) t = fma(T[i * kQrNb + j], w[i], t);
    if (j < nb) W2[(int64_t)j * ncol_tr + c] = t;
  }
}

// C[r][c] -= sum_i V[r][i] W2[i][c] on a 64 x 64 tile (4 x 4 outputs per thread).
__global__ void __launch_bounds__(256) qr_update_kernel(double* __restrict__ X, int64_t S, int64_t Q,
                                                        int64_t k0, int nb,
                                                        const double* __restrict__ W2) {
  __shared__ double sv[64][kQrNb + 1];
  __shared__ double sw[kQrNb][64 + 1];
  const int tid = threadIdx.x;
  const int64_t ncol_tr = Q - k0 - nb;
  const int64_t ct = (int64_t)blockIdx.x * 64, rt = k0 + (int64_t)blockIdx.y * 64;
  for (int q = tid; q < 64 * kQrNb; q += 256) {
    const int rr = q / kQrNb, i = q % kQrNb;
    const int64_t r = rt + rr;
    sv[rr][i] = (r < S && i < nb) ? qr_v(X, Q, k0, r, i) : 0.0;
  }
  for (int q = tid; q < kQrNb * 64; q += 256) {
    const int i = q / 64, cc = q % 64;
    const int64_t col = ct + cc;
    sw[i][cc] = (i < nb && col < ncol_tr) ? W2[(int64_t)i * ncol_tr + col] : 0.0;
  }
  __syncthreads();
  const int tr = tid >> 4, tc = tid & 15;   // 16 x 16 threads, 4 x 4 outputs each
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 8
  for (int i = 0; i < kQrNb; ++i) {
    double va[4], wb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) va[a] = sv[tr + 16 * a][i];
#pragma unroll
    for (int b = 0; b < 4; ++b) wb[b] = sw[i][tc + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(va[a], wb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = rt + tr + 16 * a;
    if (r >= S) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t col = ct + tc + 16 * b;
      if (col < ncol_tr) X[r * Q + k0 + nb + col] -= acc[a][b];
    }
  }
}

// W[j][c] = R[j][c] (upper triangle of X), zero below the diagonal
__global__ void extract_r_kernel(const double* __restrict__ X, int64_t Q, double* __restrict__ W) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Q * Q) return;
  const int64_t j = idx / Q, c = idx % Q;
  W[idx] = (c >= j) ? X[j * Q + c] : 0.0;
}

// One round of the parallel one-sided Jacobi sweep: warp per pair of rows of W.
// Round-robin (circle) schedule over P (even) players: pair 0 = (P-1, t),
// pair k >= 1 = ((t + k) mod (P-1), (t - k + P - 1) mod (P-1)).
__global__ void __launch_bounds__(256) jacobi_round_kernel(double* __restrict__ W, int64_t Q, int P,
                                                           int t, double tol,
                                                           int* __restrict__ rot_count) {
  const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= P / 2) return;
  int a, b;
  if (warp == 0) {
    a = P - 1;
    b = t;
  } else {
    a = (t + warp) % (P - 1);
    b = (t - warp + P - 1) % (P - 1);
  }
  if (a >= Q || b >= Q) return;
  if (a > b) {
    const int tmp = a;
    a = b;
    b = tmp;
  }
  double* wa = W + (int64_t)a * Q;
  double* wb = W + (int64_t)b * Q;
  double aa = 0.0, bb = 0.0, ab = 0.0;
  for (int64_t c = lane; c < Q; c += 32) {
    const double x = wa[c], y = wb[c];
    aa = fma(x, x, aa);
    bb = fma(y, y, bb);
    ab = fma(x, y, ab);
  }
  aa = group_sum<32>(aa);
  bb = group_sum<32>(bb);
  ab = group_sum<32>(ab);
  if (aa == 0.0 || bb == 0.0) return;
  if (fabs(ab) <= tol * sqrt(aa) * sqrt(bb)) return;
  const double zeta = (bb - aa) / (2.0 * ab);
  double tt;
  if (fabs(zeta) > 1e150) {
    tt = 0.5 / zeta;
  } else {
    tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  }
  const double cs = 1.0 / sqrt(1.0 + tt * tt);
  const double sn = cs * tt;
  for (int64_t c = lane; c < Q; c += 32) {
    const double x = wa[c], y = wb[c];
    wa[c] = cs * x - sn * y;
    wb[c] = sn * x + cs * y;
  }
  if (lane == 0) atomicAdd(rot_count, 1);
}

// One round with the rows of a pair held in registers: a CTA of kJacThreads per
// pair, EPT elements of each row per thread (Q <= kJacThreads * EPT).  Squared
// row norms are carried in nrm2 (exact at the start of each sweep) and updated
// after a rotation by the Hestenes identities aa' = aa - t ab, bb' = bb + t ab,
// so a pair costs one dot product unless it rotates.  A norm that falls below
// a quarter of its value is recomputed from the rotated row (cancellation).
constexpr int kJacThreads = 128;

__device__ __forceinline__ double jac_block_sum(double v, double* sh) {
  v = group_sum<32>(v);
  __syncthreads();   // sh may still be read from the previous sum
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < kJacThreads / 32; ++q) t += sh[q];
  return t;
}

// The same sum, valid in thread 0 only (the other threads do not add up the
// warp partials: on GB300 every warp-wide FP64 instruction costs 16 cycles of
// the SM's FP64 pipe).
__device__ __forceinline__ double jac_block_sum0(double v, double* sh) {
  v = group_sum<32>(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kJacThreads / 32; ++q) t += sh[q];
  }
  return t;
}

template <int EPT>
__global__ void __launch_bounds__(kJacThreads) jacobi_pair_kernel(double* __restrict__ W, int64_t Q,
                                                                  int P, int t, double tol,
                                                                  double* __restrict__ nrm2,
                                                                  int* __restrict__ rot_count) {
  __shared__ double sh[kJacThreads / 32];
  const int pr = blockIdx.x;
  int a, b;
  if (pr == 0) {
    a = P - 1;
    b = t;
  } else {
    a = (t + pr) % (P - 1);
    b = (t - pr + P - 1) % (P - 1);
  }
  if (a >= Q || b >= Q) return;
  if (a > b) {
    const int tmp = a;
    a = b;
    b = tmp;
  }
  double* wa = W + (int64_t)a * Q;
  double* wb = W + (int64_t)b * Q;
  const double aa = nrm2[a], bb = nrm2[b];   // issued with the row loads
  double x[EPT], y[EPT];
  double ab = 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int64_t c = threadIdx.x + (int64_t)kJacThreads * e;
    x[e] = c < Q ? wa[c] : 0.0;
    y[e] = c < Q ? wb[c] : 0.0;
    ab = fma(x[e], y[e], ab);
  }
  ab = jac_block_sum(ab, sh);
  if (aa == 0.0 || bb == 0.0) return;
  // the angle (square roots and divisions, ~70 FP64 operations) once per pair
  __shared__ double rot[3];
  if (threadIdx.x == 0) {
    double tt = 0.0, cs = 1.0;
    if (fabs(ab) > tol * sqrt(aa) * sqrt(bb)) {
      const double zeta = (bb - aa) / (2.0 * ab);
      if (fabs(zeta) > 1e150) {
        tt = 0.5 / zeta;
      } else {
        tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      }
      cs = 1.0 / sqrt(1.0 + tt * tt);
    }
    rot[0] = tt;
    rot[1] = cs;
    rot[2] = cs * tt;
  }
  __syncthreads();
  const double tt = rot[0], cs = rot[1], sn = rot[2];
  if (tt == 0.0) return;   // converged pair (uniform)
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int64_t c = threadIdx.x + (int64_t)kJacThreads * e;
    const double xa = cs * x[e] - sn * y[e];
    const double yb = sn * x[e] + cs * y[e];
    x[e] = xa;
    y[e] = yb;
    if (c < Q) {
      wa[c] = xa;
      wb[c] = yb;
    }
  }
  double na = aa - tt * ab, nb = bb + tt * ab;
  if (na < 0.25 * aa || nb < 0.25 * bb) {   // uniform: every thread has the same values
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      sa = fma(x[e], x[e], sa);
      sb = fma(y[e], y[e], sb);
    }
    na = jac_block_sum(sa, sh);
    nb = jac_block_sum(sb, sh);
  }
  if (threadIdx.x == 0) {
    nrm2[a] = na;
    nrm2[b] = nb;
    *rot_count = 1;   // "some pair rotated in this sweep" (every writer stores 1)
  }
}

// ---- dataflow sweep: one persistent launch per sweep (q > 1024) ----
// Work item i = t * (P/2) + k is pair k of round t of the round-robin order.
// CTAs take items in increasing order from an atomic counter.  An item waits
// until both of its rows have finished round t - 1 (per-row counters ver[row]),
// rotates them exactly as jacobi_pair_kernel does and publishes ver = t + 1.
// Every dependency of an item has a smaller index, and all smaller items were
// taken by running CTAs, so the smallest unfinished item can always proceed:
// no barrier between rounds, no tail of a partial wave, one launch per sweep.
// Each row sees the same rotations in the same order as with one launch per
// round, so the result is the same bit for bit.
// ws[0]: next item, ws[1]: error flag (a wait gave up), ws[2 + row]: ver[row].
// A wait is bounded by elapsed time on the GPU's global timer (wait_ns, one
// second by default); then the CTA raises the flag, every CTA stops at its
// next item or poll, and the preconditioner returns LSRN_ERR_TIMEOUT.
constexpr uint64_t kJacWaitNs = 1000000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// EPT = 16 is held to 95 registers (5 CTAs per SM) without spills.
template <int EPT>
__global__ void __launch_bounds__(kJacThreads, EPT >= 32 ? 1 : 5)
    jacobi_flow_kernel(double* __restrict__ W, int64_t Q, int P, double tol,
                       double* __restrict__ nrm2, int* __restrict__ rot_count,
                       int* __restrict__ ws, uint64_t wait_ns) {
  __shared__ double sh[kJacThreads / 32];
  __shared__ double rot[3];
  __shared__ int s_rec;
  __shared__ int s_item, s_ok;
  int* next = ws;
  int* err = ws + 1;
  int* ver = ws + 2;
  const int npairs = P / 2;
  const int total = (P - 1) * npairs;
  for (;;) {
    __syncthreads();   // the previous item is done with s_item, rot and sh
    if (threadIdx.x == 0) {
      const int item = atomicAdd(next, 1);
      int ok = 0;
      if (item < total && ld_acquire_gpu(err) == 0) {
        const int t = item / npairs, k = item % npairs;
        const int a = k == 0 ? P - 1 : (t + k) % (P - 1);
        const int b = k == 0 ? t : (t - k + P - 1) % (P - 1);
        ok = 1;
        const uint64_t t0 = globaltimer_ns();
        for (int it = 0;; ++it) {
          const bool ra = a >= Q || ld_acquire_gpu(ver + a) >= t;
          const bool rb = b >= Q || ld_acquire_gpu(ver + b) >= t;
          if (ra && rb) break;
          if ((it & 15) == 15 &&
              (globaltimer_ns() - t0 > wait_ns || ld_acquire_gpu(err) != 0)) {
            atomicExch(err, 1);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();   // the rows published with ver are read after this point
      }
      s_item = item;
      s_ok = ok;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= total || s_ok == 0) return;   // uniform
    const int t = item / npairs, k = item % npairs;
    int a = k == 0 ? P - 1 : (t + k) % (P - 1);
    int b = k == 0 ? t : (t - k + P - 1) % (P - 1);
    if (a >= Q || b >= Q) {   // the row without a partner this round only advances
      if (threadIdx.x == 0) {
        const int r = a < Q ? a : b;
        if (r < Q) st_release_gpu(ver + r, t + 1);
      }
      continue;
    }
    if (a > b) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    double* wa = W + (int64_t)a * Q;
    double* wb = W + (int64_t)b * Q;
    const double aa = __ldcg(nrm2 + a), bb = __ldcg(nrm2 + b);
    double x[EPT], y[EPT];
    double ab = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t c = threadIdx.x + (int64_t)kJacThreads * e;
      x[e] = c < Q ? __ldcg(wa + c) : 0.0;
      y[e] = c < Q ? __ldcg(wb + c) : 0.0;
      ab = fma(x[e], y[e], ab);
    }
    ab = jac_block_sum0(ab, sh);   // thread 0 only
    double na = aa, nb = bb;       // thread 0: the new squared norms
    if (threadIdx.x == 0) {
      double tt = 0.0, cs = 1.0;
      // |ab| > tol sqrt(aa bb): one square root where aa bb is a normal number
      const double pab = aa * bb;
      const double lim = (pab >= 0x1p-1000 && pab <= 0x1p+1000) ? tol * sqrt(pab) : tol * sqrt(aa) * sqrt(bb);
      if (aa != 0.0 && bb != 0.0 && fabs(ab) > lim) {
        const double zeta = (bb - aa) / (2.0 * ab);
        if (fabs(zeta) > 1e150) {
          tt = 0.5 / zeta;
        } else {
          tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        }
        cs = rsqrt(1.0 + tt * tt);
      }
      na = aa - tt * ab;
      nb = bb + tt * ab;
      rot[0] = tt;
      rot[1] = cs;
      rot[2] = cs * tt;
      s_rec = tt != 0.0 && (na < 0.25 * aa || nb < 0.25 * bb);
    }
    __syncthreads();
    const double tt = rot[0], cs = rot[1], sn = rot[2];
    if (tt != 0.0) {   // uniform
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int64_t c = threadIdx.x + (int64_t)kJacThreads * e;
        const double xa = cs * x[e] - sn * y[e];
        const double yb = sn * x[e] + cs * y[e];
        x[e] = xa;
        y[e] = yb;
        if (c < Q) {
          wa[c] = xa;
          wb[c] = yb;
        }
      }
      if (s_rec) {   // uniform: cancellation, the rotated rows' norms
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          sa = fma(x[e], x[e], sa);
          sb = fma(y[e], y[e], sb);
        }
        const double ra = jac_block_sum0(sa, sh);
        const double rb = jac_block_sum0(sb, sh);
        if (threadIdx.x == 0) {
          na = ra;
          nb = rb;
        }
      }
      if (threadIdx.x == 0) {
        nrm2[a] = na;
        nrm2[b] = nb;
        *rot_count = 1;
      }
      __threadfence();   // this thread's row (and norm) stores before the release below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release_gpu(ver + a, t + 1);
      st_release_gpu(ver + b, t + 1);
    }
  }
}

__global__ void set_int_kernel(int* __restrict__ p, int v) { *p = v; }

__global__ void row_sqnorms_kernel(const double* __restrict__ W, int64_t Q, double* __restrict__ nrm2) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= Q) return;
  double acc = 0.0;
  for (int64_t c = lane; c < Q; c += 32) {
    const double x = W[row * Q + c];
    acc = fma(x, x, acc);
  }
  acc = group_sum<32>(acc);
  if (lane == 0) nrm2[row] = acc;
}

__global__ void row_norms_kernel(const double* __restrict__ W, int64_t Q, double* __restrict__ nrm) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= Q) return;
  double acc = 0.0;
  for (int64_t c = lane; c < Q; c += 32) {
    const double x = W[row * Q + c];
    acc = fma(x, x, acc);
  }
  acc = group_sum<32>(acc);
  if (lane == 0) nrm[row] = sqrt(acc);
}

// Stable descending order of the norms, rank count, sigma extremes.
__global__ void __launch_bounds__(1024) sort_rank_kernel(const double* __restrict__ nrm, int64_t Q,
                                                         double rcond, int* __restrict__ perm,
                                                         double* __restrict__ sig,
                                                         int* __restrict__ rank_out) {
  __shared__ double smax[32];
  __shared__ int scount[32];
  const int tid = threadIdx.x;
  double mx = 0.0;
  for (int64_t j = tid; j < Q; j += 1024) mx = fmax(mx, nrm[j]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) smax[tid >> 5] = mx;
  __syncthreads();
  if (tid < 32) {
    double v = smax[tid];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) smax[0] = v;
  }
  __syncthreads();
  const double sigmax = smax[0];
  int cnt = 0;
  for (int64_t j = tid; j < Q; j += 1024) {
    const double sj = nrm[j];
    int64_t pos = 0;
    for (int64_t k = 0; k < Q; ++k) {
      const double sk = nrm[k];
      pos += (sk > sj) || (sk == sj && k < j);
    }
    perm[pos] = (int)j;
    sig[pos] = sj;
    cnt += (sigmax > 0.0 && sj > rcond * sigmax) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __syncthreads();
  if ((tid & 31) == 0) scount[tid >> 5] = cnt;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int w = 0; w < 32; ++w) t += scount[w];
    *rank_out = t;
  }
}

// N[i][k] = W[perm[k]][i] / sig[k]^2 ; NT[k][i] = same  (i < Q, k < r)
__global__ void form_n_kernel(const double* __restrict__ W, int64_t Q, const int* __restrict__ perm,
                              const double* __restrict__ sig, int64_t r, double* __restrict__ N,
                              double* __restrict__ NT) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Q * r) return;
  const int64_t k = idx / Q, i = idx % Q;
  const double s = sig[k];
  const double v = W[(int64_t)perm[k] * Q + i] / (s * s);
  NT[k * Q + i] = v;
  N[i * r + k] = v;
}

// out[0] = sum of squares of v[0:n] (one CTA, fixed order per thread then tree)
__global__ void __launch_bounds__(1024) sumsq_one_kernel(const double* __restrict__ v, int64_t n,
                                                         double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) acc = fma(v[i], v[i], acc);
  acc = group_sum<32>(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += sh[w];
    out[0] = t;
  }
}

// out[0] = min_i |R[i, i]| over the diagonal of the QR-factored sketch (row-major, ld Q)
__global__ void __launch_bounds__(1024) min_abs_diag_kernel(const double* __restrict__ X, int64_t Q,
                                                            double* __restrict__ out) {
  __shared__ double sh[32];
  double mn = INFINITY;
  for (int64_t i = threadIdx.x; i < Q; i += 1024) mn = fmin(mn, fabs(X[i * Q + i]));
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = INFINITY;
    for (int w = 0; w < 32; ++w) t = fmin(t, sh[w]);
    out[0] = t;
  }
}

}  // namespace

lsrn_status run_precond(Plan* p, bool bf16_check) {
  cudaStream_t st = p->stream;
  const int64_t S = p->s, Q = p->q;
  double* X = p->Xs;
  if (bf16_check) {
    // noise floor of a BF16 sketch: 2^-8 of the root-mean-square singular value
    double f2 = 0.0;
    launch(sumsq_one_kernel, 1, 1024, 0, st, (const double*)X, S * Q, p->tmpq);
    LSRN_CUDA_TRY(cudaMemcpyAsync(&f2, p->tmpq, sizeof(double), cudaMemcpyDeviceToHost, st));
    LSRN_CUDA_TRY(cudaStreamSynchronize(st));
    p->bf16_noise = 0x1p-8 * std::sqrt(f2 / (double)std::max<int64_t>(Q, 1));
  }
  // 1. Householder QR, one column at a time: all columns in one cooperative
  // launch with two grid barriers per column (k_qr_coop.cu).  Where the device
  // cannot hold that grid (or the sketch is taller than its shared-memory
  // limit): up to kQrBlockedMin columns three launches per column, the
  // trailing update spread over the whole GPU; beyond that in panels of kQrNb
  // columns, where the O(S q^2) trailing work runs as a blocked rank-32 update
  // and the serial panel factorizations are a small part.
  bool coop = false;
  LSRN_TRY(launch_qr_coop(X, S, Q, p->tau, st, &coop));
  if (coop) {
    // done in one cooperative launch (k_qr_coop.cu)
  } else if (Q <= kQrBlockedMin) {
    double* wpart = p->pvec;   // reuse pass partial buffer: needs nrb * Q doubles
    const int64_t cap_rows =
        std::max<int64_t>(1, (int64_t)(p->nblk + 1) * p->xcols / std::max<int64_t>(Q, 1));
    for (int64_t k = 0; k < Q; ++k) {
      launch(hh_reflector_kernel, 1, 256, 0, st, X, S, Q, k, p->tau);
      const int64_t ncols = Q - k - 1;
      if (ncols <= 0) continue;
      const int64_t cblk = (ncols + 127) / 128;
      const int64_t rows = S - k;
      int64_t nrb = std::max<int64_t>(1, (2 * num_sms() + cblk - 1) / cblk);
      nrb = std::min<int64_t>(nrb, (rows + 63) / 64);
      nrb = std::min<int64_t>(nrb, cap_rows);
      const int64_t rpb = (rows + nrb - 1) / nrb;
      nrb = (rows + rpb - 1) / rpb;
      dim3 grid((unsigned)cblk, (unsigned)nrb);
      launch(hh_w_kernel, grid, 128, 0, st, X, S, Q, k, rpb, wpart, p->tau);
      launch(hh_update_kernel, grid, 128, 0, st, X, S, Q, k, rpb, (int)nrb, wpart, p->tau);
    }
    LSRN_CUDA_TRY(cudaGetLastError());
  } else {
    const int64_t max_chunks = (S + kQrChunk - 1) / kQrChunk;
    const size_t ws = ((size_t)max_chunks * kQrNb * Q + (size_t)kQrNb * Q + kQrNb * kQrNb) *
                      sizeof(double);
    double* qws = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&qws, ws, st));
    double* Wpart = qws;
    double* W2 = Wpart + (size_t)max_chunks * kQrNb * Q;
    double* Tm = W2 + (size_t)kQrNb * Q;
    for (int64_t k0 = 0; k0 < Q; k0 += kQrNb) {
      const int nb = (int)std::min<int64_t>(kQrNb, Q - k0);
      launch(qr_panel_kernel, 1, kQrPanelThreads, 0, st, X, S, Q, k0, nb, p->tau, Tm);
      const int64_t ncol_tr = Q - k0 - nb;
      if (ncol_tr <= 0) continue;
      const int nchunk = (int)((S - k0 + kQrChunk - 1) / kQrChunk);
      launch(qr_vtc_kernel, dim3((unsigned)((ncol_tr + 63) / 64), (unsigned)nchunk), 256, 0, st,
             (const double*)X, S, Q, k0, nb, Wpart);
      launch(qr_w2_kernel, (unsigned)((ncol_tr + 127) / 128), 128, 0, st, (const double*)Wpart,
             nchunk, ncol_tr, nb, (const double*)Tm, W2);
      launch(qr_update_kernel, dim3((unsigned)((ncol_tr + 63) / 64), (unsigned)((S - k0 + 63) / 64)),
             256, 0, st, X, S, Q, k0, nb, (const double*)W2);
    }
    LSRN_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(qws, st);
  }
  cudaEventRecord(p->ev[8], st);
  if (bf16_check && p->opt.sketch_mode == LSRN_SKETCH_AUTO) {
    // sigma_min(R) <= min |R_ii|: below the floor already, the Jacobi is skipped
    double dmin = 0.0;
    launch(min_abs_diag_kernel, 1, 1024, 0, st, (const double*)X, Q, p->tmpq);
    LSRN_CUDA_TRY(cudaMemcpyAsync(&dmin, p->tmpq, sizeof(double), cudaMemcpyDeviceToHost, st));
    LSRN_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(dmin >= 16.0 * p->bf16_noise)) return kPrecondEscalate;
  }
  if (p->opt.precond_mode == LSRN_PRECOND_QR && p->ridge) {
    // full rank by construction: N = R^-1, no Jacobi sweeps (k_trinv.cu)
    double* T = nullptr;
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&T, (size_t)64 * Q * sizeof(double), st));
    const lsrn_status ts = launch_trinv(X, Q, p->Nm, p->NT, T, p->tmpq, st);
    cudaFreeAsync(T, st);
    LSRN_TRY(ts);
    cudaEventRecord(p->ev[9], st);
    std::vector<double> d((size_t)Q);
    LSRN_CUDA_TRY(cudaMemcpyAsync(d.data(), p->tmpq, (size_t)Q * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
    LSRN_CUDA_TRY(cudaStreamSynchronize(st));
    std::sort(d.begin(), d.end(), [](double a, double b) { return a > b; });
    LSRN_CUDA_TRY(cudaMemcpyAsync(p->sig, d.data(), (size_t)Q * sizeof(double),
                                  cudaMemcpyHostToDevice, st));
    LSRN_CUDA_TRY(cudaStreamSynchronize(st));
    p->rank = Q;
    p->sigma_max = d.front();
    p->sigma_min = d.back();
    p->sweeps = 0;
    return LSRN_OK;
  }
  // 2. One-sided Jacobi on the rows of R.
  const int64_t QQ = Q * Q;
  const int P = (int)(Q + (Q & 1));
  const double tol = (double)std::max(S, Q) * 0x1p-53;
  const int warps_per_round = P / 2;
  const unsigned rblocks = (unsigned)((warps_per_round * 32 + 255) / 256);
  int* rot = p->iscal + IC_ROT;
  int host_rot = 0;
  int sweeps = 0;
  const int max_sweeps = 40;
  // rows in registers when they fit (Q <= 4096), else the streaming warp-per-pair kernel
  const int ept = Q <= 512 ? 4 : Q <= 1024 ? 8 : Q <= 2048 ? 16 : Q <= 4096 ? 32 : 0;
  double* nrm2 = p->tmpq;
  // q > 1024 (16 or 32 elements of a row per thread): the dataflow sweep.  At
  // smaller q the rows are short and the chain of rounds bounds it, so the
  // rounds are launched one by one (from a graph).
  const bool flow = ept >= 16;
  int* jws = nullptr;
  int flow_grid = 0;
  // Test knobs (lsrn_set_test_knob): a shorter wait limit, and items of the
  // first round skipped so that every later item waits on rows that are never
  // published -- the only way to make the bounded wait run out on purpose.
  const int64_t knob_wait = test_knob(LSRN_KNOB_JACOBI_WAIT_NS);
  const uint64_t wait_ns = knob_wait > 0 ? (uint64_t)knob_wait : kJacWaitNs;
  const int skip_items = test_knob(LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND) != 0 ? P / 2 : 0;
  // Double-float pre-sweeps (k_jacobi_df.cu) leave Y = P R in Wj, nearly
  // orthogonal rows; otherwise Wj = R.
  p->sweeps_df = 0;
  if (flow && p->opt.svd_mode == LSRN_SVD_DF && jacobi_df_applies(Q)) {
    int dsw = 0;
    const lsrn_status ds = jacobi_df_phase(p, knob_wait, skip_items, &dsw);
    p->sweeps_df = dsw;
    if (ds != LSRN_OK) {
      p->sweeps = 0;
      return ds;
    }
  } else {
    launch(extract_r_kernel, (unsigned)((QQ + 255) / 256), 256, 0, st, X, Q, p->Wj);
    LSRN_CUDA_TRY(cudaGetLastError());
  }
  if (flow) {
    LSRN_CUDA_TRY(lsrn_malloc_async((void**)&jws, (Q + 2) * sizeof(int), st));
    int per_sm = 0;
    if (ept == 16)
      LSRN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_flow_kernel<16>,
                                                                  kJacThreads, 0));
    else
      LSRN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_flow_kernel<32>,
                                                                  kJacThreads, 0));
    const int64_t items = (int64_t)(P - 1) * (P / 2);
    flow_grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * num_sms(), items));
  }
  // One sweep: reset the rotation flag, exact squared norms, P - 1 rounds.
  auto issue_sweep = [&]() {
    cudaMemsetAsync(rot, 0, sizeof(int), st);
    if (ept > 0)
      launch(row_sqnorms_kernel, (unsigned)((Q * 32 + 255) / 256), 256, 0, st, p->Wj, Q, nrm2);
    if (flow) {
      cudaMemsetAsync(jws, 0, (Q + 2) * sizeof(int), st);
      if (skip_items > 0) launch(set_int_kernel, 1, 1, 0, st, jws, skip_items);
      if (ept == 16)
        launch(jacobi_flow_kernel<16>, flow_grid, kJacThreads, 0, st, p->Wj, Q, P, tol, nrm2, rot, jws,
               wait_ns);
      else
        launch(jacobi_flow_kernel<32>, flow_grid, kJacThreads, 0, st, p->Wj, Q, P, tol, nrm2, rot, jws,
               wait_ns);
      return;
    }
    for (int t = 0; t < P - 1; ++t) {
      const dim3 pg((unsigned)(P / 2));
      switch (ept) {
        case 4: launch(jacobi_pair_kernel<4>, pg, kJacThreads, 0, st, p->Wj, Q, P, t, tol, nrm2, rot); break;
        case 8: launch(jacobi_pair_kernel<8>, pg, kJacThreads, 0, st, p->Wj, Q, P, t, tol, nrm2, rot); break;
        case 16: launch(jacobi_pair_kernel<16>, pg, kJacThreads, 0, st, p->Wj, Q, P, t, tol, nrm2, rot); break;
        case 32: launch(jacobi_pair_kernel<32>, pg, kJacThreads, 0, st, p->Wj, Q, P, t, tol, nrm2, rot); break;
        default: launch(jacobi_round_kernel, dim3(rblocks), dim3(256), 0, st, p->Wj, Q, P, t, tol, rot);
      }
    }
  };
  if (P > 1) {
    // The sweep is captured once into a CUDA graph and replayed for every
    // sweep: the same kernels with the same arguments, without the host
    // launch overhead of P - 1 rounds (about 2 us a round).  If the capture
    // fails the sweeps are launched one kernel at a time.
    unsigned long long nodes = 0;
    cudaGraphExec_t sweep_graph = p->graph_sweeps ? capture_graph(st, issue_sweep, &nodes) : nullptr;
    do {
      if (sweep_graph != nullptr) {
        LSRN_CUDA_TRY(cudaGraphLaunch(sweep_graph, st));
        g_kernel_launches.fetch_add(nodes, std::memory_order_relaxed);
      } else {
        issue_sweep();
      }
      LSRN_CUDA_TRY(cudaGetLastError());
      LSRN_CUDA_TRY(cudaMemcpyAsync(&host_rot, rot, sizeof(int), cudaMemcpyDeviceToHost, st));
      int flow_err = 0;
      if (flow)
        LSRN_CUDA_TRY(cudaMemcpyAsync(&flow_err, jws + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      LSRN_CUDA_TRY(cudaStreamSynchronize(st));
      if (flow_err != 0) {   // a dependency wait of the dataflow sweep gave up
        if (sweep_graph != nullptr) cudaGraphExecDestroy(sweep_graph);
        cudaFreeAsync(jws, st);
        return LSRN_ERR_TIMEOUT;
      }
      ++sweeps;
    } while (host_rot > 0 && sweeps < max_sweeps);
    if (sweep_graph != nullptr) cudaGraphExecDestroy(sweep_graph);
  }
  cudaEventRecord(p->ev[9], st);
  if (jws != nullptr) cudaFreeAsync(jws, st);
  p->sweeps = sweeps;
  if (host_rot > 0) return LSRN_ERR_NOT_CONVERGED;
  // 3. sigma, order, rank, N.
  launch(row_norms_kernel, (unsigned)((Q * 32 + 255) / 256), 256, 0, st, p->Wj, Q, p->tmpq);
  const double rcond = p->opt.rcond >= 0.0 ? p->opt.rcond : (double)std::max(S, Q) * 0x1p-53;
  launch(sort_rank_kernel, 1, 1024, 0, st, p->tmpq, Q, rcond, p->perm, p->sig, p->iscal + IC_CAP);
  LSRN_CUDA_TRY(cudaGetLastError());
  int r = 0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&r, p->iscal + IC_CAP, sizeof(int), cudaMemcpyDeviceToHost, st));
  double smax = 0.0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&smax, p->sig, sizeof(double), cudaMemcpyDeviceToHost, st));
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  p->rank = r;
  p->sigma_max = smax;
  p->sigma_min = 0.0;
  if (r > 0) {
    LSRN_CUDA_TRY(cudaMemcpyAsync(&p->sigma_min, p->sig + (r - 1), sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
    const int64_t tot = Q * (int64_t)r;
    launch(form_n_kernel, (unsigned)((tot + 255) / 256), 256, 0, st, p->Wj, Q, p->perm, p->sig, r,
                                                                   p->Nm, p->NT);
    LSRN_CUDA_TRY(cudaGetLastError());
    LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return LSRN_OK;
}

}  // namespace lsrn
