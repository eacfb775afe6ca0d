// Batched preconditioner: Algorithm 1/2 steps 4-5 for many independent
// problems in one launch.
//
// A batch of small problems (short side q <= 128) spends most of its
// preconditioner time in launches: the per-problem path issues a kernel per
// Householder column and per Jacobi round.  Here one persistent launch takes problems from a queue
// (largest first) and gives each one CTA, which runs the whole preconditioner
// with __syncthreads between steps:
//   1. Householder QR of the sketch Xs (S x Q, row-major), one thread per
//      column for the reflector's application (coalesced along the rows);
//   2. one-sided Jacobi on the rows of R with the parallel round-robin order,
//      a warp per pair of rows (the rows in registers, the squared norms in
//      shared memory, Hestenes norm updates, exact norms at each sweep start);
//   3. singular values = row norms, sorted descending, rank r = #{sigma >
//      rcond sigma_1}, N = W_r Sigma_r^-2 and its transpose.
// The arithmetic is that of the per-problem kernels (same reflectors, rotation
// formulas, stopping test and rank rule), so results agree with them to
// rounding.  The FP64 rate of one SM bounds a single problem; the batch keeps
// every SM busy with a different one.
#include <algorithm>
#include <cmath>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int kBT = 512;               // threads per problem (16 warps)
constexpr int kBMaxQ = 512;            // short side handled in one CTA
constexpr int kBWarps = kBT / 32;
constexpr int kBEpt = kBMaxQ / 32;     // row elements per lane in a pair

__device__ double bsum(double v, double* red) {
  v = group_sum<32>(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kBWarps; ++w) t += red[w];
  return t;
}

__device__ void batch_qr(const BatchPrecond& P, double* red, double* sc) {
  double* X = P.X;
  const int64_t S = P.S, Q = P.Q;
  const int tid = threadIdx.x;
  for (int64_t k = 0; k < Q; ++k) {
    double ss = 0.0;
    for (int64_t i = k + 1 + tid; i < S; i += kBT) {
      const double v = X[i * Q + k];
      ss = fma(v, v, ss);
    }
    const double t = bsum(ss, red);
    if (tid == 0) {
      const double alpha = X[k * Q + k];
      double tk = 0.0, scal = 0.0;
      if (t > 0.0) {
        const double nrm = sqrt(alpha * alpha + t);
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        tk = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
        X[k * Q + k] = beta;
      }
      sc[0] = tk;
      sc[1] = scal;
    }
    __syncthreads();
    const double tk = sc[0], scal = sc[1];
    if (tk == 0.0) continue;   // uniform
    for (int64_t i = k + 1 + tid; i < S; i += kBT) X[i * Q + k] *= scal;
    __syncthreads();
    const int64_t c = k + 1 + tid;
    if (c < Q) {
      double w = X[k * Q + c];
      for (int64_t i = k + 1; i < S; ++i) w = fma(X[i * Q + k], X[i * Q + c], w);
      const double tw = tk * w;
      X[k * Q + c] -= tw;
      for (int64_t i = k + 1; i < S; ++i) X[i * Q + c] = fma(-X[i * Q + k], tw, X[i * Q + c]);
    }
    __syncthreads();
  }
}

// returns the number of sweeps (> max_sweeps: not converged)
__device__ int batch_jacobi(const BatchPrecond& P, double* nrm2, int* flag) {
  double* W = P.W;
  const int64_t Q = P.Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t idx = tid; idx < Q * Q; idx += kBT) {
    const int64_t j = idx / Q, c = idx % Q;
    W[idx] = (c >= j) ? P.X[j * Q + c] : 0.0;
  }
  __syncthreads();
  const int Pn = (int)(Q + (Q & 1));
  const double tol = (double)max(P.S, Q) * 0x1p-53;
  const int max_sweeps = 40;
  int sweeps = 0;
  for (;;) {
    // exact squared norms at the start of each sweep, warp per row
    for (int64_t r = warp; r < Q; r += kBWarps) {
      double a = 0.0;
      for (int64_t c = lane; c < Q; c += 32) a = fma(W[r * Q + c], W[r * Q + c], a);
      a = group_sum<32>(a);
      if (lane == 0) nrm2[r] = a;
    }
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int t = 0; t < Pn - 1; ++t) {
      for (int k = warp; k < Pn / 2; k += kBWarps) {
        int a = k == 0 ? Pn - 1 : (t + k) % (Pn - 1);
        int b = k == 0 ? t : (t - k + Pn - 1) % (Pn - 1);
        if (a >= Q || b >= Q) continue;
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        double* wa = W + (int64_t)a * Q;
        double* wb = W + (int64_t)b * Q;
        double x[kBEpt], y[kBEpt];
        double ab = 0.0;
#pragma unroll
        for (int e = 0; e < kBEpt; ++e) {
          const int64_t c = lane + 32 * e;
          x[e] = c < Q ? wa[c] : 0.0;
          y[e] = c < Q ? wb[c] : 0.0;
          ab = fma(x[e], y[e], ab);
        }
        ab = group_sum<32>(ab);
        const double aa = nrm2[a], bb = nrm2[b];
        if (aa == 0.0 || bb == 0.0 || !(fabs(ab) > tol * sqrt(aa) * sqrt(bb))) continue;  // uniform
        const double zeta = (bb - aa) / (2.0 * ab);
        double tt;
        if (fabs(zeta) > 1e150) tt = 0.5 / zeta;
        else tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt);
        const double sn = cs * tt;
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int e = 0; e < kBEpt; ++e) {
          const int64_t c = lane + 32 * e;
          const double xa = cs * x[e] - sn * y[e];
          const double yb = sn * x[e] + cs * y[e];
          x[e] = xa;
          y[e] = yb;
          sa = fma(xa, xa, sa);
          sb = fma(yb, yb, sb);
          if (c < Q) {
            wa[c] = xa;
            wb[c] = yb;
          }
        }
        double na = aa - tt * ab, nb = bb + tt * ab;
        if (na < 0.25 * aa || nb < 0.25 * bb) {   // cancellation: the rotated rows' norms
          na = group_sum<32>(sa);
          nb = group_sum<32>(sb);
        }
        if (lane == 0) {
          nrm2[a] = na;
          nrm2[b] = nb;
          *flag = 1;
        }
      }
      __syncthreads();   // the next round reads rows this one wrote
    }
    ++sweeps;
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) return sweeps;
    if (sweeps >= max_sweeps) return sweeps + 1;
  }
}

__device__ void batch_finish(const BatchPrecond& P, double* nrm, int sweeps, double* red, int* cnt) {
  const int64_t Q = P.Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t r = warp; r < Q; r += kBWarps) {
    double a = 0.0;
    for (int64_t c = lane; c < Q; c += 32) a = fma(P.W[r * Q + c], P.W[r * Q + c], a);
    a = group_sum<32>(a);
    if (lane == 0) nrm[r] = sqrt(a);
  }
  __syncthreads();
  double mx = 0.0;
  for (int64_t j = tid; j < Q; j += kBT) mx = fmax(mx, nrm[j]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  if (tid == 0) *cnt = 0;
  __syncthreads();
  double smax = 0.0;
  for (int w = 0; w < kBWarps; ++w) smax = fmax(smax, red[w]);
  int mine = 0;
  for (int64_t j = tid; j < Q; j += kBT) {   // stable descending position of row j
    const double sj = nrm[j];
    int64_t pos = 0;
    for (int64_t k = 0; k < Q; ++k) {
      const double sk = nrm[k];
      pos += (sk > sj) || (sk == sj && k < j);
    }
    P.perm[pos] = (int)j;
    P.sig[pos] = sj;
    mine += (smax > 0.0 && sj > P.rcond * smax) ? 1 : 0;
  }
  atomicAdd(cnt, mine);
  __syncthreads();
  const int r = *cnt;
  for (int64_t idx = tid; idx < Q * (int64_t)r; idx += kBT) {
    const int64_t k = idx / Q, i = idx % Q;
    const double s = P.sig[k];
    const double v = P.W[(int64_t)P.perm[k] * Q + i] / (s * s);
    P.NT[k * Q + i] = v;
    P.N[i * r + k] = v;
  }
  if (tid == 0) {
    P.out[0] = r;
    P.out[1] = sweeps;
    P.dout[0] = smax;
    P.dout[1] = r > 0 ? P.sig[r - 1] : 0.0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBT, 1) batched_precond_kernel(const BatchPrecond* __restrict__ probs,
                                                                 int count, int* __restrict__ next) {
  __shared__ double red[kBWarps];
  __shared__ double sc[2];
  __shared__ double nrm[kBMaxQ];
  __shared__ int s_idx, s_flag, s_cnt;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_idx = atomicAdd(next, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= count) return;
    const BatchPrecond P = probs[idx];
    batch_qr(P, red, sc);
    const int sweeps = batch_jacobi(P, nrm, &s_flag);
    batch_finish(P, nrm, sweeps, red, &s_cnt);
  }
}

}  // namespace

// One SM's FP64 rate bounds a problem in the batched launch (QR and Jacobi
// ~40 q^3 flop at ~8 GFLOP/s); up to q = 128 that matches the per-problem
// path, whose rounds are launch-bound (~10 ms), so larger problems keep the
// per-problem path (many CTAs per round).
constexpr int64_t kBatchMaxQ = 128;
bool batch_precond_applies(int64_t Q) { return Q >= 1 && Q <= kBatchMaxQ && Q <= kBMaxQ; }

lsrn_status launch_batched_precond(const BatchPrecond* dev_probs, int count, int* dev_next,
                                   cudaStream_t st) {
  if (count <= 0) return LSRN_OK;
  LSRN_CUDA_TRY(cudaMemsetAsync(dev_next, 0, sizeof(int), st));
  const int grid = std::max(1, std::min(count, num_sms()));
  launch(batched_precond_kernel, grid, kBT, 0, st, dev_probs, count, dev_next);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
