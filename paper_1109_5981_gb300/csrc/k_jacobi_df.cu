// Double-float pre-sweeps of the one-sided Jacobi SVD (Algorithm 1/2 step 4).
//
// GB300 runs FP32 arithmetic about 64 times faster than FP64, and the FP64
// sweeps of the preconditioner are bound by the FP64 pipe.  So the early
// sweeps, where almost every pair rotates, run on a copy of R held as
// double-float pairs (hi + lo, two FP32 values, ~2^-46 relative):
//   1. W = R and P = I, both q x q double-float;
//   2. dataflow sweeps (the same round-robin order and stopping rule as the FP64
//      sweeps, tolerance max(s, q) 2^-44) rotate the rows a, b of W and, with
//      the same rotation, the rows a, b of P, so W = P R holds throughout;
//   3. Y = P R in FP64 from the exact R, which replaces R for the FP64 sweeps.
// P is orthogonal up to ~1e-12, so Y = P R has the singular values of R up to
// that relative factor (sigma_i(P R) lies between sigma_i(R) sigma_min(P) and
// sigma_i(R) sigma_max(P)), and its rows are orthogonal to ~2^-46 relative, so
// the FP64 sweeps converge quadratically from there: usually one sweep with
// rotations and one without.  From the FP64 result W' = J^T Y with orthogonal
// rows, N = W'_r^T Sigma_r^-2 gives R N = P^-1 J[:, :r]: the same N formula,
// and A N has the singular values of the FP64 path up to cond(P).
//
// Double-float arithmetic (Dekker's two-product via FMA, Knuth's two-sum):
// a rotated element c x + s y costs 19 FP32 operations, a dot-product term
// 12; rotation angles, squared norms and the stopping test stay in FP64
// (one thread per pair).
#include <algorithm>
#include <cmath>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int kDfThreads = 256;
constexpr uint64_t kDfWaitNs = 1000000000ull;   // one second per dependency wait

__device__ __forceinline__ uint64_t df_globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int df_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void df_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// c x + s y for double-float c, x, s, y (hi in .x, lo in .y)
__device__ __forceinline__ float2 df_lin(float2 c, float2 x, float2 s, float2 y) {
  const float p1 = c.x * x.x;
  const float e1 = fmaf(c.x, x.x, -p1);
  const float p2 = s.x * y.x;
  const float e2 = fmaf(s.x, y.x, -p2);
  const float sm = p1 + p2;               // two-sum of the leading products
  const float bv = sm - p1;
  const float er = (p1 - (sm - bv)) + (p2 - bv);
  float lo = (e1 + e2) + er;
  lo = fmaf(c.x, x.y, lo);
  lo = fmaf(c.y, x.x, lo);
  lo = fmaf(s.x, y.y, lo);
  lo = fmaf(s.y, y.x, lo);
  const float hi = sm + lo;               // renormalise
  return make_float2(hi, lo - (hi - sm));
}

// (S, E) += x y for double-float x, y
__device__ __forceinline__ void df_dot_acc(float2 x, float2 y, float& S, float& E) {
  const float p = x.x * y.x;
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  const float s = S + p;
  const float bv = s - S;
  E += ((S - (s - bv)) + (p - bv)) + e;
  S = s;
}

__device__ __forceinline__ float2 df_from(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// (h, l) += (bh, bl), double-float
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float bv = s - h;
  float e = (h - (s - bv)) + (bh - bv);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

// Sum of the threads' double-float (S, E) over the CTA, in double-float on the
// FP32 pipe (on GB300 a warp-wide FP64 instruction costs 16 cycles of an SM's
// FP64 throughput, so the reduction stays off that pipe); the FP64 value is
// returned to thread 0 only.
__device__ __forceinline__ double df_block_sum0(float S, float E, float2* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, S, o);
    const float ol = __shfl_xor_sync(0xffffffffu, E, o);
    df_add(S, E, oh, ol);
  }
  __syncthreads();   // sh may still be read from the previous sum
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(S, E);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kDfThreads / 32; ++w) t += (double)sh[w].x + (double)sh[w].y;
  }
  return t;
}

// W = upper triangle of X (ld Q) as double-float, P = I
__global__ void df_init_kernel(const double* __restrict__ X, int64_t Q, float2* __restrict__ W,
                               float2* __restrict__ Pm) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Q * Q) return;
  const int64_t j = idx / Q, c = idx % Q;
  W[idx] = c >= j ? df_from(X[j * Q + c]) : make_float2(0.f, 0.f);
  Pm[idx] = make_float2(j == c ? 1.f : 0.f, 0.f);
}

// nrm2[row] = ||W[row]||^2 in FP64 (hi + lo is exact in FP64), warp per row
__global__ void df_row_sqnorms_kernel(const float2* __restrict__ W, int64_t Q, double* __restrict__ nrm2) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= Q) return;
  double acc = 0.0;
  for (int64_t c = lane; c < Q; c += 32) {
    const float2 v = W[row * Q + c];
    const double x = (double)v.x + (double)v.y;
    acc = fma(x, x, acc);
  }
  acc = group_sum<32>(acc);
  if (lane == 0) nrm2[row] = acc;
}

// One dataflow sweep (item i = t * (P/2) + k is pair k of round t; an item
// waits, bounded by wait_ns of global time, until its two rows have finished
// round t - 1).  ws[0]: next item, ws[1]: error flag, ws[2 + row]: ver[row].
template <int EPT>
__global__ void __launch_bounds__(kDfThreads, EPT >= 16 ? 1 : 2)
    jacobi_df_flow_kernel(float2* __restrict__ W, float2* __restrict__ Pm, int64_t Q, int P, double tol,
                          double* __restrict__ nrm2, int* __restrict__ rot_count, int* __restrict__ ws,
                          uint64_t wait_ns) {
  __shared__ float2 sh[kDfThreads / 32];
  __shared__ float2 s_cs, s_sn;
  __shared__ int s_item, s_ok, s_rot, s_rec;
  int* next = ws;
  int* err = ws + 1;
  int* ver = ws + 2;
  const int npairs = P / 2;
  const int total = (P - 1) * npairs;
  for (;;) {
    __syncthreads();   // the previous item is done with the shared scalars
    if (threadIdx.x == 0) {
      const int item = atomicAdd(next, 1);
      int ok = 0;
      if (item < total && df_ld_acquire(err) == 0) {
        const int t = item / npairs, k = item % npairs;
        const int a = k == 0 ? P - 1 : (t + k) % (P - 1);
        const int b = k == 0 ? t : (t - k + P - 1) % (P - 1);
        ok = 1;
        const uint64_t t0 = df_globaltimer_ns();
        for (int it = 0;; ++it) {
          const bool ra = a >= Q || df_ld_acquire(ver + a) >= t;
          const bool rb = b >= Q || df_ld_acquire(ver + b) >= t;
          if (ra && rb) break;
          if ((it & 15) == 15 && (df_globaltimer_ns() - t0 > wait_ns || df_ld_acquire(err) != 0)) {
            atomicExch(err, 1);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
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
    if (a >= Q || b >= Q) {
      if (threadIdx.x == 0) {
        const int r = a < Q ? a : b;
        if (r < Q) df_st_release(ver + r, t + 1);
      }
      continue;
    }
    if (a > b) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    float2* wa = W + (int64_t)a * Q;
    float2* wb = W + (int64_t)b * Q;
    float2* pa = Pm + (int64_t)a * Q;
    float2* pb = Pm + (int64_t)b * Q;
    const double aa = __ldcg(nrm2 + a), bb = __ldcg(nrm2 + b);
    float2 x[EPT], y[EPT];
    float S = 0.f, E = 0.f;
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int64_t c = threadIdx.x + (int64_t)kDfThreads * e;
      x[e] = c < Q ? __ldcg(wa + c) : z;
      y[e] = c < Q ? __ldcg(wb + c) : z;
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) df_dot_acc(x[e], y[e], S, E);
    const double ab = df_block_sum0(S, E, sh);   // thread 0 only
    double na = aa, nb = bb;                     // thread 0: the new squared norms
    if (threadIdx.x == 0) {
      double tt = 0.0, cs = 1.0;
      if (aa != 0.0 && bb != 0.0 && fabs(ab) > tol * sqrt(aa) * sqrt(bb)) {
        const double zeta = (bb - aa) / (2.0 * ab);
        if (fabs(zeta) > 1e150) {
          tt = 0.5 / zeta;
        } else {
          tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        }
        cs = 1.0 / sqrt(1.0 + tt * tt);
      }
      na = aa - tt * ab;
      nb = bb + tt * ab;
      s_rot = tt != 0.0;
      s_rec = tt != 0.0 && (na < 0.25 * aa || nb < 0.25 * bb);   // cancellation: recompute
      s_cs = df_from(cs);
      s_sn = df_from(cs * tt);
    }
    __syncthreads();
    if (s_rot) {   // uniform
      const float2 cs = s_cs, sn = s_sn;
      const float2 msn = make_float2(-sn.x, -sn.y);
      float Sa = 0.f, Ea = 0.f, Sb = 0.f, Eb = 0.f;
      float2 u[EPT], v[EPT];   // rows a, b of P: read only for a pair that rotates
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int64_t c = threadIdx.x + (int64_t)kDfThreads * e;
        u[e] = c < Q ? __ldcg(pa + c) : z;
        v[e] = c < Q ? __ldcg(pb + c) : z;
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int64_t c = threadIdx.x + (int64_t)kDfThreads * e;
        const float2 xa = df_lin(cs, x[e], msn, y[e]);
        const float2 yb = df_lin(sn, x[e], cs, y[e]);
        const float2 ua = df_lin(cs, u[e], msn, v[e]);
        const float2 vb = df_lin(sn, u[e], cs, v[e]);
        x[e] = xa;
        y[e] = yb;
        if (c < Q) {
          wa[c] = xa;
          wb[c] = yb;
          pa[c] = ua;
          pb[c] = vb;
        }
      }
      if (s_rec) {   // uniform
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          df_dot_acc(x[e], x[e], Sa, Ea);
          df_dot_acc(y[e], y[e], Sb, Eb);
        }
        const double ra = df_block_sum0(Sa, Ea, sh);
        const double rb = df_block_sum0(Sb, Eb, sh);
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
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      df_st_release(ver + a, t + 1);
      df_st_release(ver + b, t + 1);
    }
  }
}

// Y = P R in FP64: P double-float (q x q), R the upper triangle of X (ld q).
// 64 x 64 output tile per CTA (4 x 4 per thread), K in steps of 32; R[k, c] = 0
// for k > c, so a tile's K range ends at its last column.
__global__ void __launch_bounds__(256) df_times_r_kernel(const float2* __restrict__ Pm,
                                                         const double* __restrict__ X, int64_t Q,
                                                         double* __restrict__ Y) {
  __shared__ double sp[64][33];
  __shared__ double sr[32][65];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  const int tr = tid >> 4, tc = tid & 15;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int64_t kend = std::min<int64_t>(Q, c0 + 64);
  for (int64_t ks = 0; ks < kend; ks += 32) {
    for (int t = tid; t < 64 * 32; t += 256) {
      const int rr = t >> 5, kk = t & 31;
      const int64_t i = i0 + rr, k = ks + kk;
      double v = 0.0;
      if (i < Q && k < Q) {
        const float2 f = Pm[i * Q + k];
        v = (double)f.x + (double)f.y;
      }
      sp[rr][kk] = v;
    }
    for (int t = tid; t < 32 * 64; t += 256) {
      const int kk = t >> 6, cc = t & 63;
      const int64_t k = ks + kk, c = c0 + cc;
      sr[kk][cc] = (k < Q && c < Q && k <= c) ? X[k * Q + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      double pv[4], rv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pv[a] = sp[tr + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) rv[b] = sr[kk][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(pv[a], rv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tr + 16 * a;
    if (i >= Q) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tc + 16 * b;
      if (c < Q) Y[i * Q + c] = acc[a][b];
    }
  }
}

__global__ void df_set_int_kernel(int* __restrict__ p, int v) { *p = v; }

}  // namespace

bool jacobi_df_applies(int64_t Q) { return Q > 1024 && Q <= 4096; }

// The double-float phase: sweeps on (W, P) from R = upper triangle of Xs until
// none rotates (at most 30), then Y = P R into Wj.  Returns LSRN_ERR_TIMEOUT
// if a dependency wait gave up; *sweeps counts the sweeps run.
lsrn_status jacobi_df_phase(Plan* p, int64_t wait_ns_knob, int skip_items, int* sweeps_out) {
  cudaStream_t st = p->stream;
  const int64_t S = p->s, Q = p->q;
  const int P = (int)(Q + (Q & 1));
  const double tol = (double)std::max(S, Q) * 0x1p-44;
  const uint64_t wait_ns = wait_ns_knob > 0 ? (uint64_t)wait_ns_knob : kDfWaitNs;
  const int ept = Q <= 2048 ? 8 : 16;
  *sweeps_out = 0;
  float2* Wd = nullptr;
  int* jws = nullptr;
  const size_t qq = (size_t)Q * (size_t)Q;
  LSRN_CUDA_TRY(lsrn_malloc_async((void**)&Wd, 2 * qq * sizeof(float2), st));
  lsrn_status rs = lsrn_malloc_async((void**)&jws, (size_t)(Q + 2) * sizeof(int), st) == cudaSuccess
                       ? LSRN_OK
                       : LSRN_ERR_CUDA;
  if (rs != LSRN_OK) {
    cudaFreeAsync(Wd, st);
    return rs;
  }
  float2* Pd = Wd + qq;
  double* nrm2 = p->tmpq;
  int* rot = p->iscal + IC_ROT;
  launch(df_init_kernel, (unsigned)((qq + 255) / 256), 256, 0, st, (const double*)p->Xs, Q, Wd, Pd);
  int per_sm = 0;
  if (ept == 8)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_df_flow_kernel<8>, kDfThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_df_flow_kernel<16>, kDfThreads, 0);
  const int64_t items = (int64_t)(P - 1) * (P / 2);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * num_sms(), items));
  int host_rot = 1, sweeps = 0;
  while (host_rot > 0 && sweeps < 30 && rs == LSRN_OK) {
    cudaMemsetAsync(rot, 0, sizeof(int), st);
    launch(df_row_sqnorms_kernel, (unsigned)((Q * 32 + 255) / 256), 256, 0, st, (const float2*)Wd, Q, nrm2);
    cudaMemsetAsync(jws, 0, (size_t)(Q + 2) * sizeof(int), st);
    if (skip_items > 0) launch(df_set_int_kernel, 1, 1, 0, st, jws, skip_items);
    if (ept == 8)
      launch(jacobi_df_flow_kernel<8>, grid, kDfThreads, 0, st, Wd, Pd, Q, P, tol, nrm2, rot, jws, wait_ns);
    else
      launch(jacobi_df_flow_kernel<16>, grid, kDfThreads, 0, st, Wd, Pd, Q, P, tol, nrm2, rot, jws, wait_ns);
    int flow_err = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&host_rot, rot, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&flow_err, jws + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rs = LSRN_ERR_CUDA;
      break;
    }
    if (flow_err != 0) rs = LSRN_ERR_TIMEOUT;
    ++sweeps;
  }
  if (rs == LSRN_OK) {
    const unsigned tiles = (unsigned)((Q + 63) / 64);
    launch(df_times_r_kernel, dim3(tiles, tiles), 256, 0, st, (const float2*)Pd, (const double*)p->Xs, Q,
           p->Wj);
    if (cudaGetLastError() != cudaSuccess) rs = LSRN_ERR_CUDA;
  }
  cudaFreeAsync(jws, st);
  cudaFreeAsync(Wd, st);
  *sweeps_out = sweeps;
  return rs;
}

}  // namespace lsrn
