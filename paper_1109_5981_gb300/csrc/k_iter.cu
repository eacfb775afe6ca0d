// Iteration kernels (Algorithm 1/2 step 6 with LSQR or Algorithm 3).
//
// The fused pass streams the row-major matrix X (A for m >= n, A^T for m < n)
// once and, per row i, forms the dot product d_i = X_i . vin, turns it into a
// row coefficient t_i (the row mode: an LSQR or Chebyshev update of the state
// held for that row), and accumulates sum_i t_i X_i.  One HBM pass therefore
// applies both X and X^T: for m >= n it computes A(Nv) and A^T u in one go,
// for m < n A^T(Mu) and A t.  Per-CTA partial vectors are summed in a fixed
// order by a second kernel, so results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int kThreads = 256;

struct Coef {
  double c0, c1;
};

// Row coefficient t_i from the dot d = X_i . vin and the row's state values
// (s0, s1 read before any thread of the row group writes them).  Returns the
// multiplier of X_i in the accumulated vector; the writer thread stores the
// updated state.
__device__ __forceinline__ double row_coef(const RowArgs& a, const Coef& k, int64_t i, double d,
                                           double s0, double s1, bool writer, double& ss) {
  double t = 0.0;
  switch (a.mode) {
    case RM_ACC_STATE:
      return s0;
    case RM_LSQR_TALL:
      t = d - k.c0 * s0;
      if (writer) a.st0[i] = t;
      ss = fma(t, t, ss);
      return t;
    case RM_CS_TALL:
      t = s0 - k.c0 * d;
      if (writer) a.st0[i] = t;
      ss = fma(t, t, ss);
      return t;
    case RM_APPLY:
      return d;
    case RM_FAT_INIT:
      t = a.sx * d;
      if (writer) a.st0[i] = t;
      ss = fma(t, t, ss);
      return a.sx * t;
    case RM_FAT_LSQR:
      t = a.sx * d - k.c0 * s0;
      if (writer) a.st0[i] = t;
      ss = fma(t, t, ss);
      return a.sx * t;
    case RM_FAT_CS:
      t = k.c0 * s0 + a.sx * d;
      if (writer) {
        a.st0[i] = t;
        a.st1[i] = fma(k.c1, t, s1);
      }
      return a.sx * t;
  }
  return 0.0;
}

__device__ __forceinline__ bool mode_reads_st0(int mode) {
  return mode == RM_ACC_STATE || mode == RM_LSQR_TALL || mode == RM_CS_TALL ||
         mode == RM_FAT_LSQR || mode == RM_FAT_CS;
}

// TPR threads cover one row (2 * TPR * SLOTS columns max); R rows per step per group.
template <class T>
__device__ __forceinline__ void load_pair(const T* p, T& x, T& y);
template <>
__device__ __forceinline__ void load_pair<double>(const double* p, double& x, double& y) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  x = v.x;
  y = v.y;
}
template <>
__device__ __forceinline__ void load_pair<float>(const float* p, float& x, float& y) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  x = v.x;
  y = v.y;
}

// T = double: FP64 pass over A; T = float: the same pass over an FP32 copy of A
// with FP32 products and per-thread sums (row sums, coefficients and partials
// in FP64).
template <class T, int TPR, int SLOTS, int R>
__global__ void __launch_bounds__(kThreads) row_pass_kernel(const T* __restrict__ X, int64_t rows,
                                                            int C, int64_t ldx,
                                                            const double* __restrict__ vin,
                                                            RowArgs args, double* __restrict__ pvec,
                                                            double* __restrict__ pscal,
                                                            const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  constexpr int GPC = kThreads / TPR;
  constexpr int WPG = TPR / 32 > 0 ? TPR / 32 : 1;   // warps per group (TPR >= 32)
  __shared__ double red[2][kThreads / 32][R];
  __shared__ double cta_acc[(GPC > 1) ? GPC : 1][(GPC > 1) ? 2 * TPR * SLOTS : 1];
  __shared__ double sred[kThreads / 32];
  const int tid = threadIdx.x, gid = tid / TPR, gl = tid % TPR;
  const bool need_dot = args.mode != RM_ACC_STATE;
  const bool reads0 = mode_reads_st0(args.mode);
  const bool reads1 = args.mode == RM_FAT_CS;
  Coef k{0.0, 0.0};
  if (args.coef) {
    k.c0 = args.coef[0];
    k.c1 = args.coef[1];
  }
  T w[SLOTS][2], acc[SLOTS][2];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * gl + 2 * TPR * s;
    w[s][0] = (need_dot && c < C) ? (T)vin[c] : (T)0;
    w[s][1] = (need_dot && c + 1 < C) ? (T)vin[c + 1] : (T)0;
    acc[s][0] = acc[s][1] = (T)0;
  }
  double ss = 0.0;
  const int64_t step = (int64_t)gridDim.x * GPC * R;
  int buf = 0;
  // rows of the next step are loaded while the current ones are reduced and
  // accumulated (register double buffering keeps HBM requests in flight)
  auto load_rows = [&](T (&dst)[R][SLOTS][2], int64_t b) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = b + gid * R + r;
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int c = 2 * gl + 2 * TPR * s;
        if (i < rows && c + 1 < C) {
          load_pair<T>(X + i * ldx + c, dst[r][s][0], dst[r][s][1]);
        } else if (i < rows && c < C) {
          dst[r][s][0] = X[i * ldx + c];
          dst[r][s][1] = (T)0;
        } else {
          dst[r][s][0] = dst[r][s][1] = (T)0;
        }
      }
    }
  };
  T a[R][SLOTS][2], an[R][SLOTS][2];
  load_rows(a, (int64_t)blockIdx.x * GPC * R);
  for (int64_t base = (int64_t)blockIdx.x * GPC * R; base < rows; base += step) {
    load_rows(an, base + step);
    // row state, read by every thread of the group before the barrier below;
    // the group's writer updates it only after that barrier
    double s0v[R], s1v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = base + gid * R + r;
      s0v[r] = (i < rows && reads0) ? args.st0[i] : 0.0;
      s1v[r] = (i < rows && reads1) ? args.st1[i] : 0.0;
    }
    double d[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T t = (T)0;
      if (need_dot) {
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) t = fma(a[r][s][0], w[s][0], fma(a[r][s][1], w[s][1], t));
      }
      d[r] = (double)t;
    }
    if (need_dot) {
      if (TPR <= 32) {
#pragma unroll
        for (int r = 0; r < R; ++r) d[r] = group_sum<(TPR < 32 ? TPR : 32)>(d[r]);
        __syncwarp();
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) d[r] = group_sum<32>(d[r]);
        if ((tid & 31) == 0) {
#pragma unroll
          for (int r = 0; r < R; ++r) red[buf][tid >> 5][r] = d[r];
        }
        __syncthreads();
        const int w0 = gid * WPG;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          double t = 0.0;
          for (int q = 0; q < WPG; ++q) t += red[buf][w0 + q][r];
          d[r] = t;
        }
        buf ^= 1;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = base + gid * R + r;
      double tacc = 0.0;
      if (i < rows) {
        double ss_dummy = 0.0;
        tacc = row_coef(args, k, i, d[r], s0v[r], s1v[r], gl == 0, gl == 0 ? ss : ss_dummy);
      }
      const T tc = (T)tacc;
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        acc[s][0] = fma(tc, a[r][s][0], acc[s][0]);
        acc[s][1] = fma(tc, a[r][s][1], acc[s][1]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        a[r][s][0] = an[r][s][0];
        a[r][s][1] = an[r][s][1];
      }
  }
  // combine the groups of this CTA and write the CTA's partial vector
  double* out = pvec + (int64_t)blockIdx.x * C;
  if (GPC > 1) {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int c = 2 * gl + 2 * TPR * s;
      cta_acc[gid][2 * TPR * s + 2 * gl] = (double)acc[s][0];
      cta_acc[gid][2 * TPR * s + 2 * gl + 1] = (double)acc[s][1];
      (void)c;
    }
    __syncthreads();
    for (int c = tid; c < C; c += kThreads) {
      double t = 0.0;
      for (int g = 0; g < GPC; ++g) t += cta_acc[g][c];
      out[c] = t;
    }
  } else {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int c = 2 * gl + 2 * TPR * s;
      if (c < C) out[c] = (double)acc[s][0];
      if (c + 1 < C) out[c + 1] = (double)acc[s][1];
    }
  }
  ss = group_sum<32>(ss);
  if ((tid & 31) == 0) sred[tid >> 5] = ss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += sred[q];
    pscal[blockIdx.x] = t;
  }
}

// ---- staged variant for wide rows ------------------------------------------
// One persistent CTA per SM streams blocks of RB rows of X through a ring of
// shared-memory stages filled by bulk asynchronous copies (cp.async.bulk with
// mbarrier transaction counts), so ~150 KB per SM are in flight while earlier
// stages are reduced and accumulated.  The rows' LSQR/CS state (st0, st1)
// travels with them.  Same arithmetic and outputs as row_pass_kernel.
constexpr int kMaxStages = 8;
constexpr long long kPassSpinLimit = 1ll << 26;

__device__ __forceinline__ uint32_t sm_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sm_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kPassSpinLimit; ++it)
    if (bar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          sm_u32(dst)),
      "l"(src), "r"(bytes), "r"(sm_u32(bar))
      : "memory");
}

template <class T, int SLOTS, int RB>
__global__ void __launch_bounds__(kThreads, 1) row_pass_staged_kernel(
    const T* __restrict__ X, int64_t rows, int C, int64_t ldx, const double* __restrict__ vin,
    RowArgs args, double* __restrict__ pvec, double* __restrict__ pscal, const int* __restrict__ done,
    int* __restrict__ err, int rowbytes, int nstages) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double red[2][kThreads / 32][RB];
  __shared__ double tco[2][RB];
  __shared__ double sred[kThreads / 32];
  const int tid = threadIdx.x;
  const bool need_dot = args.mode != RM_ACC_STATE;
  const bool reads0 = mode_reads_st0(args.mode);
  const bool reads1 = args.mode == RM_FAT_CS;
  const int stage_bytes = RB * rowbytes;
  double* state = (double*)(smem + (size_t)nstages * stage_bytes);   // [nstages][2][RB]
  Coef k{0.0, 0.0};
  if (args.coef) {
    k.c0 = args.coef[0];
    k.c1 = args.coef[1];
  }
  T w[SLOTS][2], acc[SLOTS][2];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * tid + 2 * kThreads * s;
    w[s][0] = (need_dot && c < C) ? (T)vin[c] : (T)0;
    w[s][1] = (need_dot && c + 1 < C) ? (T)vin[c + 1] : (T)0;
    acc[s][0] = acc[s][1] = (T)0;
  }
  const int64_t nrb = (rows + RB - 1) / RB;
  const int64_t my_n = blockIdx.x < nrb ? (nrb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (tid == 0) {
    for (int st = 0; st < nstages; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_u32(&bars[st])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t kk) {
    if (tid != 0 || kk >= my_n) return;
    const int st = (int)(kk % nstages);
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    const int nr = (int)min((int64_t)RB, rows - r0);
    const uint32_t sbytes = (uint32_t)(((nr * 8) + 15) / 16 * 16);
    uint32_t bytes = (uint32_t)nr * rowbytes + (reads0 ? sbytes : 0u) + (reads1 ? sbytes : 0u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(&bars[st])),
                 "r"(bytes)
                 : "memory");
    unsigned char* dst = smem + (size_t)st * stage_bytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before async writes
    for (int r = 0; r < nr; ++r)
      bulk_copy(dst + (size_t)r * rowbytes, X + (r0 + r) * ldx, (uint32_t)rowbytes, &bars[st]);
    if (reads0) bulk_copy(state + (size_t)st * 2 * RB, args.st0 + r0, sbytes, &bars[st]);
    if (reads1) bulk_copy(state + (size_t)st * 2 * RB + RB, args.st1 + r0, sbytes, &bars[st]);
  };
  for (int kk = 0; kk < nstages - 1; ++kk) issue(kk);
  double ss = 0.0;
  int buf = 0;
  bool ok = true;
  int64_t kk = 0;
  for (; kk < my_n; ++kk) {
    issue(kk + nstages - 1);
    const int st = (int)(kk % nstages);
    if (!bar_wait(&bars[st], (uint32_t)((kk / nstages) & 1))) {
      ok = false;
      break;
    }
    const T* rowp = (const T*)(smem + (size_t)st * stage_bytes);
    const double* sst = state + (size_t)st * 2 * RB;
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    // dot products: per-thread partials in T, warp sums in T, cross-warp sum and
    // the row's LSQR/CS update by one thread per row (FP64), broadcast via smem
    // rows past the end of X (last block) hold stale shared memory: skipped
    const int nr = (int)min((int64_t)RB, rows - r0);
    T dp[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      T t = (T)0;
      if (need_dot && r < nr) {
        const T* row = rowp + (size_t)r * (rowbytes / sizeof(T));
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int c = 2 * tid + 2 * kThreads * s;
          if (c < C) {
            T x0, x1;
            load_pair<T>(row + c, x0, x1);
            if (c + 1 >= C) x1 = (T)0;
            t = fma(x0, w[s][0], fma(x1, w[s][1], t));
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      }
      dp[r] = t;
    }
    if ((tid & 31) == 0) {
#pragma unroll
      for (int r = 0; r < RB; ++r) red[buf][tid >> 5][r] = (double)dp[r];
    }
    __syncthreads();
    if (tid < RB) {
      const int r = tid;
      const int64_t i = r0 + r;
      double tacc = 0.0;
      if (i < rows) {
        double d = 0.0;
        if (need_dot)
          for (int q = 0; q < kThreads / 32; ++q) d += red[buf][q][r];
        const double s0 = reads0 ? sst[r] : 0.0;
        const double s1 = reads1 ? sst[RB + r] : 0.0;
        tacc = row_coef(args, k, i, d, s0, s1, true, ss);
      }
      tco[buf][r] = tacc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r >= nr) break;
      const T tc = (T)tco[buf][r];
      const T* row = rowp + (size_t)r * (rowbytes / sizeof(T));
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int c = 2 * tid + 2 * kThreads * s;
        if (c < C) {
          T x0, x1;
          load_pair<T>(row + c, x0, x1);
          if (c + 1 >= C) x1 = (T)0;
          acc[s][0] = fma(tc, x0, acc[s][0]);
          acc[s][1] = fma(tc, x1, acc[s][1]);
        }
      }
    }
    buf ^= 1;
    __syncthreads();   // stage st is free again
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let copies already issued land before the CTA exits
    for (int64_t q = kk; q < my_n && q < kk + nstages - 1; ++q)
      bar_wait(&bars[q % nstages], (uint32_t)((q / nstages) & 1));
  }
  double* out = pvec + (int64_t)blockIdx.x * C;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * tid + 2 * kThreads * s;
    if (c < C) out[c] = (double)acc[s][0];
    if (c + 1 < C) out[c + 1] = (double)acc[s][1];
  }
  ss = group_sum<32>(ss);
  if ((tid & 31) == 0) sred[tid >> 5] = ss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += sred[q];
    pscal[blockIdx.x] = t;
  }
}

// ---- double-float variant (iteration mode LSRN_ITER_F32X2) ------------------
// X is held as two FP32 planes, Xh = fl32(X / xs) and Xl = fl32(X / xs - Xh)
// with one power-of-two scale xs, so Xh + Xl carries 48 significant bits of
// each element.  Every element operation runs on the FP32 pipe with
// error-free transformations: the product of two (hi, lo) pairs is
// TwoProd(hi, hi) plus the two cross terms, and sums are TwoSum into
// (hi, lo) accumulators.  Only the per-row LSQR/CS update (one thread per
// row) is FP64.  Same staging, row modes and outputs as row_pass_staged_kernel.
//
// Range: vin enters as vin / 2^ve with ve the exponent of max |vin| (per CTA);
// row coefficients enter as t / 2^E with a running exponent E shared by the
// CTA.  E is raised when a row's |t| would exceed 2^(E + 60); the column
// accumulators are folded into FP64 (times 2^E) before it changes, and every
// kFoldRows rows, which also bounds the error of their lazy low words.  Only
// contributions below 2^-126 of the largest vin entry or row coefficient lose
// bits.
constexpr int kFoldRows = 256;
constexpr int kNoExp = -100000;

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Packed pairs: two FP32 lanes in one 64-bit register, operated on by the
// f32x2 instructions (one issue slot for both lanes, each lane rounded as the
// scalar IEEE operation).  The pass handles columns in (even, odd) pairs, so
// the error-free transformations above run on both columns of a pair at once.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float x, float y) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 upk2(f32x2 r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// (h, l) += (ah + al) * (bh + bl) lane by lane, dropping al * bl (below 2^-48
// of the product): p = fl(ah bh) and its exact error by an FMA, the cross
// terms into that error, TwoSum(h, p) with the rounding error into l.  bhn =
// -bh, so the negated product comes from one multiply and the TwoSum uses it
// directly.
__device__ __forceinline__ void df_fma2(f32x2 ah, f32x2 al, f32x2 bh, f32x2 bhn, f32x2 bl,
                                        f32x2& h, f32x2& l) {
  const f32x2 np = mul2(ah, bhn);                       // -p, p = ah bh rounded
  f32x2 e = fma2(ah, bh, np);                           // ah bh - p, exact
  e = fma2(ah, bl, fma2(al, bh, e));
  const f32x2 s = sub2(h, np);                          // TwoSum(h, p)
  const f32x2 bb = sub2(s, h);
  const f32x2 er = sub2(sub2(h, sub2(s, bb)), add2(np, bb));
  h = s;
  l = add2(l, add2(er, e));
}

__device__ __forceinline__ void split_df(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}
__device__ __forceinline__ int exp_of(double x) {   // ilogb for finite nonzero x, else kNoExp
  return (x != 0.0 && isfinite(x)) ? ilogb(x) : kNoExp;
}

// Named barriers of the pipelined pass (0 is __syncthreads).
constexpr int kBarDot = 1;     // + parity: partial dots of a stage are in shared memory
constexpr int kBarCoef = 3;    // + parity: row coefficients of a stage are in shared memory
constexpr int kBarFree = 5;    // compute warps are done with a stage
constexpr int kX2Threads = kThreads + 32;
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Warp-specialised: warps 0-7 compute the partial dots of stage k while warp 8
// turns the dots of stage k - 1 into row coefficients (FP64, one lane per row),
// then warps 0-7 accumulate stage k - 1.  The FP64 row update is thus off the
// compute warps' critical path.
template <int SLOTS, int RB>
__global__ void __launch_bounds__(kX2Threads, (RB == 2 && SLOTS <= 4) ? 3 : 1) row_pass_x2_kernel(
    const float* __restrict__ Xh, const float* __restrict__ Xl, int64_t rows, int C, int64_t ldx,
    double xs, const double* __restrict__ vin, RowArgs args, double* __restrict__ pvec,
    double* __restrict__ pscal, const int* __restrict__ done, int* __restrict__ err, int rowbytes,
    int nstages) {
  static_assert(RB * (kThreads / 32) <= 32, "one coefficient-warp lane per (row, warp) partial");
  if (done != nullptr && *done) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ float redh[2][RB][kThreads / 32], redl[2][RB][kThreads / 32];
  __shared__ float tch[2][RB], tcl[2][RB];
  __shared__ int texp[2];
  __shared__ int vexp[kThreads / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const bool coef_warp = tid >= kThreads;
  const bool need_dot = args.mode != RM_ACC_STATE;
  const bool reads0 = mode_reads_st0(args.mode);
  const bool reads1 = args.mode == RM_FAT_CS;
  const int stage_bytes = 2 * RB * rowbytes;   // RB rows of Xh, then RB rows of Xl
  double* state = (double*)(smem + (size_t)nstages * stage_bytes);   // [nstages][2][RB]
  const int rstride = rowbytes / (int)sizeof(float);
  Coef k{0.0, 0.0};
  if (args.coef) {
    k.c0 = args.coef[0];
    k.c1 = args.coef[1];
  }
  // exponent of max |vin| over the whole vector (compute threads see their slots)
  double vv[SLOTS][2];
  int ve = kNoExp;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = 2 * tid + 2 * kThreads * s + e;
      vv[s][e] = (!coef_warp && need_dot && c < C) ? vin[c] : 0.0;
      ve = max(ve, exp_of(vv[s][e]));
    }
  for (int o = 16; o > 0; o >>= 1) ve = max(ve, __shfl_xor_sync(0xffffffffu, ve, o));
  if (!coef_warp && (tid & 31) == 0) vexp[tid >> 5] = ve;
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < nstages; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_u32(&bars[st])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  ve = kNoExp;
  for (int q = 0; q < kThreads / 32; ++q) ve = max(ve, vexp[q]);
  if (ve == kNoExp) ve = 0;
  const double dscale = ldexp(xs, ve);
  const int64_t nrb = (rows + RB - 1) / RB;
  const int64_t my_n = blockIdx.x < nrb ? (nrb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  int64_t issued_upto = -1, waited_upto = -1;   // bookkeeping of thread 0 (the producer)
  auto issue = [&](int64_t kk) {
    if (tid != 0 || kk >= my_n || abort_flag != 0) return;
    issued_upto = kk;
    const int st = (int)(kk % nstages);
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    const int nr = (int)min((int64_t)RB, rows - r0);
    const uint32_t sbytes = (uint32_t)(((nr * 8) + 15) / 16 * 16);
    uint32_t bytes = 2u * (uint32_t)nr * rowbytes + (reads0 ? sbytes : 0u) + (reads1 ? sbytes : 0u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(&bars[st])),
                 "r"(bytes)
                 : "memory");
    unsigned char* dst = smem + (size_t)st * stage_bytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int r = 0; r < nr; ++r) {
      bulk_copy(dst + (size_t)r * rowbytes, Xh + (r0 + r) * ldx, (uint32_t)rowbytes, &bars[st]);
      bulk_copy(dst + (size_t)(RB + r) * rowbytes, Xl + (r0 + r) * ldx, (uint32_t)rowbytes,
                &bars[st]);
    }
    if (reads0) bulk_copy(state + (size_t)st * 2 * RB, args.st0 + r0, sbytes, &bars[st]);
    if (reads1) bulk_copy(state + (size_t)st * 2 * RB + RB, args.st1 + r0, sbytes, &bars[st]);
  };
  int E = kNoExp;   // running exponent of the row coefficients (same in every thread)

  if (coef_warp) {
    // ---- coefficient warp: lane = (row r, partial q) for the cross-warp sums ----
    const int lane = tid - kThreads;
    const int rq = lane / (kThreads / 32), qq = lane % (kThreads / 32);
    double ss = 0.0;
    for (int64_t kk = 0; kk < my_n; ++kk) {
      const int par = (int)(kk & 1);
      named_sync(kBarDot + par, kX2Threads);
      const int st = (int)(kk % nstages);
      const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
      const int nr = (int)min((int64_t)RB, rows - r0);
      const bool aborted = abort_flag != 0;
      // the stage's state words came by bulk copy: observe its completed phase
      if (!aborted && (reads0 || reads1)) bar_wait(&bars[st], (uint32_t)((kk / nstages) & 1));
      float h = 0.0f, l = 0.0f;
      if (need_dot && rq < RB) {
        h = redh[par][rq][qq];
        l = redl[par][rq][qq];
      }
#pragma unroll
      for (int o = (kThreads / 32) / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        float sum, er;
        two_sum_f(h, oh, sum, er);
        h = sum;
        l += ol + er;
      }
      double tacc = 0.0;
      const bool owner = qq == 0 && rq < nr && !aborted;
      if (owner) {
        const int64_t i = r0 + rq;
        const double d = need_dot ? dscale * ((double)h + (double)l) : 0.0;
        const double* sst = state + (size_t)st * 2 * RB;
        const double s0 = reads0 ? sst[rq] : 0.0;
        const double s1 = reads1 ? sst[RB + rq] : 0.0;
        tacc = row_coef(args, k, i, d, s0, s1, true, ss);
      }
      int me = exp_of(tacc);
      for (int o = 16; o > 0; o >>= 1) me = max(me, __shfl_xor_sync(0xffffffffu, me, o));
      if (me != kNoExp && (E == kNoExp || me > E + 60)) E = me;
      if (qq == 0 && rq < RB) {
        float th = 0.0f, tl = 0.0f;
        if (owner && E != kNoExp) split_df(ldexp(tacc, -E), th, tl);
        tch[par][rq] = th;
        tcl[par][rq] = tl;
      }
      if (lane == 0) texp[par] = E;
      __threadfence_block();
      named_arrive(kBarCoef + par, kX2Threads);
    }
    ss = group_sum<32>(ss);
    if (lane == 0) pscal[blockIdx.x] = ss;
    return;
  }

  // ---- compute warps ----
  // (even, odd) column pairs: vin as packed (hi, lo) and -hi, the column
  // accumulators as packed (hi, lo), folded into FP64 wd
  f32x2 vh[SLOTS], vhn[SLOTS], vl[SLOTS], wh[SLOTS], wl[SLOTS];
  double wd[SLOTS][2];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    float h0, l0, h1, l1;
    split_df(ldexp(vv[s][0], -ve), h0, l0);
    split_df(ldexp(vv[s][1], -ve), h1, l1);
    vh[s] = pk2(h0, h1);
    vhn[s] = pk2(-h0, -h1);
    vl[s] = pk2(l0, l1);
    wh[s] = wl[s] = 0ull;   // +0.0f in both lanes
    wd[s][0] = wd[s][1] = 0.0;
  }
  double escale = 0.0;
  int since_fold = 0;
  auto fold = [&]() {
    if (E != kNoExp) {
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const float2 h = upk2(wh[s]), l = upk2(wl[s]);
        wd[s][0] += escale * ((double)h.x + (double)l.x);
        wd[s][1] += escale * ((double)h.y + (double)l.y);
        wh[s] = wl[s] = 0ull;
      }
    }
    since_fold = 0;
  };
  auto accumulate = [&](int64_t kk) {
    const int par = (int)(kk & 1);
    named_sync(kBarCoef + par, kX2Threads);
    const int En = texp[par];
    if (En != E) {
      fold();
      E = En;
      escale = ldexp(xs, E);
    }
    const int st = (int)(kk % nstages);
    const float* hp = (const float*)(smem + (size_t)st * stage_bytes);
    const float* lp = hp + (size_t)RB * rstride;
    const int nr = (int)min((int64_t)RB, rows - (blockIdx.x + kk * gridDim.x) * RB);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r >= nr) break;
      const float th = tch[par][r], tl = tcl[par][r];
      const f32x2 th2 = pk2(th, th), thn2 = pk2(-th, -th), tl2 = pk2(tl, tl);
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int c = 2 * tid + 2 * kThreads * s;
        if (c < C) {
          const f32x2 a = *reinterpret_cast<const f32x2*>(hp + (size_t)r * rstride + c);
          const f32x2 b = *reinterpret_cast<const f32x2*>(lp + (size_t)r * rstride + c);
          df_fma2(a, b, th2, thn2, tl2, wh[s], wl[s]);
        }
      }
    }
    since_fold += RB;
    if (since_fold >= kFoldRows) fold();
  };
  for (int kk = 0; kk < nstages; ++kk) issue(kk);
  for (int64_t kk = 0; kk < my_n; ++kk) {
    const int par = (int)(kk & 1);
    const int st = (int)(kk % nstages);
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    const int nr = (int)min((int64_t)RB, rows - r0);
    bool have = abort_flag == 0;
    if (have && !bar_wait(&bars[st], (uint32_t)((kk / nstages) & 1))) {
      abort_flag = 1;   // later waits and copies are skipped; the barrier sequence continues
      have = false;
    }
    if (have && tid == 0) waited_upto = kk;
    if (need_dot) {
      const float* hp = (const float*)(smem + (size_t)st * stage_bytes);
      const float* lp = hp + (size_t)RB * rstride;
      // all rows' chains first (independent), then one transposed butterfly
      f32x2 h2[RB], l2[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) h2[r] = l2[r] = 0ull;
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int c = 2 * tid + 2 * kThreads * s;
        if (have && c < C) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            if (r < nr) {
              const f32x2 a = *reinterpret_cast<const f32x2*>(hp + (size_t)r * rstride + c);
              const f32x2 b = *reinterpret_cast<const f32x2*>(lp + (size_t)r * rstride + c);
              df_fma2(a, b, vh[s], vhn[s], vl[s], h2[r], l2[r]);   // vin is 0 past C
            }
          }
        }
      }
      float h[RB], l[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const float2 hh = upk2(h2[r]), ll = upk2(l2[r]);
        float sum, er;
        two_sum_f(hh.x, hh.y, sum, er);
        h[r] = sum;
        l[r] = ll.x + (ll.y + er);
      }
      // transposed butterfly: at width w each lane keeps half of its rows and adds the
      // partner's copy of them, until one row per lane group remains
      const int lane = tid & 31;
      int nrow = RB, w = 16;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        if (nrow > 1) {
          const bool upper = (lane & w) != 0;
          const int half = nrow / 2;
#pragma unroll
          for (int j = 0; j < RB / 2; ++j) {
            if (j < half) {
              const float sh = upper ? h[j] : h[j + half];   // rows the partner keeps
              const float sl = upper ? l[j] : l[j + half];
              const float kh = upper ? h[j + half] : h[j];   // rows this lane keeps
              const float kl = upper ? l[j + half] : l[j];
              const float oh = __shfl_xor_sync(0xffffffffu, sh, w);
              const float ol = __shfl_xor_sync(0xffffffffu, sl, w);
              float sum, er;
              two_sum_f(kh, oh, sum, er);
              h[j] = sum;
              l[j] = kl + (ol + er);
            }
          }
          nrow = half;
        } else {
          const float oh = __shfl_xor_sync(0xffffffffu, h[0], w);
          const float ol = __shfl_xor_sync(0xffffffffu, l[0], w);
          float sum, er;
          two_sum_f(h[0], oh, sum, er);
          h[0] = sum;
          l[0] = l[0] + (ol + er);
        }
        w >>= 1;
      }
      // lane groups of 32 / RB lanes hold row r = lane / (32 / RB)
      if ((lane & (32 / RB - 1)) == 0) {
        const int r = lane / (32 / RB);
        redh[par][r][tid >> 5] = h[0];
        redl[par][r][tid >> 5] = l[0];
      }
    }
    __threadfence_block();
    named_arrive(kBarDot + par, kX2Threads);
    if (kk >= 1) {
      accumulate(kk - 1);
      named_sync(kBarFree, kThreads);   // stage (kk - 1) may be refilled
      issue(kk - 1 + nstages);
    }
  }
  if (my_n >= 1) accumulate(my_n - 1);
  if (tid == 0 && abort_flag != 0) {
    atomicExch(err, 1);
    // copies issued but not observed must land before the CTA exits
    for (int64_t q = waited_upto + 1; q <= issued_upto; ++q)
      bar_wait(&bars[q % nstages], (uint32_t)((q / nstages) & 1));
  }
  fold();
  double* out = pvec + (int64_t)blockIdx.x * C;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * tid + 2 * kThreads * s;
    if (c < C) out[c] = wd[s][0];
    if (c + 1 < C) out[c + 1] = wd[s][1];
  }
}

// ---- triple-float residual pass (refinement in iteration mode LSRN_ITER_F32X2) ----
// With a third plane X3 = fl32(X / xs - Xh - Xl), Xh + Xl + X3 equals X / xs
// exactly (X3 holds the last <= 6 bits).  The refinement's residual pass
// r_i = b_i - X_i . v (m >= n) and g = sum_i t_i X_i then runs on the FP32 pipe:
// every product of two exact three-float values keeps its terms down to
// 2^-48 of the leading product (TwoProd for the two leading weights), sums are
// TwoSum chains into three-float accumulators, and column sums are folded into
// double-double every kFoldRows rows.  The result matches the FP64
// double-double pass to ~2^-65 of sum |terms|.
__device__ __forceinline__ void split_tf(double v, float& a, float& b, float& c) {
  a = __double2float_rn(v);
  const double r = v - (double)a;
  b = __double2float_rn(r);
  c = __double2float_rn(r - (double)b);
}
// (h, m, l) += (a1 + a2 + a3)(b1 + b2 + b3), terms below 2^-48 of a1 b1 dropped
__device__ __forceinline__ void tf_fma(float a1, float a2, float a3, float b1, float b2, float b3,
                                       float& h, float& m, float& l) {
  const float p0 = a1 * b1;
  const float e0 = fmaf(a1, b1, -p0);
  const float p1 = a1 * b2;
  const float e1 = fmaf(a1, b2, -p1);
  const float p2 = a2 * b1;
  const float e2 = fmaf(a2, b1, -p2);
  const float q = fmaf(a1, b3, fmaf(a2, b2, fmaf(a3, b1, e1 + e2)));
  float s, c, t, d;
  two_sum_f(h, p0, s, c);
  h = s;
  two_sum_f(m, p1, t, d);
  m = t;
  l += d;
  two_sum_f(m, p2, t, d);
  m = t;
  l += d;
  two_sum_f(m, e0, t, d);
  m = t;
  l += d;
  two_sum_f(m, c, t, d);
  m = t;
  l += d + q;
}
__device__ __forceinline__ void tf_combine(float& h, float& m, float& l, float oh, float om, float ol) {
  float s, c, t, d, d2;
  two_sum_f(h, oh, s, c);
  h = s;
  two_sum_f(m, om, t, d);
  two_sum_f(t, c, m, d2);
  l += ol + d + d2;
}
// (h + m + l) as double-double
__device__ __forceinline__ void tf_to_dd(float h, float m, float l, double& dh, double& dl) {
  two_sum((double)h, (double)m, dh, dl);
  dd_add(dh, dl, (double)l, 0.0);
}

template <int SLOTS, int RB>
__global__ void __launch_bounds__(kX2Threads, 1) dd_pass_x3_kernel(
    const float* __restrict__ Xh, const float* __restrict__ Xl, const float* __restrict__ X3,
    int64_t rows, int C, int64_t ldx, double xs, const double* __restrict__ vin,
    const double* __restrict__ rowvec, double sx, int tall, double* __restrict__ rout,
    double* __restrict__ phi, double* __restrict__ plo, int* __restrict__ err, int planebytes,
    int nstages) {
  static_assert(RB * (kThreads / 32) <= 32, "one coefficient-warp lane per (row, warp) partial");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ float redh[2][RB][kThreads / 32], redm[2][RB][kThreads / 32], redl[2][RB][kThreads / 32];
  __shared__ float tc1[2][RB], tc2[2][RB], tc3[2][RB];
  __shared__ int texp[2];
  __shared__ int vexp[kThreads / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const bool coef_warp = tid >= kThreads;
  const int stage_bytes = 3 * RB * planebytes;   // RB rows of Xh, of Xl, of X3
  double* state = (double*)(smem + (size_t)nstages * stage_bytes);   // [nstages][RB]
  const int rstride = planebytes / (int)sizeof(float);
  double vv[SLOTS][2];
  int ve = kNoExp;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = 2 * tid + 2 * kThreads * s + e;
      vv[s][e] = (!coef_warp && tall && c < C) ? vin[c] : 0.0;
      ve = max(ve, exp_of(vv[s][e]));
    }
  for (int o = 16; o > 0; o >>= 1) ve = max(ve, __shfl_xor_sync(0xffffffffu, ve, o));
  if (!coef_warp && (tid & 31) == 0) vexp[tid >> 5] = ve;
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < nstages; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_u32(&bars[st])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  ve = kNoExp;
  for (int q = 0; q < kThreads / 32; ++q) ve = max(ve, vexp[q]);
  if (ve == kNoExp) ve = 0;
  const double dscale = ldexp(xs, ve);
  const int64_t nrb = (rows + RB - 1) / RB;
  const int64_t my_n = blockIdx.x < nrb ? (nrb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  int64_t issued_upto = -1, waited_upto = -1;
  auto issue = [&](int64_t kk) {
    if (tid != 0 || kk >= my_n || abort_flag != 0) return;
    issued_upto = kk;
    const int st = (int)(kk % nstages);
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    const int nr = (int)min((int64_t)RB, rows - r0);
    const uint32_t sbytes = (uint32_t)(((nr * 8) + 15) / 16 * 16);
    const uint32_t bytes = 3u * (uint32_t)nr * planebytes + sbytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(&bars[st])),
                 "r"(bytes)
                 : "memory");
    unsigned char* dst = smem + (size_t)st * stage_bytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int r = 0; r < nr; ++r) {
      bulk_copy(dst + (size_t)r * planebytes, Xh + (r0 + r) * ldx, (uint32_t)planebytes, &bars[st]);
      bulk_copy(dst + (size_t)(RB + r) * planebytes, Xl + (r0 + r) * ldx, (uint32_t)planebytes,
                &bars[st]);
      bulk_copy(dst + (size_t)(2 * RB + r) * planebytes, X3 + (r0 + r) * ldx,
                (uint32_t)planebytes, &bars[st]);
    }
    bulk_copy(state + (size_t)st * RB, rowvec + r0, sbytes, &bars[st]);
  };
  int E = kNoExp;

  if (coef_warp) {
    const int lane = tid - kThreads;
    const int rq = lane / (kThreads / 32), qq = lane % (kThreads / 32);
    for (int64_t kk = 0; kk < my_n; ++kk) {
      const int par = (int)(kk & 1);
      named_sync(kBarDot + par, kX2Threads);
      const int st = (int)(kk % nstages);
      const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
      const int nr = (int)min((int64_t)RB, rows - r0);
      const bool aborted = abort_flag != 0;
      if (!aborted) bar_wait(&bars[st], (uint32_t)((kk / nstages) & 1));
      float h = 0.0f, m = 0.0f, l = 0.0f;
      if (tall && rq < RB) {
        h = redh[par][rq][qq];
        m = redm[par][rq][qq];
        l = redl[par][rq][qq];
      }
#pragma unroll
      for (int o = (kThreads / 32) / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float om = __shfl_xor_sync(0xffffffffu, m, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        tf_combine(h, m, l, oh, om, ol);
      }
      double t = 0.0;
      const bool owner = qq == 0 && rq < nr && !aborted;
      if (owner) {
        const double sv = state[(size_t)st * RB + rq];
        if (tall) {
          double dh, dl;
          tf_to_dd(h, m, l, dh, dl);
          double rh = sv, rl = 0.0;
          dd_add(rh, rl, -dscale * dh, -dscale * dl);
          t = rh + rl;
          rout[r0 + rq] = t;
        } else {
          t = sx * sv;
        }
      }
      int me = exp_of(t);
      for (int o = 16; o > 0; o >>= 1) me = max(me, __shfl_xor_sync(0xffffffffu, me, o));
      if (me != kNoExp && (E == kNoExp || me > E + 60)) E = me;
      if (qq == 0 && rq < RB) {
        float a = 0.0f, b = 0.0f, c = 0.0f;
        if (owner && E != kNoExp) split_tf(ldexp(t, -E), a, b, c);
        tc1[par][rq] = a;
        tc2[par][rq] = b;
        tc3[par][rq] = c;
      }
      if (lane == 0) texp[par] = E;
      __threadfence_block();
      named_arrive(kBarCoef + par, kX2Threads);
    }
    return;
  }

  float v1[SLOTS][2], v2[SLOTS][2], v3[SLOTS][2];
  float wh[SLOTS][2], wm[SLOTS][2], wl[SLOTS][2];
  double gh[SLOTS][2], gl[SLOTS][2];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      split_tf(ldexp(vv[s][e], -ve), v1[s][e], v2[s][e], v3[s][e]);
      wh[s][e] = wm[s][e] = wl[s][e] = 0.0f;
      gh[s][e] = gl[s][e] = 0.0;
    }
  double escale = 0.0;
  int since_fold = 0;
  auto fold = [&]() {
    if (E != kNoExp) {
#pragma unroll
      for (int s = 0; s < SLOTS; ++s)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          double dh, dl;
          tf_to_dd(wh[s][e], wm[s][e], wl[s][e], dh, dl);
          dd_add(gh[s][e], gl[s][e], escale * dh, escale * dl);
          wh[s][e] = wm[s][e] = wl[s][e] = 0.0f;
        }
    }
    since_fold = 0;
  };
  auto accumulate = [&](int64_t kk) {
    const int par = (int)(kk & 1);
    named_sync(kBarCoef + par, kX2Threads);
    const int En = texp[par];
    if (En != E) {
      fold();
      E = En;
      escale = ldexp(xs, E);
    }
    const int st = (int)(kk % nstages);
    const float* hp = (const float*)(smem + (size_t)st * stage_bytes);
    const float* lp = hp + (size_t)RB * rstride;
    const float* tp = hp + (size_t)2 * RB * rstride;
    const int nr = (int)min((int64_t)RB, rows - (blockIdx.x + kk * gridDim.x) * RB);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r >= nr) break;
      const float t1 = tc1[par][r], t2 = tc2[par][r], t3 = tc3[par][r];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int c = 2 * tid + 2 * kThreads * s;
        if (c < C) {
          const float2 a = *reinterpret_cast<const float2*>(hp + (size_t)r * rstride + c);
          const float2 b = *reinterpret_cast<const float2*>(lp + (size_t)r * rstride + c);
          const float2 d = *reinterpret_cast<const float2*>(tp + (size_t)r * rstride + c);
          tf_fma(t1, t2, t3, a.x, b.x, d.x, wh[s][0], wm[s][0], wl[s][0]);
          tf_fma(t1, t2, t3, a.y, b.y, d.y, wh[s][1], wm[s][1], wl[s][1]);
        }
      }
    }
    since_fold += RB;
    if (since_fold >= kFoldRows) fold();
  };
  for (int kk = 0; kk < nstages; ++kk) issue(kk);
  for (int64_t kk = 0; kk < my_n; ++kk) {
    const int par = (int)(kk & 1);
    const int st = (int)(kk % nstages);
    const int64_t r0 = (blockIdx.x + kk * gridDim.x) * RB;
    const int nr = (int)min((int64_t)RB, rows - r0);
    bool have = abort_flag == 0;
    if (have && !bar_wait(&bars[st], (uint32_t)((kk / nstages) & 1))) {
      abort_flag = 1;
      have = false;
    }
    if (have && tid == 0) waited_upto = kk;
    if (tall) {
      const float* hp = (const float*)(smem + (size_t)st * stage_bytes);
      const float* lp = hp + (size_t)RB * rstride;
      const float* tp = hp + (size_t)2 * RB * rstride;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        float h = 0.0f, m = 0.0f, l = 0.0f;
        if (have && r < nr) {
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) {
            const int c = 2 * tid + 2 * kThreads * s;
            if (c < C) {
              const float2 a = *reinterpret_cast<const float2*>(hp + (size_t)r * rstride + c);
              const float2 b = *reinterpret_cast<const float2*>(lp + (size_t)r * rstride + c);
              const float2 d = *reinterpret_cast<const float2*>(tp + (size_t)r * rstride + c);
              tf_fma(a.x, b.x, d.x, v1[s][0], v2[s][0], v3[s][0], h, m, l);
              tf_fma(a.y, b.y, d.y, v1[s][1], v2[s][1], v3[s][1], h, m, l);
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, h, o);
          const float om = __shfl_xor_sync(0xffffffffu, m, o);
          const float ol = __shfl_xor_sync(0xffffffffu, l, o);
          tf_combine(h, m, l, oh, om, ol);
        }
        if ((tid & 31) == 0) {
          redh[par][r][tid >> 5] = h;
          redm[par][r][tid >> 5] = m;
          redl[par][r][tid >> 5] = l;
        }
      }
    }
    __threadfence_block();
    named_arrive(kBarDot + par, kX2Threads);
    if (kk >= 1) {
      accumulate(kk - 1);
      named_sync(kBarFree, kThreads);
      issue(kk - 1 + nstages);
    }
  }
  if (my_n >= 1) accumulate(my_n - 1);
  if (tid == 0 && abort_flag != 0) {
    atomicExch(err, 1);
    for (int64_t q = waited_upto + 1; q <= issued_upto; ++q)
      bar_wait(&bars[q % nstages], (uint32_t)((q / nstages) & 1));
  }
  fold();
  double* oh = phi + (int64_t)blockIdx.x * C;
  double* ol = plo + (int64_t)blockIdx.x * C;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * tid + 2 * kThreads * s;
    if (c < C) {
      oh[c] = gh[s][0];
      ol[c] = gl[s][0];
    }
    if (c + 1 < C) {
      oh[c + 1] = gh[s][1];
      ol[c + 1] = gl[s][1];
    }
  }
}

// Rows appended to X by the Tikhonov augmentation: row (xrows + j) = coef * e_j.
// Writes one extra partial slot (vector of length C and one scalar).
__global__ void extra_rows_kernel(int64_t nextra, int64_t xrows, int C, double coef,
                                  const double* __restrict__ vin, RowArgs args,
                                  double* __restrict__ pvec_slot, double* __restrict__ pscal_slot,
                                  const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ double sred[32];
  Coef k{0.0, 0.0};
  if (args.coef) {
    k.c0 = args.coef[0];
    k.c1 = args.coef[1];
  }
  RowArgs a1 = args;
  a1.sx = 1.0;   // appended rows are coef * e_j, never scaled by 1/lambda
  const bool need_dot = args.mode != RM_ACC_STATE;
  double ss = 0.0;
  for (int64_t j = threadIdx.x; j < C; j += blockDim.x) {
    double v = 0.0;
    if (j < nextra) {
      const double d = need_dot ? coef * vin[j] : 0.0;
      const int64_t i = xrows + j;
      const double s0 = mode_reads_st0(a1.mode) ? a1.st0[i] : 0.0;
      const double s1 = a1.mode == RM_FAT_CS ? a1.st1[i] : 0.0;
      const double t = row_coef(a1, k, i, d, s0, s1, true, ss);
      v = coef * t;
    }
    pvec_slot[j] = v;
  }
  ss = group_sum<32>(ss);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += sred[q];
    *pscal_slot = t;
  }
}

// Double-double pass: m >= n: r_i = b_i - X_i . vin (dd), acc += r_i X_i (dd);
// m < n (bvec == nullptr): acc += (sx * vin_row[i]) X_i (dd), no dot.
template <int TPR, int SLOTS>
__global__ void __launch_bounds__(kThreads) dd_pass_kernel(const double* __restrict__ X, int64_t rows,
                                                           int C, int64_t ldx,
                                                           const double* __restrict__ vin,
                                                           const double* __restrict__ bvec,
                                                           double* __restrict__ rout, double sx,
                                                           double* __restrict__ phi,
                                                           double* __restrict__ plo) {
  constexpr int GPC = kThreads / TPR;
  constexpr int WPG = TPR / 32 > 0 ? TPR / 32 : 1;
  __shared__ double redh[2][kThreads / 32], redl[2][kThreads / 32];
  __shared__ double cta_h[(GPC > 1) ? GPC : 1][(GPC > 1) ? 2 * TPR * SLOTS : 1];
  __shared__ double cta_l[(GPC > 1) ? GPC : 1][(GPC > 1) ? 2 * TPR * SLOTS : 1];
  const int tid = threadIdx.x, gid = tid / TPR, gl = tid % TPR;
  const bool tall = bvec != nullptr;
  double w[SLOTS][2], ah[SLOTS][2], al[SLOTS][2];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int c = 2 * gl + 2 * TPR * s;
    w[s][0] = (tall && c < C) ? vin[c] : 0.0;
    w[s][1] = (tall && c + 1 < C) ? vin[c + 1] : 0.0;
    ah[s][0] = ah[s][1] = al[s][0] = al[s][1] = 0.0;
  }
  const int64_t step = (int64_t)gridDim.x * GPC;
  int buf = 0;
  for (int64_t base = (int64_t)blockIdx.x * GPC; base < rows; base += step) {
    const int64_t i = base + gid;
    double a[SLOTS][2];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int c = 2 * gl + 2 * TPR * s;
      a[s][0] = (i < rows && c < C) ? X[i * ldx + c] : 0.0;
      a[s][1] = (i < rows && c + 1 < C) ? X[i * ldx + c + 1] : 0.0;
    }
    double t = 0.0;
    if (tall) {
      double hi = 0.0, lo = 0.0;
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        dd_add_prod(hi, lo, -a[s][0], w[s][0]);
        dd_add_prod(hi, lo, -a[s][1], w[s][1]);
      }
      if (TPR <= 32) {
        group_sum_dd<(TPR < 32 ? TPR : 32)>(hi, lo);
      } else {
        group_sum_dd<32>(hi, lo);
        if ((tid & 31) == 0) {
          redh[buf][tid >> 5] = hi;
          redl[buf][tid >> 5] = lo;
        }
        __syncthreads();
        hi = 0.0;
        lo = 0.0;
        for (int q = 0; q < WPG; ++q) dd_add(hi, lo, redh[buf][gid * WPG + q], redl[buf][gid * WPG + q]);
        buf ^= 1;
      }
      if (i < rows) {
        dd_add(hi, lo, bvec[i], 0.0);
        t = hi + lo;
        if (gl == 0) rout[i] = t;
      }
    } else if (i < rows) {
      t = sx * vin[i];
    }
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      dd_add_prod(ah[s][0], al[s][0], t, a[s][0]);
      dd_add_prod(ah[s][1], al[s][1], t, a[s][1]);
    }
  }
  double* oh = phi + (int64_t)blockIdx.x * C;
  double* ol = plo + (int64_t)blockIdx.x * C;
  if (GPC > 1) {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      cta_h[gid][2 * TPR * s + 2 * gl] = ah[s][0];
      cta_h[gid][2 * TPR * s + 2 * gl + 1] = ah[s][1];
      cta_l[gid][2 * TPR * s + 2 * gl] = al[s][0];
      cta_l[gid][2 * TPR * s + 2 * gl + 1] = al[s][1];
    }
    __syncthreads();
    for (int c = tid; c < C; c += kThreads) {
      double h = 0.0, l = 0.0;
      for (int g = 0; g < GPC; ++g) dd_add(h, l, cta_h[g][c], cta_l[g][c]);
      oh[c] = h;
      ol[c] = l;
    }
  } else {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int c = 2 * gl + 2 * TPR * s;
      if (c < C) {
        oh[c] = ah[s][0];
        ol[c] = al[s][0];
      }
      if (c + 1 < C) {
        oh[c + 1] = ah[s][1];
        ol[c + 1] = al[s][1];
      }
    }
  }
}

// Extra (ridge) rows of the double-double pass, written as one more partial slot.
//  m >= n: row xrows+j = coef e_j: r = 0 - coef x_j, acc_j += coef * r
//  m <  n: row xrows+i = e_i:      acc_i += vin_row[xrows + i]
__global__ void dd_extra_kernel(int64_t nextra, int64_t xrows, int C, double coef,
                                const double* __restrict__ vin, bool tall,
                                double* __restrict__ rout, double* __restrict__ ph,
                                double* __restrict__ pl) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    double h = 0.0, l = 0.0;
    if (j < nextra) {
      if (tall) {
        double rh = 0.0, rl = 0.0;
        dd_add_prod(rh, rl, -coef, vin[j]);
        const double r = rh + rl;
        rout[xrows + j] = r;
        dd_add_prod(h, l, coef, r);
      } else {
        h = vin[xrows + j];
      }
    }
    ph[j] = h;
    pl[j] = l;
  }
}

__global__ void reduce_kernel(const double* __restrict__ pvec, int nslots, int64_t C,
                              double* __restrict__ out, const double* __restrict__ pscal,
                              double* __restrict__ scal_out, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
    double t = 0.0;
    for (int s = 0; s < nslots; ++s) t += pvec[(int64_t)s * C + c];
    out[c] = t;
  }
  if (scal_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (int s = 0; s < nslots; ++s) t += pscal[s];
    *scal_out = t;
  }
}

__global__ void reduce_dd_kernel(const double* __restrict__ ph, const double* __restrict__ pl,
                                 int nslots, int64_t C, double* __restrict__ oh,
                                 double* __restrict__ ol) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double h = 0.0, l = 0.0;
  for (int s = 0; s < nslots; ++s) dd_add(h, l, ph[(int64_t)s * C + c], pl[(int64_t)s * C + c]);
  oh[c] = h;
  if (ol) ol[c] = l;
}

// Warp per row: out[i] = c0 * (M_i . v) + c1 * y[i]; y2[i] += c2 * out[i].
__global__ void __launch_bounds__(256) gemv_kernel(const double* __restrict__ M, int64_t R, int64_t C,
                                                   const double* __restrict__ v, double* out,
                                                   const double* y, double* y2,
                                                   const double* __restrict__ c,
                                                   const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= R) return;
  const double* m = M + row * C;
  double acc = 0.0;
  for (int64_t j = lane; j < C; j += 32) acc = fma(m[j], v[j], acc);
  acc = group_sum<32>(acc);
  if (lane == 0) {
    double o = c[0] * acc;
    if (y) o = fma(c[1], y[row], o);
    out[row] = o;
    if (y2) y2[row] = fma(c[2], o, y2[row]);
  }
}

// Warp per row, double-double accumulation: out[i] = round(M_i . v).
__global__ void __launch_bounds__(256) gemv_dd_kernel(const double* __restrict__ M, int64_t R,
                                                      int64_t C, const double* __restrict__ v,
                                                      double* __restrict__ out) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= R) return;
  const double* m = M + row * C;
  double hi = 0.0, lo = 0.0;
  for (int64_t j = lane; j < C; j += 32) dd_add_prod(hi, lo, m[j], v[j]);
  group_sum_dd<32>(hi, lo);
  if (lane == 0) out[row] = hi + lo;
}

}  // namespace

lsrn_status launch_gemv_dd(const double* M, int64_t R, int64_t C, const double* v, double* out,
                           cudaStream_t st) {
  if (R == 0) return LSRN_OK;
  launch(gemv_dd_kernel, (unsigned)((R * 32 + 255) / 256), 256, 0, st, M, R, C, v, out);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

namespace {
__global__ void to_f32_kernel(const double* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                              float* __restrict__ Y, int64_t ldy) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * ldy) return;
  const int64_t i = idx / ldy, j = idx % ldy;
  Y[idx] = j < cols ? (float)X[i * ldx + j] : 0.0f;
}
// The conversion kernels below walk X row by row: a group of TPR threads (a
// power of two, 32..256) per row, 256 / TPR rows per block and pass, blocks
// striding over the rows, so no element index needs a 64-bit division.  VEC = 2
// moves two neighbouring columns per access (16-byte loads of X, 8-byte stores
// of the FP32 planes); it needs X 16-byte aligned and cols and ldx even.

// |x| as a key whose unsigned order is the order of the values (non-negative
// doubles order like their bit patterns); NaN gets key 0, so it is skipped.
// Integer compares keep the FP64 pipe, a few instructions per clock per SM on
// this part, out of a pass that is meant to stream at HBM speed.
__device__ __forceinline__ unsigned long long abs_key(double x) {
  const unsigned long long b =
      (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return b > 0x7ff0000000000000ull ? 0ull : b;
}

// Largest |X_ij| as the bit pattern of a non-negative double (ordered like the value).
template <int VEC>
__global__ void __launch_bounds__(256) maxabs_kernel(const double* __restrict__ X, int64_t rows,
                                                     int64_t cols, int64_t ldx, int tpr_log2,
                                                     unsigned long long* __restrict__ out) {
  __shared__ unsigned long long sm[8];
  const int tpr = 1 << tpr_log2, rpb = 256 >> tpr_log2;
  const int t = (int)threadIdx.x & (tpr - 1);
  const int64_t nv = cols / VEC;
  unsigned long long mx = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * rpb + (threadIdx.x >> tpr_log2); i < rows;
       i += (int64_t)gridDim.x * rpb) {
    const double* x = X + i * ldx;
#pragma unroll 4
    for (int64_t p = t; p < nv; p += tpr) {
      if constexpr (VEC == 2) {
        const double2 v = reinterpret_cast<const double2*>(x)[p];
        const unsigned long long a = abs_key(v.x), b = abs_key(v.y);
        mx = a > mx ? a : mx;
        mx = b > mx ? b : mx;
      } else {
        const unsigned long long a = abs_key(x[p]);
        mx = a > mx ? a : mx;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < 8; ++q) mx = sm[q] > mx ? sm[q] : mx;
    atomicMax(out, mx);
  }
}

// Xh = fl32(X * inv), Xl = fl32(X * inv - Xh), X3 = fl32(X * inv - Xh - Xl) (exact);
// zero padding for cols <= j < ldy.
struct Split3 {
  float h, l, e;
};
__device__ __forceinline__ Split3 split3(double x, double inv) {
  const double v = x * inv;
  const float h = __double2float_rn(v);
  const double r = v - (double)h;
  const float l = __double2float_rn(r);
  return {h, l, __double2float_rn(r - (double)l)};
}

// The same split on the integer and FP32 pipes.  v = x 2^k with exponent E;
// when every bit of v lies at or above 2^-126 (E >= -74, the significand has
// 53 bits) and E <= 126, h, l and e are normal floats or zeros, and rounding
// to float is rounding the 53-bit significand M to 24 bits to nearest, ties
// to even: h = RN24(M) 2^(E-52), r = M - RN24(M) (|r| <= 2^28, an int32),
// l = RN24(r) 2^(E-52) (the int-to-float conversion rounds the same way), e =
// (r - RN24(r)) 2^(E-52) (at most 5 bits, exact).  All scalings are by powers
// of two into the normal range, hence exact.  Other x (zero, subnormal, tiny
// after scaling, Inf, NaN) and a scale that is not a normal power of two take
// split3 itself.
__device__ __forceinline__ Split3 split3_int(double x, double inv, int k, bool pow2) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  const int E = ex - 1023 + k;
  if (!pow2 || ex == 0 || ex == 0x7ff || E < -74 || E > 126) return split3(x, inv);
  const long long M = (b & 0xfffffffffffffll) | 0x10000000000000ll;
  long long q = M >> 29;
  const int rem = (int)(M & 0x1fffffff);
  q += (rem > (1 << 28) || (rem == (1 << 28) && (q & 1))) ? 1 : 0;
  int r = (int)(M - (q << 29));
  const bool neg = b < 0;
  if (neg) r = -r;
  const float lf = __int2float_rn(r);
  const int e = r - __float2int_rz(lf);
  const float s52 = __int_as_float((E - 52 + 127) << 23);   // 2^(E-52), >= 2^-126
  const float s23 = __int_as_float((E - 23 + 127) << 23);   // 2^(E-23)
  const float hf = __int2float_rn((int)q) * s23;
  return {neg ? -hf : hf, lf * s52, __int2float_rn(e) * s52};
}

template <int VEC>
__global__ void __launch_bounds__(256, 4) to_x2_kernel(const double* __restrict__ X, int64_t rows,
                                                    int64_t cols, int64_t ldx, double inv,
                                                    int k, bool pow2, int tpr_log2,
                                                    float* __restrict__ Yh, float* __restrict__ Yl,
                                                    float* __restrict__ Y3, int64_t ldy) {
  const int tpr = 1 << tpr_log2, rpb = 256 >> tpr_log2;
  const int t = (int)threadIdx.x & (tpr - 1);
  const int64_t nv = cols / VEC, nvy = ldy / VEC;
  for (int64_t i = (int64_t)blockIdx.x * rpb + (threadIdx.x >> tpr_log2); i < rows;
       i += (int64_t)gridDim.x * rpb) {
    const double* x = X + i * ldx;
    const int64_t o = i * ldy;
#pragma unroll 4
    for (int64_t p = t; p < nvy; p += tpr) {
      if constexpr (VEC == 2) {
        Split3 a{0.f, 0.f, 0.f}, b{0.f, 0.f, 0.f};
        if (p < nv) {
          const double2 v = reinterpret_cast<const double2*>(x)[p];
          a = split3_int(v.x, inv, k, pow2);
          b = split3_int(v.y, inv, k, pow2);
        }
        reinterpret_cast<float2*>(Yh + o)[p] = make_float2(a.h, b.h);
        reinterpret_cast<float2*>(Yl + o)[p] = make_float2(a.l, b.l);
        reinterpret_cast<float2*>(Y3 + o)[p] = make_float2(a.e, b.e);
      } else {
        Split3 a{0.f, 0.f, 0.f};
        if (p < nv) a = split3_int(x[p], inv, k, pow2);
        Yh[o + p] = a.h;
        Yl[o + p] = a.l;
        Y3[o + p] = a.e;
      }
    }
  }
}

// log2 of the threads per row: about four accesses per thread on the longest
// side of the row, between a warp and a block
int conv_tpr_log2(int64_t units) {
  int lg = 5;
  while (lg < 8 && ((int64_t)1 << lg) * 4 < units) ++lg;
  return lg;
}

// One wave of resident blocks, so that every block's share of rows runs at once.
template <typename K>
unsigned conv_grid(K kernel, int64_t rows, int64_t rows_per_block) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t want = (rows + rows_per_block - 1) / rows_per_block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * num_sms()));
}
}  // namespace

lsrn_status launch_to_x2(const double* X, int64_t rows, int64_t cols, int64_t ldx, float* Yh,
                         float* Yl, float* Y3, int64_t ldy, unsigned long long* maxbits, double* xs,
                         cudaStream_t st) {
  *xs = 1.0;
  if (rows == 0 || ldy == 0) return LSRN_OK;
  // two columns per access when every row of X starts 16-byte aligned and the
  // rows hold whole pairs (ldy is a multiple of 4, so the FP32 rows do)
  const bool vec2 = ((uintptr_t)X % 16 == 0) && cols % 2 == 0 && ldx % 2 == 0 && ldy % 2 == 0;
  const int vec = vec2 ? 2 : 1;
  const int lg = conv_tpr_log2(ldy / vec);
  const int64_t rpb = 256 >> lg;
  LSRN_CUDA_TRY(cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), st));
  if (vec2)
    launch(maxabs_kernel<2>, dim3(conv_grid(maxabs_kernel<2>, rows, rpb)), dim3(256), 0, st, X,
           rows, cols, ldx, lg, maxbits);
  else
    launch(maxabs_kernel<1>, dim3(conv_grid(maxabs_kernel<1>, rows, rpb)), dim3(256), 0, st, X,
           rows, cols, ldx, lg, maxbits);
  unsigned long long bits = 0;
  LSRN_CUDA_TRY(cudaMemcpyAsync(&bits, maxbits, sizeof(bits), cudaMemcpyDeviceToHost, st));
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  double mx;
  std::memcpy(&mx, &bits, sizeof(mx));
  // power-of-two scale with the largest |X| / xs in [1, 2): no FP32 overflow,
  // and elements below 2^-126 of the largest are the only ones that lose bits
  if (mx > 0.0 && std::isfinite(mx)) *xs = std::ldexp(1.0, std::ilogb(mx));
  const double inv = 1.0 / *xs;
  int k = 0;
  const bool pow2 = std::isnormal(inv) && std::frexp(inv, &k) == 0.5;   // inv = 2^(k-1)
  k -= 1;
  if (vec2)
    launch(to_x2_kernel<2>, dim3(conv_grid(to_x2_kernel<2>, rows, rpb)), dim3(256), 0, st, X, rows,
           cols, ldx, inv, k, pow2, lg, Yh, Yl, Y3, ldy);
  else
    launch(to_x2_kernel<1>, dim3(conv_grid(to_x2_kernel<1>, rows, rpb)), dim3(256), 0, st, X, rows,
           cols, ldx, inv, k, pow2, lg, Yh, Yl, Y3, ldy);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_to_f32(const double* X, int64_t rows, int64_t cols, int64_t ldx, float* Y,
                          int64_t ldy, cudaStream_t st) {
  const int64_t tot = rows * ldy;
  if (tot == 0) return LSRN_OK;
  launch(to_f32_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, X, rows, cols, ldx,
         Y, ldy);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

bool pass_is_staged(int64_t C);

static int pick_layout(int64_t C, int* tpr, int* slots) {
  if (C <= 64) { *tpr = 32; *slots = 1; }
  else if (C <= 128) { *tpr = 32; *slots = 2; }
  else if (C <= 256) { *tpr = 64; *slots = 2; }
  else if (C <= 512) { *tpr = 128; *slots = 2; }
  else if (C <= 1024) { *tpr = 256; *slots = 2; }
  else if (C <= 2048) { *tpr = 256; *slots = 4; }
  else if (C <= 4096) { *tpr = 256; *slots = 8; }
  else return -1;
  return 0;
}

int pass_blocks(int64_t rows, int64_t C, bool x2) {
  int tpr, slots;
  if (pick_layout(C, &tpr, &slots) != 0) return 0;
  if (pass_is_staged(C)) {
    // double-float passes up to 2048 columns: three CTAs per SM (x2_geometry)
    const int per_sm = (x2 && C <= 2048) ? 3 : 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * num_sms(), rows));
  }
  const int64_t gpc = kThreads / tpr;
  const int64_t per = gpc * 2;
  const int64_t want = (rows + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 2 * num_sms()));
}

// Staged pass geometry for element size esz: rows per stage and stage count,
// or false when the staged kernel does not apply.
// With planes = 2 (the double-float pass) a staged row is one row of each plane
// and *rowbytes is the bytes of both.
static bool staged_geometry(int64_t C, int64_t ldx, size_t esz, int* rowbytes, int* rb,
                            int* nstages, int planes = 1) {
  if (C <= 512 || C > 4096) return false;
  const int64_t pbytes = (C * (int64_t)esz + 15) / 16 * 16;
  if (pbytes > ldx * (int64_t)esz || (ldx * (int64_t)esz) % 16 != 0) return false;
  const int64_t rbytes = planes * pbytes;
  int r = (int)std::max<int64_t>(2, (32768 / rbytes) / 2 * 2);
  r = std::min(r, 8);
  if (r != 2 && r != 4 && r != 8) r = r >= 8 ? 8 : (r >= 4 ? 4 : 2);
  int ns = (int)std::min<int64_t>(kMaxStages, (196608 - 1024) / (r * rbytes + 2 * r * 8));
  if (ns < 2) return false;
  *rowbytes = (int)rbytes;
  *rb = r;
  *nstages = ns;
  return true;
}

bool pass_is_staged(int64_t C) { return C > 512 && C <= 4096; }

template <class T, int SLOTS, int RB>
static lsrn_status launch_staged(const Plan* p, const T* X, int64_t ldx, const double* vin,
                                 const RowArgs& a, double* pvec, double* pscal, const int* done,
                                 int rowbytes, int nstages) {
  const size_t smem = (size_t)nstages * RB * rowbytes + (size_t)nstages * 2 * RB * sizeof(double);
  auto kern = row_pass_staged_kernel<T, SLOTS, RB>;
  // per launch: the attribute is per device, and server threads may share a device
  LSRN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  launch(kern, dim3(p->nblk), dim3(kThreads), smem, p->stream, X, p->xrows, (int)p->xcols, ldx, vin,
         a, pvec, pscal, done, p->iscal + IC_PASSERR, rowbytes, nstages);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

// Geometry of the double-float pass: RB = 2 rows of both planes per stage.  Up
// to 2048 columns two stages (64 KB), so that three CTAs share an SM: three
// times the warps of one CTA to hide the latency of the dependent double-float
// chains (4-row stages with one CTA per SM streamed at 0.40 of HBM, two CTAs
// of three stages at 0.50, three of two at 0.51).  Above 2048 columns as many
// stages as fit in 196 KB (at most 8), one CTA per SM.
static bool x2_geometry(int64_t C, int64_t ldx2, int* planebytes, int* rb, int* nstages) {
  if (C <= 512 || C > 4096) return false;
  const int64_t pbytes = (C * 4 + 15) / 16 * 16;
  if (pbytes > ldx2 * 4 || (ldx2 * 4) % 16 != 0) return false;
  const int r = 2;
  const int64_t stage = 2 * r * pbytes + 2 * r * 8;
  const int ns = C <= 2048 ? 2 : (int)std::min<int64_t>(kMaxStages, (196608 - 1024) / stage);
  if (ns < 2) return false;
  *planebytes = (int)pbytes;
  *rb = r;
  *nstages = ns;
  return true;
}

template <int SLOTS, int RB>
static lsrn_status launch_x2(const Plan* p, const double* vin, const RowArgs& a, double* pvec,
                             double* pscal, const int* done, int planebytes, int nstages) {
  const size_t smem =
      (size_t)nstages * 2 * RB * planebytes + (size_t)nstages * 2 * RB * sizeof(double);
  auto kern = row_pass_x2_kernel<SLOTS, RB>;
  LSRN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  launch(kern, dim3(p->nblk), dim3(kX2Threads), smem, p->stream, p->X2h, p->X2l, p->xrows,
         (int)p->xcols, p->ldx2, p->x2scale, vin, a, pvec, pscal, done, p->iscal + IC_PASSERR,
         planebytes, nstages);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

bool x2_applies(int64_t C) {
  int pb, rb, ns;
  return x2_geometry(C, (C + 3) / 4 * 4, &pb, &rb, &ns);
}

lsrn_status launch_row_pass(const Plan* p, const double* vin, const RowArgs& a, double* pvec,
                            double* pscal, const int* done) {
  int tpr, slots;
  if (pick_layout(p->xcols, &tpr, &slots) != 0) return LSRN_ERR_UNSUPPORTED;
  const int C = (int)p->xcols;
  int rowbytes = 0, rb = 0, ns = 0;
  if (p->X2h != nullptr && x2_geometry(C, p->ldx2, &rowbytes, &rb, &ns)) {
    if (slots == 2 && rb == 2) return launch_x2<2, 2>(p, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 4 && rb == 2) return launch_x2<4, 2>(p, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 8 && rb == 2) return launch_x2<8, 2>(p, vin, a, pvec, pscal, done, rowbytes, ns);
  }
  if (p->pass_f32 && staged_geometry(C, p->ldx32, sizeof(float), &rowbytes, &rb, &ns)) {
    const float* xp = p->X32;
    if (slots == 2 && rb == 8) return launch_staged<float, 2, 8>(p, xp, p->ldx32, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 4 && rb == 4) return launch_staged<float, 4, 4>(p, xp, p->ldx32, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 8 && rb == 2) return launch_staged<float, 8, 2>(p, xp, p->ldx32, vin, a, pvec, pscal, done, rowbytes, ns);
  }
  if (!p->pass_f32 && staged_geometry(C, p->ldx, sizeof(double), &rowbytes, &rb, &ns)) {
    const double* xp = p->X;
    if (slots == 2 && rb == 4) return launch_staged<double, 2, 4>(p, xp, p->ldx, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 4 && rb == 2) return launch_staged<double, 4, 2>(p, xp, p->ldx, vin, a, pvec, pscal, done, rowbytes, ns);
    if (slots == 8 && rb == 2) return launch_staged<double, 8, 2>(p, xp, p->ldx, vin, a, pvec, pscal, done, rowbytes, ns);
  }
  dim3 grid(p->nblk);
#define LSRN_ROWPASS(E, T, S, R)                                                        \
  launch(row_pass_kernel<E, T, S, R>, grid, kThreads, 0, p->stream, (const E*)xp, p->xrows, C, \
         ldx, vin, a, pvec, pscal, done)
#define LSRN_ROWPASS_ALL(E)                           \
  if (tpr == 32 && slots == 1) LSRN_ROWPASS(E, 32, 1, 4); \
  else if (tpr == 32) LSRN_ROWPASS(E, 32, 2, 4);          \
  else if (tpr == 64) LSRN_ROWPASS(E, 64, 2, 4);          \
  else if (tpr == 128) LSRN_ROWPASS(E, 128, 2, 4);        \
  else if (slots == 2) LSRN_ROWPASS(E, 256, 2, 4);        \
  else if (slots == 4) LSRN_ROWPASS(E, 256, 4, 2);        \
  else LSRN_ROWPASS(E, 256, 8, 1);
  if (p->pass_f32) {
    const void* xp = p->X32;
    const int64_t ldx = p->ldx32;
    LSRN_ROWPASS_ALL(float)
  } else {
    const void* xp = p->X;
    const int64_t ldx = p->ldx;
    LSRN_ROWPASS_ALL(double)
  }
#undef LSRN_ROWPASS_ALL
#undef LSRN_ROWPASS
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_extra_rows(const Plan* p, const double* vin, const RowArgs& a, double* pvec,
                              double* pscal, const int* done) {
  if (p->extra_rows == 0) return LSRN_OK;
  launch(extra_rows_kernel, 1, 1024, 0, p->stream, p->extra_rows, p->xrows, (int)p->xcols,
                                               p->extra_coef, vin, a, pvec + (int64_t)p->nblk * p->xcols,
                                               pscal + p->nblk, done);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

namespace {
__global__ void add_vec_kernel(double* __restrict__ out, const double* __restrict__ v, int64_t n,
                               const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += v[i];
}
}  // namespace

// Ridge rows for the sparse passes: their contribution is added into out.
lsrn_status launch_row_coef_extra(const Plan* p, const double* vin, const RowArgs& a, double* out,
                                  double* pscal_slot, const int* done) {
  launch(extra_rows_kernel, 1, 1024, 0, p->stream, p->extra_rows, p->xrows, (int)p->xcols,
         p->extra_coef, vin, a, p->pvec, pscal_slot, done);
  launch(add_vec_kernel, dim3((unsigned)((p->xcols + 255) / 256)), dim3(256), 0, p->stream, out,
         (const double*)p->pvec, p->xcols, done);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status csr_dd_pass(const Plan* p, const double* vin, const double* bvec, double* rout,
                        double* phi, double* plo, double* tbuf);

// Geometry of the triple-float residual pass: RB rows of the three planes per
// stage (RB = 4 up to 1024 columns, 2 above), at least three stages in 196 KB.
static bool x3_geometry(int64_t C, int64_t ldx2, int* planebytes, int* rb, int* nstages) {
  if (C <= 512 || C > 4096) return false;
  const int64_t pbytes = (C * 4 + 15) / 16 * 16;
  if (pbytes > ldx2 * 4 || (ldx2 * 4) % 16 != 0) return false;
  const int r = C <= 1024 ? 4 : 2;
  const int64_t stage = 3 * r * pbytes + ((int64_t)r * 8 + 15) / 16 * 16;
  const int ns = (int)std::min<int64_t>(kMaxStages, (196608 - 1024) / stage);
  if (ns < 3) return false;
  *planebytes = (int)pbytes;
  *rb = r;
  *nstages = ns;
  return true;
}

template <int SLOTS, int RB>
static lsrn_status launch_x3(const Plan* p, const double* vin, const double* rowvec, bool tall,
                             double* rout, double* phi, double* plo, int planebytes, int nstages) {
  const size_t stage = (size_t)3 * RB * planebytes + ((size_t)RB * 8 + 15) / 16 * 16;
  // the state region is indexed [stage][RB]: its size rounds each stage's RB doubles up
  const size_t smem = (size_t)nstages * 3 * RB * planebytes + (size_t)nstages * RB * sizeof(double) + 16;
  (void)stage;
  auto kern = dd_pass_x3_kernel<SLOTS, RB>;
  LSRN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  launch(kern, dim3(p->nblk), dim3(kX2Threads), smem, p->stream, p->X2h, p->X2l, p->X3, p->xrows,
         (int)p->xcols, p->ldx2, p->x2scale, vin, rowvec, p->xscale, tall ? 1 : 0, rout, phi, plo,
         p->iscal + IC_PASSERR, planebytes, nstages);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_dd_pass(const Plan* p, const double* vin, const double* bvec, double* rout,
                           double* pvec_hi, double* pvec_lo, const int* done) {
  (void)done;
  if (p->csr) {
    LSRN_TRY(csr_dd_pass(p, vin, bvec, rout, pvec_hi, pvec_lo, p->tcsr));
    if (p->extra_rows > 0) {
      const int C = (int)p->xcols;
      launch(dd_extra_kernel, dim3((unsigned)((p->xcols + 255) / 256)), dim3(256), 0, p->stream,
             p->extra_rows, p->xrows, C, p->extra_coef, vin, bvec != nullptr, rout,
             pvec_hi + (int64_t)p->nblk * C, pvec_lo + (int64_t)p->nblk * C);
    }
    LSRN_CUDA_TRY(cudaGetLastError());
    return LSRN_OK;
  }
  int tpr, slots;
  if (pick_layout(p->xcols, &tpr, &slots) != 0) return LSRN_ERR_UNSUPPORTED;
  const int C = (int)p->xcols;
  int pb = 0, rb = 0, ns = 0;
  if (p->X3 != nullptr && x3_geometry(C, p->ldx2, &pb, &rb, &ns)) {
    const bool tall = bvec != nullptr;
    const double* rowvec = tall ? bvec : vin;
    lsrn_status st = LSRN_ERR_UNSUPPORTED;
    if (slots == 2 && rb == 4) st = launch_x3<2, 4>(p, vin, rowvec, tall, rout, pvec_hi, pvec_lo, pb, ns);
    else if (slots == 4 && rb == 2) st = launch_x3<4, 2>(p, vin, rowvec, tall, rout, pvec_hi, pvec_lo, pb, ns);
    else if (slots == 8 && rb == 2) st = launch_x3<8, 2>(p, vin, rowvec, tall, rout, pvec_hi, pvec_lo, pb, ns);
    if (st != LSRN_ERR_UNSUPPORTED) {
      LSRN_TRY(st);
      if (p->extra_rows > 0) {
        launch(dd_extra_kernel, (unsigned)((p->xcols + 255) / 256), 256, 0, p->stream,
               p->extra_rows, p->xrows, C, p->extra_coef, vin, tall, rout,
               pvec_hi + (int64_t)p->nblk * C, pvec_lo + (int64_t)p->nblk * C);
      }
      LSRN_CUDA_TRY(cudaGetLastError());
      return LSRN_OK;
    }
  }
  dim3 grid(p->nblk);
#define LSRN_DDPASS(T, S)                                                                       \
  launch(dd_pass_kernel<T, S>, grid, kThreads, 0, p->stream, p->X, p->xrows, C, p->ldx, vin, bvec,   \
                                                         rout, p->xscale, pvec_hi, pvec_lo)
  if (tpr == 32 && slots == 1) LSRN_DDPASS(32, 1);
  else if (tpr == 32) LSRN_DDPASS(32, 2);
  else if (tpr == 64) LSRN_DDPASS(64, 2);
  else if (tpr == 128) LSRN_DDPASS(128, 2);
  else if (slots == 2) LSRN_DDPASS(256, 2);
  else if (slots == 4) LSRN_DDPASS(256, 4);
  else LSRN_DDPASS(256, 8);
#undef LSRN_DDPASS
  if (p->extra_rows > 0) {
    launch(dd_extra_kernel, (unsigned)((p->xcols + 255) / 256), 256, 0, p->stream, 
        p->extra_rows, p->xrows, C, p->extra_coef, vin, bvec != nullptr, rout,
        pvec_hi + (int64_t)p->nblk * C, pvec_lo + (int64_t)p->nblk * C);
  }
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_reduce(const double* pvec, int nslots, int64_t C, double* out,
                          const double* pscal, double* scal_out, const int* done, cudaStream_t st) {
  launch(reduce_kernel, (unsigned)((C + 255) / 256), 256, 0, st, pvec, nslots, C, out, pscal, scal_out,
                                                             done);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_reduce_dd(const double* phi, const double* plo, int nslots, int64_t C,
                             double* out_hi, double* out_lo, cudaStream_t st) {
  launch(reduce_dd_kernel, (unsigned)((C + 255) / 256), 256, 0, st, phi, plo, nslots, C, out_hi,
                                                                out_lo);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status launch_gemv(const double* M, int64_t R, int64_t C, const double* v, double* out,
                        const double* y, double* y2, const double* c, const int* done,
                        cudaStream_t st) {
  if (R == 0) return LSRN_OK;
  launch(gemv_kernel, (unsigned)((R * 32 + 255) / 256), 256, 0, st, M, R, C, v, out, y, y2, c, done);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

namespace {

// Row updates of an operator pass: mult[i] = row_coef(d[i]) (the same row modes
// as the fused pass), block partials of the sum of squares into part.
__global__ void op_rows_kernel(RowArgs a, const double* __restrict__ coef, const double* __restrict__ d,
                               int64_t rows, double* __restrict__ mult, double* __restrict__ part,
                               const int* __restrict__ done) {
  __shared__ double sh[8];
  double ss = 0.0;
  if (done == nullptr || !*done) {
    Coef k{0.0, 0.0};
    if (coef) {
      k.c0 = coef[0];
      k.c1 = coef[1];
    }
    const bool r0 = mode_reads_st0(a.mode), r1 = a.mode == RM_FAT_CS;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double s0 = r0 ? a.st0[i] : 0.0, s1 = r1 ? a.st1[i] : 0.0;
      mult[i] = row_coef(a, k, i, d ? d[i] : 0.0, s0, s1, true, ss);
    }
  }
  ss = group_sum<32>(ss);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void op_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

}  // namespace

lsrn_status op_row_pass(Plan* p, const double* vin, const RowArgs& a, double* pvec, double* pscal,
                        const int* done) {
  if (done != nullptr) {   // after convergence nothing is applied
    int d = 0;
    LSRN_CUDA_TRY(cudaMemcpyAsync(&d, done, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (d != 0) return LSRN_OK;
  }
  // X = A (m >= n) or A^T (m < n): d = X vin, then pvec = X^T mult
  const lsrn_matmat_fn fwd = p->tall ? p->op.matmat : p->op.rmatmat;
  const lsrn_matmat_fn bwd = p->tall ? p->op.rmatmat : p->op.matmat;
  const bool need_dot = a.mode != RM_ACC_STATE;
  if (need_dot) {
    LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (fwd(p->op.ctx, 1, vin, p->opd) != 0) return LSRN_ERR_COMM;
  }
  const int64_t rows = p->xrows;
  const int parts = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 4 * num_sms()));
  launch(op_rows_kernel, parts, 256, 0, p->stream, a, a.coef, need_dot ? (const double*)p->opd : nullptr,
         rows, p->opt_mult, pscal + 2, (const int*)nullptr);
  launch(op_sum_kernel, 1, 32, 0, p->stream, (const double*)(pscal + 2), parts, pscal);
  LSRN_CUDA_TRY(cudaGetLastError());
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  if (bwd(p->op.ctx, 1, p->opt_mult, pvec) != 0) return LSRN_ERR_COMM;
  return LSRN_OK;
}

}  // namespace lsrn
