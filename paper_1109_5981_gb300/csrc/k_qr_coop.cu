// Householder QR of the sketch in one cooperative launch (Algorithm 1/2 step 4:
// the R whose SVD the one-sided Jacobi computes).
//
// The column-at-a-time QR issues three kernels per column (reflector, w = v^T C,
// C -= tau v w^T).  Each of them is small, so at q = 2000 the 6000 launches
// cost ~65 us a column against ~10 us of FP64 work.  Here one persistent grid
// of one CTA per SM (two from q = 1024 on) runs all columns, with two
// grid-wide barriers per column (the CTAs wait on one another, so the launch
// is cooperative: all are resident at once).  The same reflectors as the
// per-column kernels:
//   alpha = X[k, k], t = sum_{i > k} X[i, k]^2, beta = -sign(alpha) sqrt(alpha^2 + t),
//   tau = (beta - alpha) / beta, v_k = 1, v_i = X[i, k] / (alpha - beta) (i > k),
//   w_c = sum_{i >= k} v_i X[i, c], X[i, c] -= tau v_i w_c for c > k;
// R is left in the upper triangle, v below it, tau[k] as before.
//
// Work split: CTA b owns the rows i = rb (mod 8) (rb = b mod 8) and the
// 32-column chunks j = cb (mod CB) (cb = b / 8, CB = grid / 8), so the shrinking
// trailing matrix stays spread over all CTAs.  Per column k:
//   1. every CTA sums the eight row-group partial norms of column k (fixed
//      order, so all CTAs get the same tau) and forms v for its rows;
//   2. partial w over its rows for its chunks -> wpart[rb][c];   barrier A
//   3. w_c = sum over the eight row groups (fixed order), update of its rows and
//      chunks; the CTAs owning column k + 1 leave its partial norms;   barrier B
// Every barrier wait is bounded by elapsed global time; a CTA that gives up
// raises the error flag, the others leave at their next barrier, and the
// caller returns LSRN_ERR_TIMEOUT.
#include <algorithm>
#include <mutex>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

constexpr int kCqThreads = 256;
constexpr int kCqRG = 8;          // row groups
constexpr int kCqChunk = 32;      // columns per chunk
constexpr int kCqU = 8;           // rows a warp has in flight (independent loads)
constexpr int kCqMaxSmem = 160 * 1024;   // v of a CTA's rows: up to 8 * 20480 rows of the sketch
constexpr uint64_t kCqWaitNs = 10000000000ull;   // ten seconds per barrier wait

__device__ __forceinline__ uint64_t cq_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned cq_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int cq_ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void cq_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier: bar[0] counts arrivals, bar[1] is the generation.  Returns false
// (in every thread of the CTA) once any CTA has raised the error flag.
__device__ bool cq_grid_sync(unsigned* bar, unsigned& gen, int* err, uint64_t wait_ns, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      cq_st_release(&bar[1], gen + 1);
    } else {
      const uint64_t t0 = cq_timer_ns();
      for (int it = 0;; ++it) {
        if (cq_ld_acquire(&bar[1]) != gen) break;
        if ((it & 15) == 15 && (cq_timer_ns() - t0 > wait_ns || cq_ld_acquire_i(err) != 0)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *s_ok = ok && cq_ld_acquire_i(err) == 0;
  }
  __syncthreads();
  ++gen;
  return *s_ok != 0;
}

// Sum of v over the CTA, result in thread 0.
__device__ __forceinline__ double cq_block_sum0(double v, double* red) {
  v = group_sum<32>(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kCqThreads / 32; ++w) t += red[w];
  return t;
}

struct CoopQr {
  double* X;
  int64_t S, Q;
  double* tau;
  double* npart;   // [kCqRG] partial sums of squares of the next column
  double* wpart;   // [kCqRG][Q]
  unsigned* bar;   // [2], zero at launch
  int* err;
  uint64_t wait_ns;
  int absent;      // test knob: CTA 0 leaves before the first barrier
};

__global__ void __launch_bounds__(kCqThreads, 2) qr_coop_kernel(CoopQr a) {
  extern __shared__ double vbuf[];   // v for this CTA's rows (row t: i = rg + 8 t)
  __shared__ double red[kCqThreads / 32];
  __shared__ double part[kCqThreads / 32][kCqChunk];
  __shared__ double wsh[kCqChunk];
  __shared__ double s_tk, s_scal, s_beta;
  __shared__ int s_ok;
  double* X = a.X;
  const int64_t S = a.S, Q = a.Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = (int)(blockIdx.x % kCqRG), cg = (int)(blockIdx.x / kCqRG);
  const int CB = (int)(gridDim.x / kCqRG);
  const int64_t nrow = S > rg ? (S - rg + kCqRG - 1) / kCqRG : 0;   // rows i = rg + 8 t
  const int64_t nchunk = (Q + kCqChunk - 1) / kCqChunk;
  unsigned gen = 0;
  auto owns_col = [&](int64_t c) { return (int)((c / kCqChunk) % CB) == cg; };

  // partial norms of column k over this CTA's rows i > k (CTAs owning column k)
  auto norm_partial = [&](int64_t k) {
    double ss = 0.0;
    for (int64_t t = tid; t < nrow; t += kCqThreads) {
      const int64_t i = rg + (int64_t)kCqRG * t;
      if (i > k) {
        const double x = X[i * Q + k];
        ss = fma(x, x, ss);
      }
    }
    const double tot = cq_block_sum0(ss, red);
    if (tid == 0) a.npart[rg] = tot;
  };

  if (Q > 0 && owns_col(0)) norm_partial(0);
  if (a.absent && blockIdx.x == 0) return;   // the others' first barrier wait runs out
  if (!cq_grid_sync(a.bar, gen, a.err, a.wait_ns, &s_ok)) return;

  for (int64_t k = 0; k < Q; ++k) {
    if (tid == 0) {
      double t = 0.0;
      for (int r = 0; r < kCqRG; ++r) t += __ldcg(a.npart + r);
      const double alpha = __ldcg(X + k * Q + k);
      double tk = 0.0, scal = 0.0, beta = alpha;
      if (t > 0.0) {
        const double nrm = sqrt(alpha * alpha + t);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tk = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      s_tk = tk;
      s_scal = scal;
      s_beta = beta;
    }
    __syncthreads();
    const double tk = s_tk, scal = s_scal;
    const int64_t jk = (k + 1) / kCqChunk;   // first chunk with columns > k
    const int64_t t0 = k > rg ? (k - rg + kCqRG - 1) / kCqRG : 0;   // first own row i >= k
    if (tk != 0.0) {   // uniform over the grid
      for (int64_t t = tid; t < nrow; t += kCqThreads) {
        const int64_t i = rg + (int64_t)kCqRG * t;
        vbuf[t] = i < k ? 0.0 : (i == k ? 1.0 : __ldcg(X + i * Q + k) * scal);
      }
      __syncthreads();
      // 2. partial w for this CTA's chunks: warp w takes rows t = w (mod 8)
      for (int64_t j = jk + ((cg - jk % CB) % CB + CB) % CB; j < nchunk; j += CB) {
        const int64_t c = j * kCqChunk + lane;
        double acc = 0.0;
        if (c > k && c < Q) {
          const double* xc = X + (int64_t)rg * Q + c;   // row t of this CTA: xc[8 t Q]
          int64_t t = t0 + warp;
          for (; t + 8 * (kCqU - 1) < nrow; t += 8 * kCqU) {
            double x[kCqU];
#pragma unroll
            for (int u = 0; u < kCqU; ++u) x[u] = __ldcg(xc + (t + 8 * u) * kCqRG * Q);
#pragma unroll
            for (int u = 0; u < kCqU; ++u) acc = fma(vbuf[t + 8 * u], x[u], acc);
          }
          for (; t < nrow; t += 8) acc = fma(vbuf[t], __ldcg(xc + t * kCqRG * Q), acc);
        }
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
          double s = 0.0;
#pragma unroll
          for (int w = 0; w < kCqThreads / 32; ++w) s += part[w][lane];
          if (c > k && c < Q) a.wpart[(int64_t)rg * Q + c] = s;
        }
        __syncthreads();
      }
    }
    if (!cq_grid_sync(a.bar, gen, a.err, a.wait_ns, &s_ok)) return;   // barrier A
    if (tk != 0.0) {
      // column k: the reflector below the diagonal, beta on it
      if (owns_col(k)) {
        for (int64_t t = tid; t < nrow; t += kCqThreads) {
          const int64_t i = rg + (int64_t)kCqRG * t;
          if (i > k) X[i * Q + k] = vbuf[t];
          if (i == k) X[k * Q + k] = s_beta;
        }
      }
      // 3. update this CTA's rows and chunks
      for (int64_t j = jk + ((cg - jk % CB) % CB + CB) % CB; j < nchunk; j += CB) {
        const int64_t c = j * kCqChunk + lane;
        if (warp == 0) {
          double w = 0.0;
          if (c > k && c < Q)
#pragma unroll
            for (int r = 0; r < kCqRG; ++r) w += __ldcg(a.wpart + (int64_t)r * Q + c);
          wsh[lane] = tk * w;
        }
        __syncthreads();
        const double tw = wsh[lane];
        if (c > k && c < Q) {
          double* xc = X + (int64_t)rg * Q + c;
          int64_t t = t0 + warp;
          for (; t + 8 * (kCqU - 1) < nrow; t += 8 * kCqU) {
            double x[kCqU];
#pragma unroll
            for (int u = 0; u < kCqU; ++u) x[u] = xc[(t + 8 * u) * kCqRG * Q];
#pragma unroll
            for (int u = 0; u < kCqU; ++u) xc[(t + 8 * u) * kCqRG * Q] = fma(-vbuf[t + 8 * u], tw, x[u]);
          }
          for (; t < nrow; t += 8) xc[t * kCqRG * Q] = fma(-vbuf[t], tw, xc[t * kCqRG * Q]);
        }
        __syncthreads();
      }
    }
    if (tid == 0 && owns_col(k) && rg == 0) a.tau[k] = tk;
    if (k + 1 < Q && owns_col(k + 1)) norm_partial(k + 1);
    if (!cq_grid_sync(a.bar, gen, a.err, a.wait_ns, &s_ok)) return;   // barrier B
  }
}

// One cooperative grid at a time in this process: plans of a server or a
// batch run on several streams, and two partly resident grids could each hold
// SMs that the other's waiting CTAs need.
std::mutex g_coop_mutex;

}  // namespace

// Cooperative QR of X (S x Q row-major, in place).  Returns LSRN_OK with *ran
// false, and nothing launched, when the device cannot hold the grid (then the
// caller runs the per-column kernels); LSRN_ERR_TIMEOUT if a barrier wait gave
// up.
lsrn_status launch_qr_coop(double* X, int64_t S, int64_t Q, double* tau, cudaStream_t st, bool* ran) {
  *ran = false;
  if (Q <= 0 || S <= 0) return LSRN_OK;
  int dev = 0, coop = 0, per_sm = 0;
  LSRN_CUDA_TRY(cudaGetDevice(&dev));
  LSRN_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  const int nsm = num_sms();
  // two CTAs per SM from q = 1024 on (59 vs 66 ms at q = 2000); at smaller q
  // the wider barrier costs more than the extra warps give
  const int CB = (Q >= 1024 ? 2 : 1) * nsm / kCqRG;
  const size_t smem = (size_t)((S + kCqRG - 1) / kCqRG) * sizeof(double);
  if (!coop || CB < 1 || smem > (size_t)kCqMaxSmem) return LSRN_OK;
  // one fixed limit: plans on other threads set it too, and a per-call value
  // could fall below another thread's launch in between
  LSRN_CUDA_TRY(cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kCqMaxSmem));
  LSRN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_coop_kernel, kCqThreads, smem));
  const int grid = CB * kCqRG;
  if (per_sm < 1 || grid > per_sm * nsm) return LSRN_OK;
  // the sketch is done before the lock is taken; a plan that finds another
  // plan's grid running waits for it (taking the per-column kernels instead
  // would round differently, and a result must not depend on what else runs)
  LSRN_CUDA_TRY(cudaStreamSynchronize(st));
  std::lock_guard<std::mutex> lock(g_coop_mutex);   // until the grid has finished
  double* ws = nullptr;
  const size_t wbytes = ((size_t)kCqRG + (size_t)kCqRG * Q) * sizeof(double) + 4 * sizeof(int);
  LSRN_CUDA_TRY(lsrn_malloc_async((void**)&ws, wbytes, st));
  CoopQr a;
  a.X = X;
  a.S = S;
  a.Q = Q;
  a.tau = tau;
  a.npart = ws;
  a.wpart = ws + kCqRG;
  a.bar = (unsigned*)(ws + kCqRG + (size_t)kCqRG * Q);
  a.err = (int*)(a.bar + 2);
  a.absent = test_knob(LSRN_KNOB_QR_ABSENT_CTA) != 0 ? 1 : 0;
  const int64_t knob_wait = test_knob(LSRN_KNOB_JACOBI_WAIT_NS);
  a.wait_ns = (a.absent && knob_wait > 0) ? (uint64_t)knob_wait : kCqWaitNs;
  lsrn_status rs = LSRN_OK;
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(int), st) != cudaSuccess) rs = LSRN_ERR_CUDA;
  void* args[] = {(void*)&a};
  if (rs == LSRN_OK &&
      cudaLaunchCooperativeKernel((const void*)qr_coop_kernel, dim3(grid), dim3(kCqThreads), args, smem,
                                  st) != cudaSuccess)
    rs = LSRN_ERR_CUDA;
  if (rs == LSRN_OK) {
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    int e = 0;
    if (cudaMemcpyAsync(&e, a.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rs = LSRN_ERR_CUDA;
    else if (e != 0)
      rs = LSRN_ERR_TIMEOUT;
  }
  cudaGetLastError();
  cudaFreeAsync(ws, st);
  *ran = rs == LSRN_OK || rs == LSRN_ERR_TIMEOUT;
  return rs;
}

}  // namespace lsrn
