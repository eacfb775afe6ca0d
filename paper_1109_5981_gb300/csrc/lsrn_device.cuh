// Device-side building blocks of the LSRN library (GB300, sm_103a).
//
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
//    Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
//    increments 0x9E3779B9 / 0xBB67AE85.
//  * Box-Muller normals in binary32 with our own logarithm (atanh series) and
//    sin/cos of 2*pi*u (exact quarter-turn reduction + Taylor series), every
//    step one correctly rounded binary32 operation (explicit __f*_rn intrinsics
//    so that nothing is contracted), so the sketching matrix G of Algorithms 1
//    and 2 (section 4.1, step 2) is a fixed function of (seed, tag, row, col).
//  * Double-double error-free transformations for accurate residuals.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

namespace lsrn {

// Kernel launches issued by the library since it was loaded (diagnostic).
extern std::atomic<unsigned long long> g_kernel_launches;

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args&&... args) {
  kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

// Capture the stream work that `issue` enqueues on `st` into an executable
// CUDA graph (capture mode local to the calling thread, so other threads'
// plans and servers are unaffected).  Returns nullptr, with the stream back in
// normal mode and the error cleared, if capture or instantiation fails; the
// caller then issues the work directly.  *kernels receives the number of
// kernel launches in the graph; they are not counted as launched until the
// graph is.
template <class F>
inline cudaGraphExec_t capture_graph(cudaStream_t st, F issue, unsigned long long* kernels) {
  *kernels = 0;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const unsigned long long before = g_kernel_launches.load(std::memory_order_relaxed);
  issue();
  const unsigned long long after = g_kernel_launches.load(std::memory_order_relaxed);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess && g != nullptr) e = cudaGraphInstantiate(&ex, g, 0);
  if (g != nullptr) cudaGraphDestroy(g);
  g_kernel_launches.fetch_sub(after - before, std::memory_order_relaxed);
  if (e != cudaSuccess || ex == nullptr) {
    if (ex != nullptr) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    return nullptr;
  }
  *kernels = after - before;
  return ex;
}

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// (2*(x>>9)+1) * 2^-24: odd multiple of 2^-24 in (0,1); both steps exact.
__device__ __forceinline__ float uniform01(uint32_t x) {
  return __fmul_rn(__uint2float_rn(2u * (x >> 9) + 1u), 0x1p-24f);
}

// ln(u), u in [2^-24, 1): u = 2^e f, f in [1/sqrt2, sqrt2), ln f = 2 atanh(s).
__device__ __forceinline__ float own_logf(float u) {
  const uint32_t b = __float_as_uint(u);
  int e = (int)(b >> 23) - 127;
  float f = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  if (f > __uint_as_float(0x3FB504F3u)) {
    f = __fmul_rn(f, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = __fmaf_rn(s2, __uint_as_float(0x3D9D89D9u), __uint_as_float(0x3DBA2E8Cu));
  p = __fmaf_rn(s2, p, __uint_as_float(0x3DE38E39u));
  p = __fmaf_rn(s2, p, __uint_as_float(0x3E124925u));
  p = __fmaf_rn(s2, p, __uint_as_float(0x3E4CCCCDu));
  p = __fmaf_rn(s2, p, __uint_as_float(0x3EAAAAABu));
  const float t = __fadd_rn(s, s);
  const float ts2 = __fmul_rn(t, s2);
  const float lnf = __fmaf_rn(ts2, p, t);
  const float ef = __int2float_rn(e);
  const float lo = __fmaf_rn(ef, __uint_as_float(0x35BFBE8Eu), lnf);
  return __fmaf_rn(ef, __uint_as_float(0x3F317200u), lo);
}

// sin(2 pi u), cos(2 pi u) for u in (0,1).
__device__ __forceinline__ void own_sincos2pi(float u, float* sn, float* cs) {
  const float t = __fmul_rn(u, 4.0f);
  int q = __float2int_rz(t);
  float f = __fsub_rn(t, __int2float_rn(q));
  if (f > 0.5f) {
    f = __fsub_rn(f, 1.0f);
    q += 1;
  }
  const float x = __fmul_rn(f, __uint_as_float(0x3FC90FDBu));
  const float x2 = __fmul_rn(x, x);
  float ps = __fmaf_rn(x2, __uint_as_float(0x3638EF1Du), __uint_as_float(0xB9500D01u));
  ps = __fmaf_rn(x2, ps, __uint_as_float(0x3C088889u));
  ps = __fmaf_rn(x2, ps, __uint_as_float(0xBE2AAAABu));
  const float x3 = __fmul_rn(x, x2);
  const float sx = __fmaf_rn(x3, ps, x);
  float pc = __fmaf_rn(x2, __uint_as_float(0xB493F27Eu), __uint_as_float(0x37D00D01u));
  pc = __fmaf_rn(x2, pc, __uint_as_float(0xBAB60B61u));
  pc = __fmaf_rn(x2, pc, __uint_as_float(0x3D2AAAABu));
  pc = __fmaf_rn(x2, pc, -0.5f);
  const float cx = __fmaf_rn(x2, pc, 1.0f);
  switch (q & 3) {
    case 0: *sn = sx; *cs = cx; break;
    case 1: *sn = cx; *cs = -sx; break;
    case 2: *sn = -sx; *cs = -cx; break;
    default: *sn = -cx; *cs = sx; break;
  }
}

// The four normals of columns 4*q4 .. 4*q4+3 of row `row` of the drawing
// array with key `seed` and counter word 3 = tag.
__device__ __forceinline__ float4 normal4(uint64_t seed, uint32_t tag, uint64_t row, uint64_t q4) {
  const U4 w = philox4x32_10(U4{(uint32_t)q4, (uint32_t)(q4 >> 32), (uint32_t)row, tag},
                             (uint32_t)seed, (uint32_t)(seed >> 32));
  float4 z;
  {
    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, own_logf(uniform01(w.x))));
    float sn, cs;
    own_sincos2pi(uniform01(w.y), &sn, &cs);
    z.x = __fmul_rn(rad, cs);
    z.y = __fmul_rn(rad, sn);
  }
  {
    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, own_logf(uniform01(w.z))));
    float sn, cs;
    own_sincos2pi(uniform01(w.w), &sn, &cs);
    z.z = __fmul_rn(rad, cs);
    z.w = __fmul_rn(rad, sn);
  }
  return z;
}

// G entry: the normal rounded to the grid 2^-12, |q| <= 32767.
__device__ __forceinline__ float quantize_g(float z) {
  float q = rintf(__fmul_rn(z, 4096.0f));
  q = fminf(fmaxf(q, -32767.0f), 32767.0f);
  return __fmul_rn(q, 0x1p-12f);
}

// ---- double-double -------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  const double t = __dadd_rn(a, b);
  const double bb = __dsub_rn(t, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(t, bb)), __dsub_rn(b, bb));
  s = t;
}

// (hi, lo) += a * b
__device__ __forceinline__ void dd_add_prod(double& hi, double& lo, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double pe = __fma_rn(a, b, -p);
  double s, se;
  two_sum(hi, p, s, se);
  const double l = __dadd_rn(__dadd_rn(lo, se), pe);
  two_sum(s, l, hi, lo);
}

// (hi, lo) += (bh, bl)
__device__ __forceinline__ void dd_add(double& hi, double& lo, double bh, double bl) {
  double s, e;
  two_sum(hi, bh, s, e);
  const double l = __dadd_rn(__dadd_rn(lo, bl), e);
  two_sum(s, l, hi, lo);
}

// ---- reductions -------------------------------------------------------------
template <int WIDTH>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int WIDTH>
__device__ __forceinline__ void group_sum_dd(double& hi, double& lo) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) {
    const double oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const double ol = __shfl_xor_sync(0xffffffffu, lo, o);
    dd_add(hi, lo, oh, ol);
  }
}

}  // namespace lsrn
