// Measurement aid (no counterpart in the paper): FP64 fused multiply-add
// throughput of the device, the denominator of the roofline of kernels whose
// bound is FP64 arithmetic (the FP64 sketch, the FP64 passes).
#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {
namespace {

// 8 independent FMA chains per thread, 16 steps per loop trip.
__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(double* out, int iters, double a,
                                                             double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace
}  // namespace lsrn

using namespace lsrn;

extern "C" lsrn_status lsrn_probe_fp64_fma(double* tflops) {
  if (tflops == nullptr) return LSRN_ERR_INVALID_ARG;
  const int blocks = num_sms() * 8, threads = 256, iters = 2000;
  double* buf = nullptr;
  LSRN_CUDA_TRY(cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, 0);
    launch(fp64_fma_probe_kernel, dim3(blocks), dim3(threads), 0, (cudaStream_t)0, buf, iters,
           0.999999, 1e-7);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) {
    record_cuda_error(e, "fp64 probe", __FILE__, __LINE__);
    return LSRN_ERR_CUDA;
  }
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LSRN_OK;
}
