// Allocation-free sketch entry point.
//
// Some callers cannot or must not allocate device memory: services that reserve
// all device memory for their own pool at start-up, code running inside another
// allocator's callbacks, or latency-critical paths where cudaMalloc/cudaFree
// (which may synchronise the device) are not allowed.  For them
// lsrn_sketch_f64_noalloc computes the FP64 sketch A~ = G A with its split-K
// partial sums in a fixed, file-scope device array instead of allocated
// workspace.  The array (kNoAllocScratchDoubles doubles, 32 MiB) is part of the
// library's device image: every GPU that loads the library holds it until the
// process exits.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)4 << 20;   // 32 MiB of FP64 partial sums

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device.
// The host-side name g_noalloc_scratch is only a stand-in and must never be
// handed to a kernel.
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};

lsrn_status noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return LSRN_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      lsrn::record_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      cudaGetLastError();
      return LSRN_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return LSRN_OK;
}

}  // namespace

extern "C" lsrn_status lsrn_sketch_f64_noalloc(const double* A, int64_t m, int64_t n, int64_t lda,
                                               double gamma, uint64_t seed, double* out,
                                               void* stream) {
  if (A == nullptr || out == nullptr || m < 1 || n < 1 || m < n || lda < n) return LSRN_ERR_INVALID_ARG;
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return LSRN_ERR_INVALID_ARG;
  if (!lsrn::is_device_pointer(A) || !lsrn::is_device_pointer(out)) return LSRN_ERR_INVALID_ARG;
  // size check in double arithmetic first, so a huge gamma cannot overflow s or s * n
  const double sd = std::max(std::ceil(gamma * (double)n), (double)n + 1.0);
  if (!(sd * (double)n <= (double)kNoAllocScratchDoubles)) return LSRN_ERR_INVALID_ARG;
  const int64_t s = (int64_t)sd;
  double* scratch = nullptr;
  lsrn_status st = noalloc_scratch(&scratch);
  if (st != LSRN_OK) return st;
  return lsrn::launch_sketch_f64_splitk_into(A, m, n, lda, s, seed, 0u, out, n, scratch,
                                             kNoAllocScratchDoubles, (cudaStream_t)stream);
}
