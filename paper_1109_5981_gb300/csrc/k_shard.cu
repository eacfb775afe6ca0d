// Exchanges of a row-sharded solve (section 4.4: the matrix is partitioned by
// rows, each process computes its part of every product with A or A^T, and
// the n-vectors are summed over processes).  The library does not talk to a
// network itself: it hands a staging buffer to the caller's allgather
// callback (NCCL, MPI, gloo or host threads) and adds the gathered copies in
// rank order on the device, so every shard gets the same bits.
#include "lsrn_device.cuh"
#include "lsrn_internal.h"

namespace lsrn {

namespace {

// out[i] = sum_p recv[p * count + i], p = 0 .. world - 1 in order
__global__ void shard_sum_kernel(const double* __restrict__ recv, int world, int64_t count,
                                 double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = recv[i];
    for (int q = 1; q < world; ++q) acc += recv[(int64_t)q * count + i];
    out[i] = acc;
  }
}

// recv holds, per shard, [hi (count), lo (count)]; (hi, lo)[i] = double-double sum in rank order
__global__ void shard_sum_dd_kernel(const double* __restrict__ recv, int world, int64_t count,
                                    double* __restrict__ hi, double* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double h = recv[i], l = recv[count + i];
    for (int q = 1; q < world; ++q) {
      const int64_t base = (int64_t)q * 2 * count;
      dd_add(h, l, recv[base + i], recv[base + count + i]);
    }
    hi[i] = h;
    lo[i] = l;
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * (int64_t)num_sms()));
}

lsrn_status ensure_staging(Plan* p, int64_t count) {
  Shard& sh = p->shard;
  if (count <= sh.cap) return LSRN_OK;
  if (sh.send) cudaFreeAsync(sh.send, p->stream);
  if (sh.recv) cudaFreeAsync(sh.recv, p->stream);
  sh.send = sh.recv = nullptr;
  sh.cap = 0;
  LSRN_CUDA_TRY(lsrn_malloc_async((void**)&sh.send, (size_t)count * sizeof(double), p->stream));
  LSRN_CUDA_TRY(lsrn_malloc_async((void**)&sh.recv, (size_t)count * sh.world * sizeof(double),
                                  p->stream));
  sh.cap = count;
  return LSRN_OK;
}

// send <- the values, wait for them, gather through the callback
lsrn_status gather(Plan* p, int64_t count) {
  LSRN_CUDA_TRY(cudaStreamSynchronize(p->stream));
  const int32_t rc = p->shard.fn(p->shard.ctx, p->shard.send, p->shard.recv, count);
  if (rc != 0) {
    record_cuda_error(cudaSuccess, "allgather callback of a sharded plan returned nonzero",
                      __FILE__, __LINE__);
    return LSRN_ERR_COMM;
  }
  return LSRN_OK;
}

}  // namespace

lsrn_status shard_sum(Plan* p, double* buf, int64_t count) {
  if (!p->sharded || count <= 0) return LSRN_OK;
  LSRN_TRY(ensure_staging(p, count));
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->shard.send, buf, (size_t)count * sizeof(double),
                                cudaMemcpyDeviceToDevice, p->stream));
  LSRN_TRY(gather(p, count));
  launch(shard_sum_kernel, grid_of(count), 256, 0, p->stream, (const double*)p->shard.recv,
         p->shard.world, count, buf);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

lsrn_status shard_sum_dd(Plan* p, double* hi, double* lo, int64_t count) {
  if (!p->sharded || count <= 0) return LSRN_OK;
  LSRN_TRY(ensure_staging(p, 2 * count));
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->shard.send, hi, (size_t)count * sizeof(double),
                                cudaMemcpyDeviceToDevice, p->stream));
  LSRN_CUDA_TRY(cudaMemcpyAsync(p->shard.send + count, lo, (size_t)count * sizeof(double),
                                cudaMemcpyDeviceToDevice, p->stream));
  LSRN_TRY(gather(p, 2 * count));
  launch(shard_sum_dd_kernel, grid_of(count), 256, 0, p->stream, (const double*)p->shard.recv,
         p->shard.world, count, hi, lo);
  LSRN_CUDA_TRY(cudaGetLastError());
  return LSRN_OK;
}

}  // namespace lsrn
