// Serving front end: a request queue with admission by a device-memory budget.
//
// lsrn_submit copies a request (A into server-owned device memory, b and the
// options into host memory), queues it and returns a ticket.  Worker threads,
// one per slot and each with its own CUDA stream, take the oldest queued
// request whose estimated device footprint fits the remaining budget, run
// lsrn_plan + lsrn_solve_* on it, and park the result until lsrn_poll collects
// it.  Requests admitted together run concurrently on the device; each plan's
// arithmetic has a fixed order, so a result does not depend on what ran beside
// it.  Their preconditioners (short side up to 128) are packed by the batcher
// below into shared launches of the batched preconditioner kernel, which
// computes each problem as the per-problem kernels do.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lsrn.h"
#include "lsrn_internal.h"

namespace {

struct Request {
  uint64_t ticket = 0;
  lsrn_matrix A{};            // points into the owned copies below
  void* dev_values = nullptr;
  int64_t* dev_rp = nullptr;
  int32_t* dev_ci = nullptr;
  std::vector<double> b;
  lsrn_options opt{};
  int32_t solver = 0;
  size_t bytes = 0;           // admission estimate (includes the copy of A)
};

struct Result {
  bool done = false;
  lsrn_status status = LSRN_PENDING;
  std::vector<double> x;
  lsrn_info info{};
};

size_t estimate_bytes(const lsrn_matrix& A, const lsrn_options& o) {
  const int64_t m = A.m, n = A.n;
  const bool tall = m >= n;
  const int64_t q = tall ? n : m, rows = tall ? m : n;
  const int64_t extra = o.lambda > 0 ? q : 0;
  const int64_t s = (int64_t)std::ceil(o.gamma * (double)q) + 1;
  size_t a_bytes;
  if (A.format == LSRN_CSR)
    a_bytes = (size_t)(A.m + 1) * 8 + (size_t)A.nnz * 12 * 2 + (size_t)(A.n + 1) * 8;
  else
    a_bytes = (size_t)m * n * 8 * 2;   // owned copy + possible re-layout
  size_t work = 8 * ((size_t)s * q + 3 * (size_t)q * q + 6 * (size_t)(rows + extra) + 16 * (size_t)q);
  const int32_t iter = lsrn::resolve_iter_mode(o.iter_mode, m, n, A.format == LSRN_CSR);
  if (iter == LSRN_ITER_F32 && A.format != LSRN_CSR) work += (size_t)m * n * 4;
  if (iter == LSRN_ITER_F32X2 && A.format != LSRN_CSR) work += (size_t)m * n * 12;   // 3 planes
  if ((o.sketch_mode == LSRN_SKETCH_TC_SLICED || o.sketch_mode == LSRN_SKETCH_AUTO) &&
      A.format != LSRN_CSR)   // the plan's exact sizing
    work += lsrn::sketch_tc_scratch_bytes(lsrn::sketch_tc_plan_segment_rows(rows, q, s - 1), q, s - 1);
  if ((o.sketch_mode == LSRN_SKETCH_BF16 || o.sketch_mode == LSRN_SKETCH_AUTO) && A.format != LSRN_CSR)
    work += lsrn::sketch_bf16_scratch_bytes(
        lsrn::sketch_bf16_segment_rows(rows, q, s - 1, lsrn::kTcScratchBudget), q, s - 1);
  return a_bytes + work + ((size_t)64 << 20);
}

// Continuous batching of the preconditioner phase: workers that reach it hand
// their sketched plan over; the batcher packs the plans into one launch of the
// batched preconditioner kernel, then releases the workers into their
// iterations.  A worker announces an eligible plan before its sketch
// (expect), so after the first arrival the batcher waits, up to kGatherMs,
// until every announced plan has arrived; then it packs all waiting plans.
struct PrecondBatcher {
  struct Item {
    lsrn::Plan* plan;
    lsrn_status status;
    bool done;
  };
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Item*> pending;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> th;   // several batchers: a long batch does not hold up the next
  uint64_t batches = 0, packed = 0;
  int expecting = 0;             // announced plans still sketching
  static constexpr int kGatherMs = 2;

  void expect(int d) {
    {
      std::lock_guard<std::mutex> lk(mu);
      expecting += d;
    }
    cv.notify_all();
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Item*> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !pending.empty(); });
        if (pending.empty()) return;   // stopping with nothing left
        // gather: the announced plans still sketching, for at most kGatherMs
        cv.wait_for(lk, std::chrono::milliseconds(kGatherMs), [&] { return stop || expecting <= 0; });
        if (pending.empty()) continue;   // another batcher took them meanwhile
        batch.assign(pending.begin(), pending.end());
        pending.clear();
      }
      std::vector<lsrn::Plan*> ps;
      for (Item* it : batch) ps.push_back(it->plan);
      std::vector<lsrn_status> st(ps.size(), LSRN_OK);
      lsrn::precond_batch(ps, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t k = 0; k < batch.size(); ++k) {
          batch[k]->status = st[k];
          batch[k]->done = true;
        }
        batches += 1;
        packed += batch.size();
      }
      cv.notify_all();
    }
  }

  // The plan must have been announced with expect(+1).
  lsrn_status submit(lsrn::Plan* p) {
    Item it{p, LSRN_OK, false};
    std::unique_lock<std::mutex> lk(mu);
    --expecting;
    pending.push_back(&it);
    cv.notify_all();
    cv.wait(lk, [&] { return it.done; });
    return it.status;
  }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    for (auto& t : th)
      if (t.joinable()) t.join();
  }
};

}  // namespace

struct lsrn_server_s {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Result> results;
  std::vector<std::thread> workers;
  PrecondBatcher batcher;
  std::atomic<int> batch_max_q{0};   // 0: every request preconditions on its own

  void worker_loop() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      Request* req = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stopping) break;   // requests not yet started are dropped by destroy
          auto it = std::find_if(queue.begin(), queue.end(),
                                 [&](Request* r) { return in_use + r->bytes <= budget; });
          if (it != queue.end()) {
            req = *it;
            queue.erase(it);
            in_use += req->bytes;
            break;
          }
          cv.wait(lk);
        }
      }
      if (req == nullptr) break;
      Result res;
      lsrn_plan_t plan = nullptr;
      res.x.assign((size_t)req->A.n, 0.0);
      lsrn_status s = lsrn_plan(&req->A, &req->opt, st, &plan);
      if (s == LSRN_OK) {
        lsrn::plan_disable_sweep_graphs(plan);
        const int bq = batch_max_q.load();
        if (bq > 0 && lsrn::plan_short_side(plan) <= bq &&
            lsrn::batch_precond_applies(lsrn::plan_short_side(plan))) {
          batcher.expect(+1);
          s = lsrn_sketch(plan);
          if (s == LSRN_OK && lsrn::precond_batchable(lsrn::plan_internal(plan)))
            s = batcher.submit(lsrn::plan_internal(plan));
          else
            batcher.expect(-1);   // not coming: the batcher stops waiting for it
        }
      }
      if (s == LSRN_OK) {
        s = req->solver == 1 ? lsrn_solve_cs(plan, req->b.data(), res.x.data(), &res.info)
                             : lsrn_solve_lsqr(plan, req->b.data(), res.x.data(), &res.info);
        lsrn_plan_destroy(plan);
      }
      res.status = s;
      res.done = true;
      if (req->dev_values) cudaFree(req->dev_values);
      if (req->dev_rp) cudaFree(req->dev_rp);
      if (req->dev_ci) cudaFree(req->dev_ci);
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= req->bytes;
        results[req->ticket] = std::move(res);
      }
      cv.notify_all();
      delete req;
    }
    cudaStreamDestroy(st);
  }
};

extern "C" {

lsrn_status lsrn_server_create(size_t hbm_budget_bytes, int32_t max_slots, lsrn_server_t* out) {
  if (out == nullptr || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0)
    return LSRN_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LSRN_ERR_CUDA;
  }
  lsrn_server_s* s = new (std::nothrow) lsrn_server_s();
  if (s == nullptr) return LSRN_ERR_OOM;
  cudaGetDevice(&s->device);
  s->budget = hbm_budget_bytes;
  s->batcher.device = s->device;
  for (int i = 0; i < 4; ++i) s->batcher.th.emplace_back([s] { s->batcher.run(); });
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s] { s->worker_loop(); });
  *out = s;
  return LSRN_OK;
}

lsrn_status lsrn_submit(lsrn_server_t s, const lsrn_matrix* A, const double* b,
                        const lsrn_options* opt, int32_t solver, uint64_t* ticket) {
  if (s == nullptr || A == nullptr || b == nullptr || ticket == nullptr) return LSRN_ERR_INVALID_ARG;
  if (solver != 0 && solver != 1) return LSRN_ERR_INVALID_ARG;
  if (A->m < 1 || A->n < 1 || A->values == nullptr) return LSRN_ERR_INVALID_ARG;
  if (A->format == LSRN_CSR && (A->row_ptr == nullptr || A->col_idx == nullptr || A->nnz < 0))
    return LSRN_ERR_INVALID_ARG;
  if (A->format != LSRN_CSR && A->ld < (A->format == LSRN_DENSE_ROWMAJOR ? A->n : A->m))
    return LSRN_ERR_INVALID_ARG;
  Request* r = new (std::nothrow) Request();
  if (r == nullptr) return LSRN_ERR_OOM;
  if (opt) r->opt = *opt;
  else lsrn_default_options(&r->opt);
  r->solver = solver;
  r->A = *A;
  r->bytes = estimate_bytes(*A, r->opt);
  if (r->bytes > s->budget) {
    delete r;
    return LSRN_ERR_QUEUE_FULL;
  }
  cudaSetDevice(s->device);
  // copy A into server-owned device memory (host or device source)
  const size_t esz = A->dtype == LSRN_F32 ? 4 : 8;
  size_t vbytes;
  if (A->format == LSRN_CSR) vbytes = (size_t)A->nnz * esz;
  else if (A->format == LSRN_DENSE_ROWMAJOR) vbytes = ((size_t)(A->m - 1) * A->ld + A->n) * esz;
  else vbytes = ((size_t)(A->n - 1) * A->ld + A->m) * esz;
  cudaError_t e = cudaMalloc(&r->dev_values, std::max<size_t>(vbytes, 16));
  if (e == cudaSuccess) e = cudaMemcpy(r->dev_values, A->values, vbytes, cudaMemcpyDefault);
  if (e == cudaSuccess && A->format == LSRN_CSR) {
    e = cudaMalloc((void**)&r->dev_rp, (size_t)(A->m + 1) * 8);
    if (e == cudaSuccess) e = cudaMemcpy(r->dev_rp, A->row_ptr, (size_t)(A->m + 1) * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMalloc((void**)&r->dev_ci, std::max<size_t>((size_t)A->nnz * 4, 16));
    if (e == cudaSuccess && A->nnz > 0)
      e = cudaMemcpy(r->dev_ci, A->col_idx, (size_t)A->nnz * 4, cudaMemcpyDefault);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (r->dev_values) cudaFree(r->dev_values);
    if (r->dev_rp) cudaFree(r->dev_rp);
    if (r->dev_ci) cudaFree(r->dev_ci);
    delete r;
    return e == cudaErrorMemoryAllocation ? LSRN_ERR_OOM : LSRN_ERR_CUDA;
  }
  r->A.values = r->dev_values;
  r->A.row_ptr = r->dev_rp;
  r->A.col_idx = r->dev_ci;
  r->b.resize((size_t)A->m);
  if (cudaMemcpy(r->b.data(), b, (size_t)A->m * 8, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(r->dev_values);
    if (r->dev_rp) cudaFree(r->dev_rp);
    if (r->dev_ci) cudaFree(r->dev_ci);
    delete r;
    return LSRN_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      cudaFree(r->dev_values);
      delete r;
      return LSRN_ERR_STATE;
    }
    r->ticket = s->next_ticket++;
    s->results[r->ticket] = Result();
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return LSRN_OK;
}

lsrn_status lsrn_server_set_batching(lsrn_server_t s, int32_t max_short_side) {
  if (s == nullptr || max_short_side < 0 || max_short_side > 512) return LSRN_ERR_INVALID_ARG;
  s->batch_max_q.store(max_short_side);
  return LSRN_OK;
}

lsrn_status lsrn_server_stats(lsrn_server_t s, uint64_t* batches, uint64_t* batched_requests) {
  if (s == nullptr) return LSRN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->batcher.mu);
  if (batches) *batches = s->batcher.batches;
  if (batched_requests) *batched_requests = s->batcher.packed;
  return LSRN_OK;
}

lsrn_status lsrn_poll(lsrn_server_t s, uint64_t ticket, double* x_out, lsrn_info* info) {
  if (s == nullptr) return LSRN_ERR_INVALID_ARG;
  Result res;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return LSRN_ERR_INVALID_ARG;
    if (!it->second.done) return LSRN_PENDING;
    res = std::move(it->second);
    s->results.erase(it);
  }
  if (x_out != nullptr && !res.x.empty()) {
    cudaSetDevice(s->device);
    if (cudaMemcpy(x_out, res.x.data(), res.x.size() * 8, cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      return LSRN_ERR_CUDA;
    }
  }
  if (info) *info = res.info;
  return res.status;
}

lsrn_status lsrn_server_destroy(lsrn_server_t s) {
  if (s == nullptr) return LSRN_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  s->batcher.shutdown();
  for (Request* r : s->queue) {
    if (r->dev_values) cudaFree(r->dev_values);
    if (r->dev_rp) cudaFree(r->dev_rp);
    if (r->dev_ci) cudaFree(r->dev_ci);
    delete r;
  }
  delete s;
  return LSRN_OK;
}

}  // extern "C"
