// Continuous-batching request server: factor-and-solve jobs of mixed sizes
// arrive at any time, are admitted while their device-memory footprint fits
// the budget and a slot is free, and run concurrently on the device (one
// handle, stream and worker thread per slot).  Each job is Algorithm 1 with
// a step chosen from n alone (never from the load), then the solve with
// FP64 refinement for the reduced-precision dtypes, so a job's arithmetic --
// and its result -- is the same whether it runs alone or among others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gb_internal.cuh"

using Clock = std::chrono::steady_clock;

namespace gb {
namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

bool dev_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Step of a served job: a function of (n, dtype) only.
int64_t served_step(int64_t n, gb_dtype dt) {
  if (dt == GB_F64) return std::min<int64_t>(256, std::max<int64_t>(n, 1));
  if (n <= 512) return 64;
  if (n <= 2048) return 256;
  return 1024;
}

// Device bytes a job holds while it runs: the FP64 copy of A (refinement or
// host input), the factor, right-hand sides and solution, the refinement
// residual (with the digit planes of its tensor-core method) and the packed
// tensor-core operands.
// Leading dimension of a job's factor buffer: a multiple of 64 elements, so
// that every row starts on a 256-byte boundary and the tensor-core update's
// epilogue can reduce into it with TMA (its row pitch must be a multiple of
// 16 bytes); the factor's layout is the job's own business.
int64_t factor_ld(int64_t n) { return (n + 63) / 64 * 64; }

size_t footprint(const gb_request &r) {
  const size_t n = (size_t)r.n, k = (size_t)r.nrhs;
  const size_t fac = (r.dtype == GB_F64 ? 8 : 4) * n * (size_t)factor_ld(r.n);
  const size_t s = (size_t)served_step(r.n, r.dtype);
  const size_t planes = r.dtype == GB_MIX_BF16X3 ? 6 : 1;
  const size_t pack = (r.dtype >= GB_MIX_BF16) ? 2 * n * ((s + 63) / 64 * 64) * 2 * planes : 0;
  // refinement's residual by digit products (the default from this order)
  const size_t split = (r.dtype != GB_F64 && r.n >= SPLIT_RESIDUAL_MIN_N)
                           ? split_a_bytes(r.n) + split_x_bytes(r.n, r.nrhs, 1024)
                           : 0;
  return 8 * n * n + fac + 3 * 8 * n * k + pack + split + (8u << 20);
}

}  // namespace
}  // namespace gb

struct gb_server {
  struct Job {
    uint64_t ticket = 0;
    gb_request req{};
    size_t bytes = 0;
    Clock::time_point submitted, started, finished;
    gb_result result{};
    bool done = false;
  };
  struct Slot {
    gb_handle *h = nullptr;
    cudaStream_t stream = nullptr;
    std::thread thread;
    Job *job = nullptr;  // assigned work (guarded by mu)
  };
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_slots = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_work, cv_done;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  std::vector<Slot> slots;
  std::thread scheduler;
  bool stop = false;
  uint64_t next_ticket = 1;
  int running = 0, max_running = 0;
  uint64_t completed = 0, rejected = 0;
  std::vector<double> latencies_ms;  // total latency of completed jobs
  Clock::time_point first_submit{}, last_finish{};
  bool any_submit = false;
};

namespace gb {
namespace {

// Run one job on a slot's handle and stream.
void run_job(gb_server *S, gb_server::Slot &slot, gb_server::Job &J) {
  const gb_request &r = J.req;
  gb_handle *h = slot.h;
  cudaStream_t st = slot.stream;
  gb_result &res = J.result;
  const int64_t n = r.n, k = r.nrhs;
  const bool refine = r.dtype != GB_F64;
  const int64_t s = r.s > 0 ? r.s : served_step(n, r.dtype);
  double *dA = nullptr, *dB = nullptr, *dX = nullptr;
  void *dL = nullptr;
  int *dinfo = nullptr;
  gb_status st_all = GB_OK;
  auto fail = [&](gb_status e) {
    if (st_all == GB_OK) st_all = e;
  };
  const bool a_dev = dev_ptr(r.A), b_dev = dev_ptr(r.B), x_dev = dev_ptr(r.X);
  const int64_t lda = a_dev ? r.lda : n, ldb = b_dev ? r.ldb : k, ldx = x_dev ? r.ldx : k;
  if (cudaMallocAsync((void **)&dinfo, sizeof(int), st) != cudaSuccess) fail(GB_ERR_NOMEM);
  if (!a_dev && cudaMallocAsync((void **)&dA, 8 * (size_t)n * n, st) != cudaSuccess) fail(GB_ERR_NOMEM);
  if (!b_dev && cudaMallocAsync((void **)&dB, 8 * (size_t)n * k, st) != cudaSuccess) fail(GB_ERR_NOMEM);
  if (!x_dev && cudaMallocAsync((void **)&dX, 8 * (size_t)n * k, st) != cudaSuccess) fail(GB_ERR_NOMEM);
  const int64_t ldl = factor_ld(n);
  if (cudaMallocAsync(&dL, (r.dtype == GB_F64 ? 8 : 4) * (size_t)n * ldl, st) != cudaSuccess)
    fail(GB_ERR_NOMEM);
  const double *A = a_dev ? r.A : dA;
  const double *B = b_dev ? r.B : dB;
  double *X = x_dev ? r.X : dX;
  if (st_all == GB_OK && !a_dev &&
      cudaMemcpy2DAsync(dA, n * 8, r.A, r.lda * 8, n * 8, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    fail(GB_ERR_CUDA);
  if (st_all == GB_OK && !b_dev &&
      cudaMemcpy2DAsync(dB, k * 8, r.B, r.ldb * 8, k * 8, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    fail(GB_ERR_CUDA);
  int info = 0;
  if (st_all == GB_OK) {
    gb_status e;
    if (r.dtype == GB_F32) {
      // GB_F32 factors read float input: cast A's lower triangle into the
      // factor buffer and factor it in place
      const cudaError_t ce = launch_copy_matrix<double, float>(A, lda, (float *)dL, ldl, n, true, st);
      e = ce == cudaSuccess ? gb_chol_factor(h, n, s, r.dtype, dL, ldl, dL, ldl, dinfo, st)
                            : GB_ERR_CUDA;
    } else {
      e = gb_chol_factor(h, n, s, r.dtype, A, lda, dL, ldl, dinfo, st);
    }
    if (e != GB_OK) fail(e);
  }
  if (st_all == GB_OK) {
    if (cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      fail(GB_ERR_CUDA);
  }
  gb_solve_stats stats{0, 0, 0.0};
  if (st_all == GB_OK && info == 0) {
    gb_refine_opts opts{r.tol > 0 ? r.tol : 1e-14, r.max_iter > 0 ? r.max_iter : 30};
    gb_status e = gb_chol_solve(h, n, k, r.dtype, dL, ldl, refine ? A : nullptr, lda, B, ldb, X,
                                ldx, &opts, &stats, st);
    if (e != GB_OK) fail(e);
    if (!x_dev && (e == GB_OK || e == GB_ERR_NOT_CONVERGED) &&
        cudaMemcpy2DAsync(r.X, r.ldx * 8, dX, k * 8, k * 8, n, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
      fail(GB_ERR_CUDA);
  }
  cudaStreamSynchronize(st);
  for (void *p : {(void *)dA, (void *)dB, (void *)dX, dL, (void *)dinfo})
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  res.status = st_all;
  res.info = info;
  res.iterations = stats.iterations;
  res.eta = stats.eta;
  (void)S;
}

void worker_loop(gb_server *S, int idx) {
  cudaSetDevice(S->device);
  for (;;) {
    gb_server::Job *J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || S->slots[idx].job != nullptr; });
      if (S->slots[idx].job == nullptr && S->stop) return;
      J = S->slots[idx].job;
    }
    run_job(S, S->slots[idx], *J);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      J->finished = Clock::now();
      J->result.queue_ms = ms_between(J->submitted, J->started);
      J->result.compute_ms = ms_between(J->started, J->finished);
      J->result.total_ms = ms_between(J->submitted, J->finished);
      J->done = true;
      S->latencies_ms.push_back(J->result.total_ms);
      S->completed++;
      S->last_finish = J->finished;
      S->in_use -= J->bytes;
      S->running--;
      S->slots[idx].job = nullptr;
    }
    S->cv_sched.notify_all();
    S->cv_done.notify_all();
  }
}

// FIFO admission: the head of the queue starts as soon as a slot is free
// and its footprint fits the remaining budget.
void scheduler_loop(gb_server *S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_sched.wait(lk, [&] {
      if (S->stop) return true;
      if (S->queue.empty()) return false;
      if (S->in_use + S->queue.front()->bytes > S->budget) return false;
      for (auto &sl : S->slots)
        if (!sl.job) return true;
      return false;
    });
    if (S->stop) return;
    gb_server::Job *J = S->queue.front();
    S->queue.pop_front();
    for (auto &sl : S->slots) {
      if (sl.job) continue;
      sl.job = J;
      break;
    }
    S->in_use += J->bytes;
    S->running++;
    S->max_running = std::max(S->max_running, S->running);
    J->started = Clock::now();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" gb_status gb_server_create(int device, size_t hbm_budget, int max_slots,
                                      gb_server **out) {
  if (!out) return -4;
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64) return -3;
  gb_server *S = new (std::nothrow) gb_server();
  if (!S) return GB_ERR_NOMEM;
  S->device = device;
  S->max_slots = max_slots;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return GB_ERR_CUDA;
  }
  if (hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    hbm_budget = free_b / 10 * 8;  // 80% of the free memory
  }
  S->budget = hbm_budget;
  S->slots.resize(max_slots);
  for (auto &sl : S->slots) {
    gb_status e = gb_create(&sl.h, device);
    if (e != GB_OK || cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto &t : S->slots) {
        if (t.h) gb_destroy(t.h);
        if (t.stream) cudaStreamDestroy(t.stream);
      }
      delete S;
      return e != GB_OK ? e : GB_ERR_CUDA;
    }
  }
  for (int i = 0; i < max_slots; ++i) S->slots[i].thread = std::thread(worker_loop, S, i);
  S->scheduler = std::thread(scheduler_loop, S);
  *out = S;
  return GB_OK;
}

extern "C" gb_status gb_server_submit(gb_server *S, const gb_request *r, uint64_t *ticket) {
  if (!S) return -1;
  if (!r) return -2;
  if (!ticket) return -3;
  if (r->n < 1 || r->nrhs < 1) return -2;
  if (r->dtype < GB_F64 || r->dtype > GB_MIX_BF16X3) return -2;
  if (!r->A || !r->B || !r->X) return -2;
  if (r->lda < r->n || r->ldb < r->nrhs || r->ldx < r->nrhs) return -2;
  auto *J = new (std::nothrow) gb_server::Job();
  if (!J) return GB_ERR_NOMEM;
  J->req = *r;
  J->bytes = footprint(*r);
  std::lock_guard<std::mutex> lk(S->mu);
  if (J->bytes > S->budget) {
    S->rejected++;
    delete J;
    return GB_ERR_REJECTED;
  }
  J->ticket = S->next_ticket++;
  J->submitted = Clock::now();
  if (!S->any_submit) {
    S->first_submit = J->submitted;
    S->any_submit = true;
  }
  S->jobs[J->ticket] = J;
  S->queue.push_back(J);
  *ticket = J->ticket;
  S->cv_sched.notify_all();
  return GB_OK;
}

extern "C" gb_status gb_server_wait(gb_server *S, uint64_t ticket, double timeout_s,
                                    gb_result *out) {
  if (!S) return -1;
  if (!out) return -4;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return -2;
  gb_server::Job *J = it->second;
  auto ready = [&] { return J->done; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return GB_ERR_TIMEOUT;
  }
  *out = J->result;
  S->jobs.erase(it);
  delete J;
  return GB_OK;
}

extern "C" gb_status gb_server_poll(gb_server *S, uint64_t ticket, gb_result *out) {
  const gb_status r = gb_server_wait(S, ticket, 0.0, out);
  return r == GB_ERR_TIMEOUT ? GB_ERR_STATE : r;
}

extern "C" gb_status gb_server_get_stats(gb_server *S, gb_server_stats *out) {
  if (!S) return -1;
  if (!out) return -2;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
    return v[i];
  };
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->queued = S->queue.size();
  out->running = S->running;
  out->max_running = S->max_running;
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->max_ms = v.empty() ? 0.0 : v.back();
  const double span = S->any_submit && S->completed ? ms_between(S->first_submit, S->last_finish) : 0.0;
  out->solves_per_s = span > 0 ? 1e3 * (double)S->completed / span : 0.0;
  out->budget_bytes = S->budget;
  out->bytes_in_use = S->in_use;
  return GB_OK;
}

extern "C" gb_status gb_server_reset_stats(gb_server *S) {
  if (!S) return -1;
  std::lock_guard<std::mutex> lk(S->mu);
  S->latencies_ms.clear();
  S->completed = 0;
  S->rejected = 0;
  S->max_running = S->running;
  S->any_submit = false;
  return GB_OK;
}

extern "C" gb_status gb_server_destroy(gb_server *S) {
  if (!S) return GB_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // let admitted and queued work finish
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_work.notify_all();
  if (S->scheduler.joinable()) S->scheduler.join();
  for (auto &sl : S->slots)
    if (sl.thread.joinable()) sl.thread.join();
  for (auto &sl : S->slots) {
    if (sl.h) gb_destroy(sl.h);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  for (auto &kv : S->jobs) delete kv.second;
  delete S;
  return GB_OK;
}
