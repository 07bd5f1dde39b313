// Request runtime: continuous batching of recovery jobs of mixed N, M, K,
// kind, precision and algorithm on one GPU (the paper has no counterpart; it
// is the serving side of the same path).
//
// A fixed set of worker threads each own one CUDA stream.  Submitted jobs
// wait in a queue; a worker admits the next job when its device footprint
// (plan tables, workspace, inputs and outputs: solve_footprint) fits in
// what the memory budget has left, builds the job's plan on its own stream,
// solves, copies the results back and releases everything on that stream.
// All device memory of a job is stream-ordered (cudaMallocAsync /
// cudaFreeAsync), so admitting or retiring a job never synchronises the
// device and the jobs of different workers overlap on the GPU.
//
// Admission is first come, first served with a bounded bypass: when the
// oldest job does not fit, a later one that fits may start, but once the
// oldest has been passed kMaxBypass times nothing else starts before it
// (no starvation of large jobs).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/csfast.h"
#include "cs_internal.h"

namespace csf {
cs_status plan_create_ordered(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                              cudaStream_t stream, cs_plan_t* out);
void plan_release_ordered(cs_plan_t plan);
size_t solve_footprint(int64_t N, int64_t M, int32_t kind, int32_t prec, int32_t K, int32_t algo);
void set_last_error(const char* msg);
}  // namespace csf

using namespace csf;

namespace {

constexpr int kMaxBypass = 8;

struct Job {
  int64_t ticket = 0;
  cs_request req{};
  std::vector<int32_t> omega;
  std::vector<unsigned char> y;
  void* x_host = nullptr;
  int32_t* supp_host = nullptr;
  double t_submit = 0.0;
  int64_t fp = 0;
  int bypassed = 0;
};

size_t elem_size(int kind, int prec) { return (kind == CS_DFT ? 2 : 1) * (prec == CS_FP32 ? 4 : 8); }

}  // namespace

struct cs_server_s {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::deque<cs_result> done;
  int64_t in_use = 0, running = 0, completed = 0, next_ticket = 1;
  bool closing = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  double now_us() const {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  }
};

extern "C" int32_t cs_admit_next(const int64_t* footprints, const int32_t* bypassed, int32_t n_pending,
                                 int64_t in_use, int64_t budget, int32_t max_bypass) {
  if (n_pending <= 0 || !footprints) return -1;
  if (in_use + footprints[0] <= budget) return 0;
  if (bypassed && bypassed[0] >= max_bypass) return -1;  // the oldest job waits for memory, nobody passes it
  for (int32_t i = 1; i < n_pending; ++i)
    if (in_use + footprints[i] <= budget) return i;
  return -1;
}

namespace {

// Index of the pending job to admit now, or -1; caller holds the lock.
int pick(cs_server_s* S) {
  const int n = (int)S->pending.size();
  if (n == 0) return -1;
  std::vector<int64_t> fp((size_t)n);
  std::vector<int32_t> by((size_t)n);
  for (int i = 0; i < n; ++i) {
    fp[(size_t)i] = S->pending[(size_t)i]->fp;
    by[(size_t)i] = S->pending[(size_t)i]->bypassed;
  }
  return cs_admit_next(fp.data(), by.data(), n, S->in_use, S->budget, kMaxBypass);
}

cs_result run_job(cs_server_s* S, Job* j, cudaStream_t st) {
  cs_result r{};
  r.ticket = j->ticket;
  r.t_submit_us = j->t_submit;
  r.t_admit_us = S->now_us();
  r.footprint_bytes = j->fp;
  const cs_request& q = j->req;
  const size_t eb = elem_size(q.kind, q.prec), wb = q.kind == CS_DFT ? 16 : 8;
  cs_plan_t plan = nullptr;
  void *y = nullptr, *x = nullptr;
  int32_t *supp = nullptr, *iters = nullptr;
  double* res = nullptr;
  int32_t it_h = 0;
  double rn_h = 0.0;
  cs_status s = plan_create_ordered(q.N, j->omega.data(), q.M, q.kind, q.prec, st, &plan);
  const size_t Kc = (size_t)(q.K > 0 ? q.K : 1);
  cudaError_t e = cudaSuccess;
  if (s == CS_OK) {
    e = cudaMallocAsync(&y, (size_t)(q.M > 0 ? q.M : 1) * eb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&x, Kc * wb, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&supp, Kc * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&iters, 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&res, 8, st);
    if (e == cudaSuccess && q.M > 0) e = cudaMemcpyAsync(y, j->y.data(), (size_t)q.M * eb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = e == cudaErrorMemoryAllocation ? CS_ERR_NOMEM : CS_ERR_CUDA;
  }
  if (s == CS_OK) {
    if (q.algo == CS_ALGO_OMP) s = cs_omp(plan, y, 1, q.K, &q.halt, x, supp, iters, res, st);
    else if (q.algo == CS_ALGO_COSAMP) s = cs_cosamp(plan, y, 1, q.K, &q.halt, x, supp, iters, res, st);
    else s = cs_sp(plan, y, 1, q.K, &q.halt, x, supp, iters, res, st);
  }
  if (s == CS_OK) {
    if (q.K > 0) {
      e = cudaMemcpyAsync(j->x_host, x, (size_t)q.K * wb, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(j->supp_host, supp, (size_t)q.K * 4, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&it_h, iters, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rn_h, res, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = CS_ERR_CUDA;
  }
  if (s == CS_OK) {
    int32_t dev_err = 0;
    s = cs_plan_status(plan, &dev_err, st);
    r.device_error = dev_err;
  }
  void* bufs[] = {y, x, supp, iters, res};
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, st);
  if (plan) plan_release_ordered(plan);
  cudaStreamSynchronize(st);  // the job's memory is back in the pool before the budget is credited
  r.status = s;
  r.iters = it_h;
  r.resnorm = rn_h;
  r.t_done_us = S->now_us();
  return r;
}

void worker(cs_server_s* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      int idx = -1;
      S->cv_work.wait(lk, [&] {
        if (S->closing && S->pending.empty()) return true;
        idx = pick(S);
        return idx >= 0;
      });
      if (idx < 0) break;  // closing and nothing left
      j = S->pending[(size_t)idx];
      for (int i = 0; i < idx; ++i) S->pending[(size_t)i]->bypassed++;
      S->pending.erase(S->pending.begin() + idx);
      S->in_use += j->fp;
      S->running++;
    }
    cs_result r{};
    if (ok) {
      r = run_job(S, j, st);
    } else {
      r.ticket = j->ticket;
      r.status = CS_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= j->fp;
      S->running--;
      S->completed++;
      S->done.push_back(r);
    }
    delete j;
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

cs_status check_request(const cs_request* q) {
  if (!q) return CS_ERR_INVALID;
  if (q->kind != CS_WHT && q->kind != CS_DFT) return CS_ERR_INVALID;
  if (q->prec != CS_FP64 && q->prec != CS_FP32) return CS_ERR_INVALID;
  if (q->N < 1 || (q->N & (q->N - 1)) || q->M < 0 || q->M > q->N) return CS_ERR_INVALID;
  if (q->M > 0 && (!q->omega_host || !q->y_host)) return CS_ERR_INVALID;
  if (q->N > (int64_t(1) << kMaxLogNLarge)) return CS_ERR_UNSUPPORTED;
  if (q->algo == CS_ALGO_OMP) {
    if (q->K < 0 || q->K > q->M) return CS_ERR_INVALID;
    if (q->K > (q->N > (int64_t(1) << kMaxLogN) ? kMaxKLarge : kMaxK)) return CS_ERR_UNSUPPORTED;
  } else if (q->algo == CS_ALGO_COSAMP || q->algo == CS_ALGO_SP) {
    if (q->K < 1 || (q->algo == CS_ALGO_SP ? 2 : 3) * (int64_t)q->K > q->M) return CS_ERR_INVALID;
    if (q->K > (q->N > (int64_t(1) << kMaxLogN) ? kMaxPursuitKLarge : kMaxPursuitK)) return CS_ERR_UNSUPPORTED;
  } else {
    return CS_ERR_INVALID;
  }
  for (int64_t m = 0; m < q->M; ++m) {
    if (q->omega_host[m] < 0 || q->omega_host[m] >= q->N) return CS_ERR_INVALID;
    if (m > 0 && q->omega_host[m] <= q->omega_host[m - 1]) return CS_ERR_INVALID;
  }
  return CS_OK;
}

}  // namespace

extern "C" cs_status cs_server_create(int32_t workers, int64_t hbm_budget_bytes, cs_server_t* out) {
  if (!out || workers < 1 || workers > 64 || hbm_budget_bytes <= 0) return CS_ERR_INVALID;
  *out = nullptr;
  cs_server_s* S = new (std::nothrow) cs_server_s();
  if (!S) return CS_ERR_NOMEM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    set_last_error("cs_server_create: no usable current device");
    return CS_ERR_CUDA;
  }
  S->budget = hbm_budget_bytes;
  S->t0 = std::chrono::steady_clock::now();
  // Keep up to the budget of freed job memory in the device's stream-ordered
  // pool instead of returning it to the CUDA driver at every synchronisation, so
  // that admitting a job reuses memory rather than allocating it anew.
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
    uint64_t cur = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur);
    uint64_t want = (uint64_t)hbm_budget_bytes;
    if (want > cur) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
  }
  for (int i = 0; i < workers; ++i) S->workers.emplace_back(worker, S);
  *out = S;
  return CS_OK;
}

extern "C" cs_status cs_server_submit(cs_server_t S, const cs_request* req, void* x_host, int32_t* supp_host,
                                      int64_t* ticket) {
  if (!S || !ticket) return CS_ERR_INVALID;
  const cs_status c = check_request(req);
  if (c != CS_OK) return c;
  if (req->K > 0 && (!x_host || !supp_host)) return CS_ERR_INVALID;
  const int64_t fp = (int64_t)solve_footprint(req->N, req->M, req->kind, req->prec, req->K, req->algo);
  if (fp > S->budget) {
    set_last_error("cs_server_submit: the job's device footprint exceeds the server's memory budget");
    return CS_ERR_NOMEM;
  }
  Job* j = new (std::nothrow) Job();
  if (!j) return CS_ERR_NOMEM;
  j->req = *req;
  j->omega.assign(req->omega_host, req->omega_host + req->M);
  const size_t yb = (size_t)req->M * elem_size(req->kind, req->prec);
  j->y.resize(yb);
  if (yb) std::memcpy(j->y.data(), req->y_host, yb);
  j->req.omega_host = nullptr;
  j->req.y_host = nullptr;
  j->x_host = x_host;
  j->supp_host = supp_host;
  j->fp = fp;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->closing) {
      delete j;
      return CS_ERR_INVALID;
    }
    j->ticket = S->next_ticket++;
    j->t_submit = S->now_us();
    *ticket = j->ticket;
    S->pending.push_back(j);
  }
  S->cv_work.notify_all();
  return CS_OK;
}

extern "C" cs_status cs_server_poll(cs_server_t S, cs_result* out, int32_t max, int32_t wait_ms, int32_t* n) {
  if (!S || !n || max < 0 || (max > 0 && !out)) return CS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  if (wait_ms > 0 && S->done.empty())
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  int32_t k = 0;
  while (k < max && !S->done.empty()) {
    out[k++] = S->done.front();
    S->done.pop_front();
  }
  *n = k;
  return CS_OK;
}

extern "C" cs_status cs_server_stats(cs_server_t S, int64_t* pending, int64_t* running, int64_t* completed,
                                     int64_t* bytes_in_use) {
  if (!S) return CS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  if (pending) *pending = (int64_t)S->pending.size();
  if (running) *running = S->running;
  if (completed) *completed = S->completed;
  if (bytes_in_use) *bytes_in_use = S->in_use;
  return CS_OK;
}

extern "C" cs_status cs_server_destroy(cs_server_t S) {
  if (!S) return CS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->closing = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return CS_OK;
}
