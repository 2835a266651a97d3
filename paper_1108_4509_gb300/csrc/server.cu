// Request server: eigenproblems of different sizes are submitted as they
// arrive and solved concurrently on one GPU (continuous batching of whole
// solves). A request is admitted, in arrival order, while the device
// footprints of the live solves fit the memory budget and fewer than
// max_live solves run; each live solve has its own CUDA stream and host
// thread, so the kernels of different solves overlap on the device and a
// short problem never waits behind a long one that is already running.
// Results are those of trm_solve on a private handle: the same bytes alone
// and in the mix (every reduction in the library has a fixed order).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  trm_problem p{};
  std::vector<double> V;   // copy of the caller's potential
  std::vector<double> C0;  // copy of the caller's warm start (or empty)
  size_t bytes = 0;
  int status = TRM_OK;
  std::string err;
  std::vector<double> lambda;
  double E_G = 0.0;
  trm_stats stats{};
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  bool claimed = false;  // a caller is waiting on (or has taken) the result
};

}  // namespace

struct trm_server_ctx {
  size_t budget = 0;
  int max_live = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;  // any state change
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<int64_t, std::shared_ptr<Request>> requests;
  size_t in_use = 0;
  int live = 0;
  bool stop = false;
  int64_t next_id = 1;
  std::thread scheduler;
  trm_server_fn fn = nullptr;  // set: requests call it instead of solving
  void* fn_ctx = nullptr;
};

namespace {

// A request is done: record its result and return its memory and slot.
void finish(trm_server_ctx* s, const std::shared_ptr<Request>& r, int status,
            const std::string& err) {
  std::lock_guard<std::mutex> lock(s->mu);
  r->status = status;
  r->err = err;
  r->t_done = Clock::now();
  r->done = true;
  s->in_use -= r->bytes;
  s->live -= 1;
  s->cv.notify_all();
}

void run_request(trm_server_ctx* s, std::shared_ptr<Request> r) {
  int status = TRM_OK;
  std::string err;
  if (s->fn) {
    r->lambda.assign(r->p.m, 0.0);
    status = s->fn(&r->p, r->lambda.data(), &r->E_G, &r->stats, s->fn_ctx);
    if (status != TRM_OK) err = "the server's solve function failed";
    finish(s, r, status, err);
    return;
  }
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    status = TRM_ECUDA;
    err = "stream creation failed";
  }
  if (status == TRM_OK) {
    trm_options o = r->p.opt;
    o.stream = st;
    trm_handle h = nullptr;
    status = trm_create_stencil(&h, r->p.nx, r->p.ny, r->p.nz, r->p.order,
                                r->p.h, r->V.empty() ? nullptr : r->V.data(),
                                r->p.m, r->p.tol, &o);
    if (status != TRM_OK) {
      err = trm_last_global_error();
    } else {
      r->lambda.assign(r->p.m, 0.0);
      status = trm_solve(h, r->lambda.data(), &r->E_G, r->p.C_out, 0,
                         r->C0.empty() ? nullptr : r->C0.data(), &r->stats);
      if (status != TRM_OK) err = trm_last_error(h);
      trm_destroy(h);
    }
    cudaStreamDestroy(st);
  }
  finish(s, r, status, err);
}

void schedule(trm_server_ctx* s) {
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    s->cv.wait(lock, [s] {
      if (s->stop && s->pending.empty()) return true;
      if (s->pending.empty()) return false;
      const auto& head = s->pending.front();
      return s->live < s->max_live && s->in_use + head->bytes <= s->budget;
    });
    if (s->stop && s->pending.empty()) return;
    auto r = s->pending.front();
    s->pending.pop_front();
    s->in_use += r->bytes;
    s->live += 1;
    r->t_start = Clock::now();
    std::thread(run_request, s, r).detach();
  }
}

}  // namespace

extern "C" {

size_t trm_footprint_bytes(int64_t N, int m) {
  if (N < 2 || m < 1) return 0;
  return trm::Solver::footprint(N, m);
}

trm_status trm_server_create(trm_server* out, size_t device_bytes,
                             int max_live) {
  if (!out) return TRM_EINVAL;
  *out = nullptr;
  if (device_bytes == 0 || max_live < 1) {
    trm::set_global_error("device_bytes and max_live must be positive");
    return TRM_EINVAL;
  }
  auto* s = new (std::nothrow) trm_server_ctx;
  if (!s) return TRM_ENOMEM;
  s->budget = device_bytes;
  s->max_live = max_live;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    trm::set_global_error("no CUDA device");
    return TRM_ECUDA;
  }
  s->scheduler = std::thread(schedule, s);
  *out = s;
  return TRM_OK;
}

trm_status trm_server_create_fn(trm_server* out, size_t device_bytes,
                                int max_live, trm_server_fn fn, void* ctx) {
  if (!out) return TRM_EINVAL;
  *out = nullptr;
  if (device_bytes == 0 || max_live < 1 || !fn) {
    trm::set_global_error("device_bytes and max_live must be positive and fn non-NULL");
    return TRM_EINVAL;
  }
  auto* s = new (std::nothrow) trm_server_ctx;
  if (!s) return TRM_ENOMEM;
  s->budget = device_bytes;
  s->max_live = max_live;
  s->fn = fn;
  s->fn_ctx = ctx;
  s->scheduler = std::thread(schedule, s);
  *out = s;
  return TRM_OK;
}

trm_status trm_server_submit(trm_server s, const trm_problem* p,
                             int64_t* ticket) {
  if (!s || !p || !ticket) return TRM_EINVAL;
  const int64_t N = (int64_t)p->nx * p->ny * p->nz;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->m < 1 || p->m >= N ||
      p->m > 1024) {
    trm::set_global_error("need grid dimensions >= 1 and 1 <= m < N, m <= 1024");
    return TRM_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->p = *p;
  if (p->V) r->V.assign(p->V, p->V + N);
  r->p.V = nullptr;
  if (p->C0) r->C0.assign(p->C0, p->C0 + N * p->m);
  r->p.C0 = nullptr;
  r->bytes = trm::Solver::footprint(N, p->m);
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return TRM_EINVAL;
  if (r->bytes > s->budget) {
    trm::set_global_error("the problem's device footprint exceeds the budget");
    return TRM_ENOMEM;
  }
  r->id = s->next_id++;
  r->t_submit = Clock::now();
  s->requests[r->id] = r;
  s->pending.push_back(r);
  *ticket = r->id;
  s->cv.notify_all();
  return TRM_OK;
}

trm_status trm_server_wait(trm_server s, int64_t ticket, double* lambda,
                           double* E_G, trm_stats* stats, double* latency) {
  if (!s) return TRM_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) {
      trm::set_global_error("unknown ticket");
      return TRM_EINVAL;
    }
    r = it->second;
    if (r->claimed) {
      trm::set_global_error("another caller is already waiting on this ticket");
      return TRM_EINVAL;
    }
    r->claimed = true;
    // the wait releases the lock: a submit may rehash the map meanwhile, so
    // the entry is removed by key afterwards, not through the iterator
    s->cv.wait(lock, [&] { return r->done; });
    s->requests.erase(ticket);
  }
  if (lambda && !r->lambda.empty())
    std::copy(r->lambda.begin(), r->lambda.end(), lambda);
  if (E_G) *E_G = r->E_G;
  if (stats) *stats = r->stats;
  if (latency)
    *latency = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (r->status != TRM_OK) trm::set_global_error(r->err);
  return static_cast<trm_status>(r->status);
}

trm_status trm_server_destroy(trm_server s) {
  if (!s) return TRM_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->scheduler.join();  // returns once nothing is pending
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv.wait(lock, [s] { return s->live == 0; });
  }
  delete s;
  return TRM_OK;
}

}  // extern "C"
