// The request server's scheduler under the host sanitizers: several client
// threads submit and wait concurrently on one server whose requests run a
// host function (trm_server_create_fn); then one thread keeps submitting a
// burst (the ticket table grows and rehashes) while others wait on earlier
// tickets; then two threads wait on the same ticket, and exactly one of them
// may get the result. Exit code 0 when every result and status reached its
// ticket and the bound on concurrent requests held.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <mutex>
#include <thread>
#include <vector>

#include "trm.h"

namespace {

std::atomic<int> g_live{0}, g_max_live{0};

int run(const trm_problem* p, double* lambda, double* E_G, trm_stats* stats,
        void*) {
  const int live = ++g_live;
  int seen = g_max_live.load();
  while (live > seen && !g_max_live.compare_exchange_weak(seen, live)) {
  }
  std::this_thread::sleep_for(std::chrono::microseconds(300));
  const int id = (int)p->opt.seed;
  for (int j = 0; j < p->m; ++j) lambda[j] = id + j;
  *E_G = id;
  stats->iterations = id;
  --g_live;
  return id % 7 == 3 ? TRM_ENOCONV : TRM_OK;
}

trm_problem problem(int id, int k) {
  trm_problem p{};
  p.nx = p.ny = p.nz = 16;
  p.order = 2;
  p.h = 1.0;
  p.m = 8 + (k % 3) * 4;
  p.tol = 1e-8;
  p.opt.seed = (uint64_t)id;
  return p;
}

bool check(trm_server s, int64_t ticket, int id, int m) {
  double lambda[16], E_G = 0.0, latency = 0.0;
  trm_stats st{};
  const trm_status rc = trm_server_wait(s, ticket, lambda, &E_G, &st, &latency);
  const trm_status want = id % 7 == 3 ? TRM_ENOCONV : TRM_OK;
  bool ok = rc == want && E_G == id && st.iterations == id && latency > 0.0;
  for (int j = 0; j < m; ++j) ok = ok && lambda[j] == id + j;
  return ok;
}

// One thread submits kBurst requests without waiting while kWaiters threads
// take the tickets it publishes and wait on them.
int submit_while_waiting(trm_server s) {
  const int kBurst = 1500, kWaiters = 4;
  std::mutex mu;
  std::vector<std::pair<int64_t, int>> tickets;  // (ticket, id)
  std::atomic<bool> producing{true};
  std::atomic<int> bad{0}, taken{0};
  std::thread producer([&] {
    for (int k = 0; k < kBurst; ++k) {
      const int id = 50000 + k;
      trm_problem p = problem(id, k);
      int64_t t = 0;
      if (trm_server_submit(s, &p, &t) != TRM_OK) {
        ++bad;
        continue;
      }
      std::lock_guard<std::mutex> lock(mu);
      tickets.emplace_back(t, id);
    }
    producing = false;
  });
  std::vector<std::thread> waiters;
  for (int w = 0; w < kWaiters; ++w)
    waiters.emplace_back([&] {
      for (;;) {
        std::pair<int64_t, int> job{0, 0};
        {
          std::lock_guard<std::mutex> lock(mu);
          const int i = taken.load();
          if (i < (int)tickets.size()) {
            job = tickets[i];
            taken = i + 1;
          }
        }
        if (job.first == 0) {
          std::lock_guard<std::mutex> lock(mu);
          if (!producing && taken.load() >= (int)tickets.size()) return;
          continue;
        }
        if (!check(s, job.first, job.second, problem(job.second, job.second - 50000).m))
          ++bad;
      }
    });
  producer.join();
  for (auto& w : waiters) w.join();
  return bad.load() + (taken.load() == kBurst ? 0 : 1);
}

// Two threads wait on one ticket: one gets the result, the other TRM_EINVAL
// (the ticket is claimed, or already released).
int double_wait(trm_server s) {
  int bad = 0;
  for (int k = 0; k < 50; ++k) {
    const int id = 90000 + 7 * k + 1;  // id % 7 != 3: status TRM_OK
    trm_problem p = problem(id, k);
    int64_t t = 0;
    if (trm_server_submit(s, &p, &t) != TRM_OK) return 1;
    std::atomic<int> ok{0}, inval{0};
    auto wait = [&] {
      double lambda[16], E_G = 0.0;
      const trm_status rc = trm_server_wait(s, t, lambda, &E_G, nullptr, nullptr);
      if (rc == TRM_OK && E_G == id) ++ok;
      else if (rc == TRM_EINVAL) ++inval;
    };
    std::thread a(wait), b(wait);
    a.join();
    b.join();
    if (ok.load() != 1 || inval.load() != 1) ++bad;
  }
  return bad;
}

}  // namespace

int main() {
  const int kThreads = 6, kPerThread = 40, kMaxLive = 4;
  trm_server s = nullptr;
  const size_t fp = trm_footprint_bytes(16 * 16 * 16, 16);
  if (trm_server_create_fn(&s, 3 * fp, kMaxLive, run, nullptr) != TRM_OK)
    return 1;
  std::atomic<int> bad{0};
  std::vector<std::thread> clients;
  for (int t = 0; t < kThreads; ++t) {
    clients.emplace_back([&, t] {
      for (int k = 0; k < kPerThread; ++k) {
        const int id = t * 1000 + k;
        trm_problem p = problem(id, k);
        int64_t ticket = 0;
        if (trm_server_submit(s, &p, &ticket) != TRM_OK) {
          ++bad;
          continue;
        }
        if (!check(s, ticket, id, p.m)) ++bad;
      }
    });
  }
  for (auto& c : clients) c.join();
  const int bad_burst = submit_while_waiting(s);
  const int bad_double = double_wait(s);
  bad += bad_burst + bad_double;
  trm_server_destroy(s);
  std::printf("bad %d (burst %d, double wait %d) max_live %d\n", bad.load(),
              bad_burst, bad_double, g_max_live.load());
  return bad.load() == 0 && g_max_live.load() <= kMaxLive &&
                 g_max_live.load() >= 2
             ? 0
             : 2;
}
