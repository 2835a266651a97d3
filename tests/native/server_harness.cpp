// The request server's scheduler under the host sanitizers: several client
// threads submit and wait concurrently on one server whose requests run a
// host function (trm_server_create_fn). Exit code 0 when every result and
// status reached its ticket and the bound on concurrent requests held.
#include <atomic>
#include <chrono>
#include <cstdio>
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
        trm_problem p{};
        p.nx = p.ny = p.nz = 16;
        p.order = 2;
        p.h = 1.0;
        p.m = 8 + (k % 3) * 4;
        p.tol = 1e-8;
        const int id = t * 1000 + k;
        p.opt.seed = (uint64_t)id;
        int64_t ticket = 0;
        if (trm_server_submit(s, &p, &ticket) != TRM_OK) {
          ++bad;
          continue;
        }
        double lambda[16], E_G = 0.0, latency = 0.0;
        trm_stats st{};
        const trm_status rc = trm_server_wait(s, ticket, lambda, &E_G, &st,
                                              &latency);
        const trm_status want = id % 7 == 3 ? TRM_ENOCONV : TRM_OK;
        bool ok = rc == want && E_G == id && st.iterations == id &&
                  latency > 0.0;
        for (int j = 0; j < p.m; ++j) ok = ok && lambda[j] == id + j;
        if (!ok) ++bad;
      }
    });
  }
  for (auto& c : clients) c.join();
  trm_server_destroy(s);
  std::printf("bad %d max_live %d\n", bad.load(), g_max_live.load());
  return bad.load() == 0 && g_max_live.load() <= kMaxLive &&
                 g_max_live.load() >= 2
             ? 0
             : 2;
}
