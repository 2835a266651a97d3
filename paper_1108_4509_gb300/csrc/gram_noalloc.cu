// trm_gram_noalloc: the Gram product A^T B of trm_gram for callers that must
// not allocate device memory. Some callers cannot call cudaMalloc: they have
// handed the device's memory to their own allocator (a framework's caching
// pool, a fixed arena sized at start-up), or they run under a memory budget
// that must not grow and cannot pay the device-wide synchronisation that
// cudaMalloc/cudaFree imply in a latency-critical loop. This entry point keeps
// the split partial sums in a fixed array compiled into the library instead.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/trm.h"
#include "ops.cuh"

namespace trm {
namespace {

// 1 Mi doubles = 8 MiB of partial sums. Every GPU that loads the library holds
// this array until the process exits.
constexpr size_t kScratchDoubles = (size_t)1 << 20;
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// In host code g_gram_scratch names a host-side stand-in, not device memory:
// the device address is looked up once per device, with that device current.
double* scratch_address() {
  int dev = 0;
  TRM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    throw Error(-1, "device ordinal out of range for the fixed scratch");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    TRM_CUDA(cudaGetSymbolAddress(&p, g_gram_scratch));
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

}  // namespace
}  // namespace trm

extern "C" trm_status trm_gram_noalloc(int64_t N, int m, int n, int dtype,
                                       const void* A, const void* B,
                                       double* out, void* stream) {
  using namespace trm;
  if (N < 1 || m < 1 || n < 1 || !A || !B || !out ||
      (dtype != TRM_F32 && dtype != TRM_F64)) {
    set_global_error("invalid arguments to trm_gram_noalloc");
    return TRM_EINVAL;
  }
  if ((size_t)m * (size_t)n > kScratchDoubles) {
    set_global_error("trm_gram_noalloc: m*n = " +
                     std::to_string((long long)m * n) + " exceeds the fixed " +
                     "scratch of " + std::to_string(kScratchDoubles) +
                     " doubles; use trm_gram");
    return TRM_EINVAL;
  }
  try {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* scratch = scratch_address();
    if (dtype == TRM_F32) {
      Blocks<float> b;
      b.p[0] = static_cast<const float*>(B);
      b.cols = n;
      b.count = 1;
      gram_in_scratch<float>(N, m, static_cast<const float*>(A), b, out,
                             scratch, kScratchDoubles, s);
    } else {
      Blocks<double> b;
      b.p[0] = static_cast<const double*>(B);
      b.cols = n;
      b.count = 1;
      gram_in_scratch<double>(N, m, static_cast<const double*>(A), b, out,
                              scratch, kScratchDoubles, s);
    }
    TRM_CUDA(cudaStreamSynchronize(s));
  } catch (const Error& e) {
    set_global_error(e.what());
    return static_cast<trm_status>(e.status);
  }
  return TRM_OK;
}
