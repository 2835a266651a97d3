// trm_gram_noalloc: the Gram product A^T B of trm_gram for callers that must
// not allocate device memory. Some callers cannot call cudaMalloc: they have
// handed the device's memory to their own allocator (a framework's caching
// pool, a fixed arena sized at start-up), or they run under a memory budget
// that must not grow and cannot pay the device-wide synchronisation that
// cudaMalloc/cudaFree imply in a latency-critical loop. This entry point keeps
// the split partial sums in a fixed array compiled into the library instead.
#include <cuda_runtime.h>

#include <mutex>
#include <new>
#include <string>

#include "../../include/trm.h"
#include "ops.cuh"

namespace trm {
namespace {

// 3 Mi doubles = 24 MiB of partial sums. Every GPU that loads the library
// holds this array until the process exits; the last double holds the
// tensor-core kernel's status word.
constexpr size_t kScratchDoubles = (size_t)3 << 20;
// Largest m * n accepted: 2^20 (1024 x 1024).
constexpr size_t kMaxEntries = (size_t)1 << 20;
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

int gram_noalloc(int64_t N, int m, int n, int dtype, const void* A,
                 const void* B, double* out, cudaStream_t s) {
  if ((size_t)m * (size_t)n > kMaxEntries)
    throw Error(-1, "trm_gram_noalloc: m*n = " +
                        std::to_string((long long)m * n) +
                        " exceeds the fixed scratch's limit of " +
                        std::to_string(kMaxEntries) + "; use trm_gram");
  double* scratch = scratch_address();
  const size_t cap = kScratchDoubles - 1;  // partials; then the status word
  if (dtype == TRM_F32) {
    const float* a = static_cast<const float*>(A);
    Blocks<float> b;
    b.p[0] = static_cast<const float*>(B);
    b.cols = n;
    b.count = 1;
    // the tensor-core kernel trm_gram runs for these operands; with the
    // same row slices (so the same bytes) whenever their partials fit the
    // array, else with fewer, longer slices
    if (gram_tc_eligible(N, m, a, b)) {
      int* err = reinterpret_cast<int*>(scratch + cap);
      int herr = 0;
      TRM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      gram_tc(N, m, a, b, out, scratch, cap, err, s, nullptr,
              (int)(cap / ((size_t)m * n)));
      TRM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRM_CUDA(cudaStreamSynchronize(s));
      if (herr & 2) throw Error(-6, "trm_gram_noalloc: a device wait timed out");
      return TRM_OK;
    }
    gram_in_scratch<float>(N, m, a, b, out, scratch, cap, s);
  } else {
    Blocks<double> b;
    b.p[0] = static_cast<const double*>(B);
    b.cols = n;
    b.count = 1;
    gram_in_scratch<double>(N, m, static_cast<const double*>(A), b, out,
                            scratch, cap, s);
  }
  TRM_CUDA(cudaStreamSynchronize(s));
  return TRM_OK;
}

}  // namespace
}  // namespace trm

extern "C" trm_status trm_gram_noalloc(int64_t N, int m, int n, int dtype,
                                       const void* A, const void* B,
                                       double* out, void* stream) {
  using namespace trm;
  try {
    if (N < 1 || m < 1 || n < 1 || !A || !B || !out ||
        (dtype != TRM_F32 && dtype != TRM_F64)) {
      set_global_error("invalid arguments to trm_gram_noalloc");
      return TRM_EINVAL;
    }
    return static_cast<trm_status>(gram_noalloc(
        N, m, n, dtype, A, B, out, reinterpret_cast<cudaStream_t>(stream)));
  } catch (const Error& e) {
    capture_launches(nullptr);  // (a tuner's counting scope, as in api.cu)
    set_global_error(e.what());
    return static_cast<trm_status>(e.status);
  } catch (const std::bad_alloc&) {
    capture_launches(nullptr);
    set_global_error("trm_gram_noalloc: host allocation failed");
    return TRM_ENOMEM;
  } catch (const std::exception& e) {
    capture_launches(nullptr);
    set_global_error(e.what());
    return TRM_ECUDA;
  } catch (...) {
    capture_launches(nullptr);
    set_global_error("trm_gram_noalloc: unknown error");
    return TRM_ECUDA;
  }
}
