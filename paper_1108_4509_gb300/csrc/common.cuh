// Shared device/host helpers of the trace-minimization library (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

namespace trm {

// Library error carried to the C ABI boundary, where it becomes a status.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& msg) : std::runtime_error(msg), status(s) {}
};

#define TRM_CUDA(expr)                                                        \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess)                                                    \
      throw ::trm::Error(-5, std::string(#expr) + ": " +                      \
                                 cudaGetErrorString(e_) + " (" + __FILE__ +   \
                                 ":" + std::to_string(__LINE__) + ")");       \
  } while (0)

// Every kernel launch of the library is followed by this check, which also
// counts the launch (process-wide, all devices).
void count_launch();
#define TRM_CHECK_LAUNCH()           \
  do {                               \
    TRM_CUDA(cudaGetLastError());    \
    ::trm::count_launch();           \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per process).
int sm_count();
// Kernel launches issued by the library so far in this process.
long long launch_count();
long long thread_launch_count();  // launches by the calling host thread
void count_launches(long long n);  // n kernels launched at once (a graph)
// While sink is set, launches of the calling thread are counted into *sink
// (kernels captured into a graph) instead of as launches.
void capture_launches(long long* sink);
// Message returned by trm_last_global_error() on this host thread.
void set_global_error(const std::string& msg);

// ---------------------------------------------------------------------------
// Deterministic reductions: warp xor-shuffle trees and fixed block trees.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 -> FP64 on the integer pipe. The conversion instruction runs on the
// FP64 pipe, where one warp instruction holds a sub-partition for about 64
// cycles on this part; in the FP32 stencil a few conversions per warp kept
// that pipe half busy. The sign, the exponent rebiased from 127 to 1023,
// the 23 fraction bits moved to the top of the 52: exact for normal numbers,
// zeros, infinities and NaN; FP32 subnormals (below 1.2e-38) become signed
// zeros.
__device__ __forceinline__ double to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ex =
      e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(
      sign | (ex << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

// Sum of NQ values over the block (blockDim.x a multiple of 32, <= 1024).
// Result valid in thread 0. scratch: >= 32*NQ doubles of shared memory.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) scratch[q * 32 + warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nwarp ? scratch[q * 32 + lane] : 0.0;
      v[q] = warp_sum(x);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Scalars of one iteration, resident in device memory.
// ---------------------------------------------------------------------------
struct IterScalars {
  double E;        // energy trace(C^T H C) = sum_j H_D,j
  double gg;       // tr(G^T G)
  double gMg;      // tr(G^T M G)
  double gpMg;     // tr(G_prev^T M G)
  double gPp;      // tr(G^T P_prev)
  double a_prev;   // tr(G_prev^T M G_prev)
  double gamma;    // Polak-Ribiere coefficient used for P
  double slope0;   // E'(0) = -tr(G^T P)
  double alpha;    // step taken
  double alpha_prev;
  double rms;      // ||G||_F / (2 sqrt(m))
  double c2;       // curvature of the quadratic line model
  double dE;       // predicted energy change of the step
  int restart;     // 1: next P uses gamma = 0
  int status;      // bit flags: 1 = overlap not positive definite
  int iter;
  unsigned grad_done;  // CTAs of the tensor-core gradient that have finished
};

// The Polak-Ribiere scalars from the four gradient sums
// v = {tr(G^T G), tr(G^T M G), tr(G_prev^T M G), tr(G^T P_prev)}: gamma =
// tr((G - G_prev)^T M G) / tr(G_prev^T M G_prev), or 0 on a restart (the
// previous blocks are not read then) or where P would not be a descent
// direction; the RMS residual ||G||_F / (2 sqrt(m)).
__device__ __forceinline__ void cg_scalars(const double (&v)[4], int m,
                                           IterScalars* sc) {
  const double gg = v[0], gMg = v[1], gpMg = v[2], gPp = v[3];
  sc->gg = gg;
  sc->gMg = gMg;
  sc->gpMg = gpMg;
  sc->gPp = gPp;
  sc->rms = sqrt(gg) / (2.0 * sqrt((double)m));
  double gamma = 0.0;
  if (!sc->restart && sc->a_prev > 0.0) {
    gamma = (gMg - gpMg) / sc->a_prev;
    if (!(gMg + gamma * gPp > 0.0)) gamma = 0.0;  // keep a descent direction
  }
  sc->gamma = gamma;
  sc->slope0 = gamma != 0.0 ? -(gMg + gamma * gPp) : -gMg;
  sc->a_prev = gMg;
  sc->restart = 0;
}

}  // namespace trm
