// Device steps specific to the generalized problem H e = lambda S e: the
// diagonal preconditioner of the pencil (H, S).
#include "ops.cuh"

namespace trm {

namespace {

constexpr int kMinBlocks = 256;

// Block-wise minima of H_ii / S_ii.
__global__ void __launch_bounds__(256)
    k_min_ratio(const double* __restrict__ dH, const double* __restrict__ dS,
                int64_t N, double* out) {
  __shared__ double sm[256];
  double v = INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    v = fmin(v, dH[i] / dS[i]);
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

__global__ void k_precond_gen(const double* __restrict__ dH,
                              const double* __restrict__ dS, int64_t N,
                              const double* __restrict__ mins, int nmins,
                              double* minv64, float* minv32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double lo = INFINITY;
  for (int k = 0; k < nmins; ++k) lo = fmin(lo, mins[k]);
  const double sigma = lo - 1.0;
  const double mi = 1.0 / (dH[i] - sigma * dS[i]);
  minv64[i] = mi;
  minv32[i] = (float)mi;
}

}  // namespace

void diag_preconditioner_gen(const double* diagH, const double* diagS,
                             int64_t N, double* minv64, float* minv32,
                             double* work, cudaStream_t s) {
  k_min_ratio<<<kMinBlocks, 256, 0, s>>>(diagH, diagS, N, work);
  TRM_CHECK_LAUNCH();
  k_precond_gen<<<ceil_div(N, 256), 256, 0, s>>>(diagH, diagS, N, work,
                                                 kMinBlocks, minv64, minv32);
  TRM_CHECK_LAUNCH();
}

}  // namespace trm
