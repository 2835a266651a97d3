// Device steps of the initial-guess extrapolation (trm_extrapolate): the
// orthogonal factor of a polar decomposition, which aligns one block's basis
// to another's (orthogonal Procrustes), and a linear combination of blocks.
#include "ops.cuh"

namespace trm {

namespace {

// T = Z diag(w)^{-1/2} for the polar factor M (M^T M)^{-1/2}, w ascending
// (the eigenvalues of M^T M); an eigenvalue at or below 1e-12 of the largest
// (M singular to working accuracy: no unique alignment) sets status bit 1.
__global__ void __launch_bounds__(256)
    k_polar_scale(int m, const double* __restrict__ w,
                  const double* __restrict__ Z, double* __restrict__ T,
                  int* status) {
  const double wmax = w[m - 1];
  if (blockIdx.x == 0 && threadIdx.x == 0 && !(w[0] > 1e-12 * wmax))
    atomicOr(status, 1);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       e < (int64_t)m * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / m);
    const double wj = w[j] > 1e-12 * wmax ? w[j] : 1e-12 * wmax;
    T[e] = Z[e] / sqrt(wj);
  }
}

__global__ void k_lin_comb(int64_t n, double a, const double* X, double b,
                           const double* Y, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * X[i] + b * Y[i];
}

}  // namespace

size_t polar_work_doubles(int m) {
  return sym_eig_work_doubles(m) + (size_t)4 * m * m + m;
}

void polar_factor(int m, const double* M, double* U, double* work, int* status,
                  int* info, cudaStream_t s) {
  const size_t mm = (size_t)m * m;
  double* A = work;
  double* Z = A + mm;
  double* T = Z + mm;
  double* T2 = T + mm;
  double* w = T2 + mm;
  double* ew = w + m;
  mm_gemm(m, M, true, M, false, A, 1.0, 0.0, s);     // A = M^T M
  sym_eig(m, A, w, Z, ew, info, s);                   // A = Z diag(w) Z^T
  const int64_t blocks = ceil_div((int64_t)mm, 256);
  k_polar_scale<<<blocks < 64 ? (int)blocks : 64, 256, 0, s>>>(m, w, Z, T,
                                                               status);
  TRM_CHECK_LAUNCH();
  mm_gemm(m, T, false, Z, true, T2, 1.0, 0.0, s);    // (M^T M)^{-1/2}
  mm_gemm(m, M, false, T2, false, U, 1.0, 0.0, s);   // U = M (M^T M)^{-1/2}
}

void lin_comb(int64_t n, double a, const double* X, double b, const double* Y,
              double* out, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ceil_div(n, 1024);
  if (blocks > 4096) blocks = 4096;
  k_lin_comb<<<(int)blocks, 256, 0, s>>>(n, a, X, b, Y, out);
  TRM_CHECK_LAUNCH();
}

}  // namespace trm
