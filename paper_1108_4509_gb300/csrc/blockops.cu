// Row-local and tall-skinny (N x m times m x m) block kernels of the step:
// Fig. EGFIG Algorithm-2 steps (2), (3), (5), (7); the Polak-Ribiere sums and
// the direction update of Fig. TMFIG; the rotation C (+ alpha P) L^{-T} of
// Fig. ONFIG step (4), including the split form C L_D + C L' of Sec. 2.2
// (MP1 (ii)); column residual norms; the random initial block.
#include "dfmath.cuh"
#include "ops.cuh"

namespace trm {

namespace {

constexpr int RCHUNK = 4096;  // rows per partial in column reductions

// ---------------------------------------------------------------------------
// Column dot products: part[chunk*m + j] = sum_{i in chunk} A_ij B_ij
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
    k_coldot(int64_t N, int m, const T* __restrict__ A,
             const T* __restrict__ B, double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.y;
  const int64_t rb = (int64_t)blockIdx.x * RCHUNK;
  const int64_t re = min(N, rb + RCHUNK);
  const T* a = A + (int64_t)j * N;
  const T* b = B + (int64_t)j * N;
  T s = 0;
  for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) s += a[i] * b[i];
  double v[1] = {(double)s};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * m + j] = v[0];
}

// out[j] = sum_chunks part[chunk*m + j]; optional total into *tot (one CTA)
// out[j] = sum_c part[c m + j] (then sqrt when do_sqrt), *tot = sum_j out[j];
// one CTA of 1024 threads, m <= 1024: warp w takes the 32 columns of group
// w % G (G = ceil(m / 32); loads coalesced across columns) and the chunks
// c = w / G (mod 32 / G); the slices are added in a fixed order.
__global__ void __launch_bounds__(1024)
    k_colsum(const double* __restrict__ part, int chunks, int m,
             double* __restrict__ out, double* tot, int do_sqrt) {
  __shared__ double sl_sum[1024];  // [slice][column], S m <= 1024
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = (m + 31) >> 5, S = 32 / G;
  const int cg = warp % G, sl = warp / G;
  const int j = 32 * cg + lane;
  if (sl < S && j < m) {
    double s0 = 0.0, s1 = 0.0;
    int c = sl;
    for (; c + S < chunks; c += 2 * S) {
      s0 += part[(size_t)c * m + j];
      s1 += part[(size_t)(c + S) * m + j];
    }
    if (c < chunks) s0 += part[(size_t)c * m + j];
    sl_sum[sl * m + j] = s0 + s1;
  }
  __syncthreads();
  double t = 0.0;
  for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
    double s = sl_sum[jj];
    for (int q = 1; q < S; ++q) s += sl_sum[q * m + jj];
    if (do_sqrt) s = sqrt(s);
    out[jj] = s;
    t += s;
  }
  double v[1] = {t};
  block_sum<1>(v, red);
  if (threadIdx.x == 0 && tot) *tot = v[0];
}

// ---------------------------------------------------------------------------
// X' = X - C diag(H_D) (Alg-2 step (5)), optionally emitting FP32 copies.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_xprime(int64_t N, const T* __restrict__ C, T* __restrict__ X,
                         const double* __restrict__ HD, float* C32,
                         float* Xp32, int write_x) {
  const int j = blockIdx.y;
  const T h = (T)HD[j];
  const int64_t off = (int64_t)j * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T c = C[off + i];
    const T x = X[off + i] - c * h;
    if (write_x) X[off + i] = x;
    if (C32) C32[off + i] = (float)c;
    if (Xp32) Xp32[off + i] = (float)x;
  }
}

// ---------------------------------------------------------------------------
// Tiled N x k times k x n products (64 x 64 output tile, 32-deep stages).
// Thread (tx, ty): rows r0 + 4 tx .. +3 (one vector per column), columns
// c0 + 4 ty .. +3.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 32, GLD = 68;

// 4 consecutive shared-memory elements at a 16-byte aligned address
__device__ __forceinline__ void ldv4(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ldv4(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// acc += A[r0:r0+64, kb:ke] M[kb:ke, c0:c0+64], A via loadA(row, k) and M via
// loadM(k, col) (both return T; out-of-range reads must return 0).
template <typename T, class LA, class LM>
__device__ __forceinline__ void tile_product(int kb, int ke, LA loadA,
                                             LM loadM, T (&acc)[4][4],
                                             T (*As)[GLD], T (*Ms)[GLD]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      const int r = e & (GT - 1), kk = e >> 6;  // A: rows fastest
      As[kk][r] = (k0 + kk < ke) ? loadA(r, k0 + kk) : (T)0;
      const int c = e & (GT - 1), k2 = e >> 6;  // M: columns fastest
      Ms[k2][c] = (k0 + k2 < ke) ? loadM(k0 + k2, c) : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      T a[4], b[4];
      ldv4(&As[kk][tx * 4], a);
      ldv4(&Ms[kk][ty * 4], b);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
}

// The same tile product for FP64 inputs in double-float (the FP32 pipe):
// each staged value is split into FP32 (hi, lo) terms; the accumulators
// are pair sums (DfAcc), renormalised after every stage.
template <typename LA, typename LM>
__device__ __forceinline__ void tile_product_df(
    int kb, int ke, LA loadA, LM loadM, DfAcc (&acc)[4][4], float (*Ah)[GLD],
    float (*Al)[GLD], float (*Mh)[GLD], float (*Ml)[GLD]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      const int r = e & (GT - 1), kk = e >> 6;  // A: rows fastest
      const F2 a = df_of((k0 + kk < ke) ? loadA(r, k0 + kk) : 0.0);
      Ah[kk][r] = a.h;
      Al[kk][r] = a.l;
      const int c = e & (GT - 1), k2 = e >> 6;  // M: columns fastest
      const F2 b = df_of((k0 + k2 < ke) ? loadM(k0 + k2, c) : 0.0);
      Mh[k2][c] = b.h;
      Ml[k2][c] = b.l;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
      ldv4(&Ah[kk][tx * 4], ah);
      ldv4(&Al[kk][tx * 4], al);
      ldv4(&Mh[kk][ty * 4], bh);
      ldv4(&Ml[kk][ty * 4], bl);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y].fma(ah[x], al[x], bh[y], bl[y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y].norm();
    __syncthreads();
  }
}

// Y = A M (N x k times k x n, FP64 blocks) in double-float; with tri the
// product is C R for R upper triangular (only k <= column contributes).
__global__ void __launch_bounds__(256)
    k_mult_df(int64_t N, int k, int n, const double* __restrict__ A,
              const double* __restrict__ M, double* __restrict__ Y,
              int tri) {
  __shared__ __align__(16) float Ah[GK][GLD], Al[GK][GLD];
  __shared__ __align__(16) float Mh[GK][GLD], Ml[GK][GLD];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  DfAcc acc[4][4];
  auto loadA = [&](int r, int kk) -> double {
    const int64_t row = r0 + r;
    return row < N ? A[row + (int64_t)kk * N] : 0.0;
  };
  auto loadM = [&](int kk, int c) -> double {
    return (c0 + c < n) ? M[kk + (int64_t)(c0 + c) * k] : 0.0;
  };
  const int kend = tri ? min(k, c0 + GT) : k;
  tile_product_df(0, kend, loadA, loadM, acc, Ah, Al, Mh, Ml);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col < n)
        Y[row + (int64_t)col * N] = (double)acc[x][y].h + (double)acc[x][y].l;
    }
  }
}

// G = -2 (X' - C H'), with per-CTA partial sums of
// tr(G^T G), tr(G^T M G), tr(G_prev^T M G), tr(G^T P_prev).
template <typename T>
__global__ void __launch_bounds__(256)
    k_gradient(int64_t N, int m, const T* __restrict__ C,
               const T* __restrict__ Xp, const double* __restrict__ Hp,
               T* __restrict__ G, const T* __restrict__ Gprev,
               const T* __restrict__ Pprev, const T* __restrict__ minv,
               double* __restrict__ part) {
  __shared__ __align__(16) T As[GK][GLD];
  __shared__ __align__(16) T Ms[GK][GLD];
  __shared__ double red[4 * 32];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  T acc[4][4] = {};
  auto loadA = [&](int r, int k) -> T {
    const int64_t row = r0 + r;
    return row < N ? C[row + (int64_t)k * N] : (T)0;
  };
  auto loadM = [&](int k, int c) -> T {
    return (c0 + c < m) ? (T)Hp[k + (int64_t)(c0 + c) * m] : (T)0;
  };
  tile_product<T>(0, m, loadA, loadM, acc, As, Ms);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T s_gg = 0, s_gmg = 0, s_pmg = 0, s_gpp = 0;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
    const T mi = minv ? minv[row] : (T)1;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col >= m) continue;
      const int64_t idx = row + (int64_t)col * N;
      const T g = (T)-2 * (Xp[idx] - acc[x][y]);
      G[idx] = g;
      const T mg = mi * g;
      s_gg += g * g;
      s_gmg += g * mg;
      if (Gprev) s_pmg += Gprev[idx] * mg;
      if (Pprev) s_gpp += g * Pprev[idx];
    }
  }
  double v[4] = {(double)s_gg, (double)s_gmg, (double)s_pmg, (double)s_gpp};
  block_sum<4>(v, red);
  if (threadIdx.x == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) part[b * 4 + q] = v[q];
  }
}

// Sum the gradient partials and update the CG scalars (one CTA).
__global__ void k_cg_scalars(const double* __restrict__ part, int nparts,
                             int m, IterScalars* sc) {
  __shared__ double red[4 * 32];
  double v[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] += part[(size_t)p * 4 + q];
  block_sum<4>(v, red);
  if (threadIdx.x == 0) cg_scalars(v, m, sc);
}

// FP32 blocks with N % 4 == 0: the same updates on 16-byte vectors.
__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z),
                     fmaf(a, x.w, y.w));
}
__global__ void k_update_p4(int64_t N, const float4* __restrict__ G,
                            float4* __restrict__ P,
                            const float4* __restrict__ minv,
                            const IterScalars* __restrict__ sc) {
  const int j = blockIdx.y;
  const float gamma = (float)sc->gamma;
  const int64_t n4 = N >> 2, off = (int64_t)j * n4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 mg = G[off + i];
    if (minv) {
      const float4 w = minv[i];
      mg = make_float4(w.x * mg.x, w.y * mg.y, w.z * mg.z, w.w * mg.w);
    }
    P[off + i] = gamma == 0.f ? mg : f4_fma(gamma, P[off + i], mg);
  }
}

// X' = X - C diag(H_D), FP32, vectors of four (the FP32 copies are not
// needed on this path)
__global__ void k_xprime4(int64_t N, const float4* __restrict__ C,
                          float4* __restrict__ X,
                          const double* __restrict__ HD) {
  const int j = blockIdx.y;
  const float h = (float)HD[j];
  const int64_t n4 = N >> 2, off = (int64_t)j * n4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x)
    X[off + i] = f4_fma(-h, C[off + i], X[off + i]);
}

// P = M G + gamma P
template <typename T>
__global__ void k_update_p(int64_t N, const T* __restrict__ G, T* __restrict__ P,
                           const T* __restrict__ minv,
                           const IterScalars* __restrict__ sc) {
  const int j = blockIdx.y;
  const T gamma = (T)sc->gamma;
  const int64_t off = (int64_t)j * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T mg = (minv ? minv[i] : (T)1) * G[off + i];
    P[off + i] = gamma == (T)0 ? mg : mg + gamma * P[off + i];
  }
}

// Cn = (C + alpha P) R, R upper triangular (only k <= col contributes).
template <typename T, typename TP>
__global__ void __launch_bounds__(256)
    k_rotate(int64_t N, int m, const T* __restrict__ C,
             const TP* __restrict__ P, const double* __restrict__ R,
             T* __restrict__ Cn, const IterScalars* __restrict__ sc) {
  __shared__ __align__(16) T As[GK][GLD];
  __shared__ __align__(16) T Ms[GK][GLD];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  const T alpha = (P && sc) ? (T)sc->alpha : (T)0;
  T acc[4][4] = {};
  auto loadA = [&](int r, int k) -> T {
    const int64_t row = r0 + r;
    if (row >= N) return (T)0;
    const int64_t idx = row + (int64_t)k * N;
    T y = C[idx];
    if (P) y += alpha * (T)P[idx];
    return y;
  };
  auto loadM = [&](int k, int c) -> T {
    return (c0 + c < m) ? (T)R[k + (int64_t)(c0 + c) * m] : (T)0;
  };
  const int kend = min(m, c0 + GT);
  tile_product<T>(0, kend, loadA, loadM, acc, As, Ms);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col < m) Cn[row + (int64_t)col * N] = acc[x][y];
    }
  }
}

// MP1 (ii): Cn = Y L_D + fl32(Y) L', Y = C + alpha P; L_D = diag(R) in FP64,
// L' = R - L_D in FP32.
__global__ void __launch_bounds__(256)
    k_rotate_split(int64_t N, int m, const double* __restrict__ C,
                   const float* __restrict__ P, const double* __restrict__ R,
                   double* __restrict__ Cn, const IterScalars* __restrict__ sc) {
  __shared__ __align__(16) float As[GK][GLD];
  __shared__ __align__(16) float Ms[GK][GLD];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  const double alpha = sc->alpha;
  float acc[4][4] = {};
  auto loadA = [&](int r, int k) -> float {
    const int64_t row = r0 + r;
    if (row >= N) return 0.f;
    const int64_t idx = row + (int64_t)k * N;
    return (float)(C[idx] + alpha * (double)P[idx]);
  };
  auto loadM = [&](int k, int c) -> float {
    const int col = c0 + c;
    return (col < m && k != col) ? (float)R[k + (int64_t)col * m] : 0.f;
  };
  const int kend = min(m, c0 + GT);
  tile_product<float>(0, kend, loadA, loadM, acc, As, Ms);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col >= m) continue;
      const int64_t idx = row + (int64_t)col * N;
      const double yv = C[idx] + alpha * (double)P[idx];
      Cn[idx] = yv * R[col + (int64_t)col * m] + (double)acc[x][y];
    }
  }
}

// The same split update with C and Cn as FP32 pairs: the FP32 operand is
// Ch + alpha P, and Y diag(R) is formed in double-float.
__global__ void __launch_bounds__(256)
    k_rotate_split_df(int64_t N, int m, const float* __restrict__ Ch,
                      const float* __restrict__ Cl,
                      const float* __restrict__ P, const double* __restrict__ R,
                      float* __restrict__ Cnh, float* __restrict__ Cnl,
                      const IterScalars* __restrict__ sc) {
  __shared__ __align__(16) float As[GK][GLD];
  __shared__ __align__(16) float Ms[GK][GLD];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  const float alpha = (float)sc->alpha;
  const F2 alpha2 = df_of(sc->alpha);
  float acc[4][4] = {};
  auto loadA = [&](int r, int k) -> float {
    const int64_t row = r0 + r;
    if (row >= N) return 0.f;
    const int64_t idx = row + (int64_t)k * N;
    return fmaf(alpha, P[idx], Ch[idx]);
  };
  auto loadM = [&](int k, int c) -> float {
    const int col = c0 + c;
    return (col < m && k != col) ? (float)R[k + (int64_t)col * m] : 0.f;
  };
  const int kend = min(m, c0 + GT);
  tile_product<float>(0, kend, loadA, loadM, acc, As, Ms);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col >= m) continue;
      const int64_t idx = row + (int64_t)col * N;
      const F2 yv = df_add(F2{Ch[idx], Cl[idx]}, df_mul(alpha2, F2{P[idx], 0.f}));
      const F2 t = df_add(df_mul(yv, df_of(R[col + (int64_t)col * m])),
                          F2{acc[x][y], 0.f});
      Cnh[idx] = t.h;
      Cnl[idx] = t.l;
    }
  }
}

// Y = A M, A: N x k FP64, M: k x n FP64
__global__ void __launch_bounds__(256)
    k_mult(int64_t N, int k, int n, const double* __restrict__ A,
           const double* __restrict__ M, double* __restrict__ Y) {
  __shared__ __align__(16) double As[GK][GLD];
  __shared__ __align__(16) double Ms[GK][GLD];
  const int64_t r0 = (int64_t)blockIdx.x * GT;
  const int c0 = blockIdx.y * GT;
  double acc[4][4] = {};
  auto loadA = [&](int r, int kk) -> double {
    const int64_t row = r0 + r;
    return row < N ? A[row + (int64_t)kk * N] : 0.0;
  };
  auto loadM = [&](int kk, int c) -> double {
    return (c0 + c < n) ? M[kk + (int64_t)(c0 + c) * k] : 0.0;
  };
  tile_product<double>(0, k, loadA, loadM, acc, As, Ms);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = r0 + tx * 4 + x;
    if (row >= N) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = c0 + ty * 4 + y;
      if (col < n) Y[row + (int64_t)col * N] = acc[x][y];
    }
  }
}

// part[chunk*m + j] = sum_i (X_ij - lam_j C_ij)^2
__global__ void __launch_bounds__(256)
    k_resid(int64_t N, int m, const double* __restrict__ X,
            const double* __restrict__ C, const double* __restrict__ lam,
            double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.y;
  const int64_t rb = (int64_t)blockIdx.x * RCHUNK;
  const int64_t re = min(N, rb + RCHUNK);
  const double l = lam[j];
  double s = 0.0;
  for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) {
    const double d = X[(int64_t)j * N + i] - l * C[(int64_t)j * N + i];
    s += d * d;
  }
  double v[1] = {s};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * m + j] = v[0];
}

// Largest |C_ij| per (chunk, column), ties to the smaller row.
__global__ void __launch_bounds__(256)
    k_colmax(int64_t N, int m, const double* __restrict__ C,
             double* __restrict__ val, int64_t* __restrict__ idx) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int j = blockIdx.y;
  const int64_t rb = (int64_t)blockIdx.x * RCHUNK;
  const int64_t re = min(N, rb + RCHUNK);
  double bv = -1.0;
  int64_t bi = 0;
  for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) {
    const double a = fabs(C[(int64_t)j * N + i]);
    if (a > bv) { bv = a; bi = i; }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double ov = sv[threadIdx.x + o];
      const int64_t oi = si[threadIdx.x + o];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    val[(size_t)blockIdx.x * m + j] = sv[0];
    idx[(size_t)blockIdx.x * m + j] = si[0];
  }
}

__global__ void k_sign_of_max(int64_t N, int m, int chunks,
                              const double* __restrict__ val,
                              const int64_t* __restrict__ idx,
                              const double* __restrict__ C,
                              double* __restrict__ sgn) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double bv = -1.0;
  int64_t bi = 0;
  for (int c = 0; c < chunks; ++c) {
    const double v = val[(size_t)c * m + j];
    if (v > bv) { bv = v; bi = idx[(size_t)c * m + j]; }
  }
  sgn[j] = C[(int64_t)j * N + bi] < 0.0 ? -1.0 : 1.0;
}

__global__ void k_scale_cols(int64_t N, double* __restrict__ C,
                             double* __restrict__ X,
                             const double* __restrict__ sgn) {
  const int j = blockIdx.y;
  const double s = sgn[j];
  if (s == 1.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    C[(int64_t)j * N + i] *= s;
    if (X) X[(int64_t)j * N + i] *= s;
  }
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y,
                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_to_f64(const float* __restrict__ x, double* __restrict__ y,
                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// SplitMix64 (Steele, Lea and Flood 2014): mix(x + golden gamma).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_random(int64_t total, uint64_t seed, double* __restrict__ C) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = splitmix64(seed ^ splitmix64((uint64_t)i));
    C[i] = (double)(u >> 11) * 0x1.0p-53 - 0.5;
  }
}

int elem_grid_x(int64_t N) {
  int g = ceil_div(N, 256 * 4);
  return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void energy_diag(int64_t N, int m, const T* C, const T* X, double* HD,
                 IterScalars* sc, double* partials, cudaStream_t s) {
  const int chunks = ceil_div(N, RCHUNK);
  k_coldot<T><<<dim3(chunks, m), 256, 0, s>>>(N, m, C, X, partials);
  TRM_CHECK_LAUNCH();
  k_colsum<<<1, 1024, 0, s>>>(partials, chunks, m, HD, sc ? &sc->E : nullptr,
                              0);
  TRM_CHECK_LAUNCH();
}

void energy_from_dots(const double* dots, int chunks, int m, double* HD,
                      IterScalars* sc, cudaStream_t s) {
  k_colsum<<<1, 1024, 0, s>>>(dots, chunks, m, HD, sc ? &sc->E : nullptr, 0);
  TRM_CHECK_LAUNCH();
}

template <typename T>
void xprime(int64_t N, int m, const T* C, T* X, const double* HD, float* C32,
            float* Xp32, cudaStream_t s, bool write_x) {
  if constexpr (sizeof(T) == 4) {
    if (!C32 && !Xp32 && write_x && N % 4 == 0 &&
        ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(X)) &
         15) == 0) {
      k_xprime4<<<dim3(elem_grid_x(N), m), 256, 0, s>>>(
          N, reinterpret_cast<const float4*>(C), reinterpret_cast<float4*>(X),
          HD);
      TRM_CHECK_LAUNCH();
      return;
    }
  }
  k_xprime<T><<<dim3(elem_grid_x(N), m), 256, 0, s>>>(N, C, X, HD, C32, Xp32,
                                                      write_x ? 1 : 0);
  TRM_CHECK_LAUNCH();
}

static bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

template <typename T>
void gradient(int64_t N, int m, const T* C, const T* Xp, const double* Hp,
              T* G, const T* Gprev, const T* Pprev, const T* minv,
              IterScalars* sc, double* partials, size_t cap, cudaStream_t s,
              const TcWork* tw) {
  if constexpr (sizeof(T) == 4) {
    // TMA reads C and the epilogue operands X', G_prev, P_prev
    if (mul_tc_eligible(N, m, m, tw) && aligned16(C) && aligned16(Xp) &&
        aligned16(Gprev) && aligned16(Pprev)) {
      if ((size_t)mul_tc_parts(N, m) * 4 > cap)
        throw Error(-2, "gradient: partials buffer too small");
      // the kernel's last CTA forms the CG scalars from the per-CTA sums
      mul_tc_grad(N, m, C, Hp, Xp, G, Gprev, Pprev, minv, partials, sc, *tw,
                  s);
      return;
    }
  }
  dim3 grid(ceil_div(N, GT), ceil_div(m, GT));
  const size_t nparts = (size_t)grid.x * grid.y;
  if (nparts * 4 > cap) throw Error(-2, "gradient: partials buffer too small");
  k_gradient<T><<<grid, 256, 0, s>>>(N, m, C, Xp, Hp, G, Gprev, Pprev, minv,
                                     partials);
  TRM_CHECK_LAUNCH();
  k_cg_scalars<<<1, 1024, 0, s>>>(partials, (int)nparts, m, sc);
  TRM_CHECK_LAUNCH();
}

template <typename T>
void update_p(int64_t N, int m, const T* G, T* P, const T* minv,
              const IterScalars* sc, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (N % 4 == 0 &&
        ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(P) |
          reinterpret_cast<uintptr_t>(minv)) & 15) == 0) {
      k_update_p4<<<dim3(elem_grid_x(N), m), 256, 0, s>>>(
          N, reinterpret_cast<const float4*>(G), reinterpret_cast<float4*>(P),
          reinterpret_cast<const float4*>(minv), sc);
      TRM_CHECK_LAUNCH();
      return;
    }
  }
  k_update_p<T><<<dim3(elem_grid_x(N), m), 256, 0, s>>>(N, G, P, minv, sc);
  TRM_CHECK_LAUNCH();
}

template <typename T, typename TP>
void rotate(int64_t N, int m, const T* C, const TP* P, const double* R, T* Cn,
            const IterScalars* sc, cudaStream_t s, const TcWork* tw) {
  if constexpr (sizeof(T) == 4 && sizeof(TP) == 4) {
    if (mul_tc_eligible(N, m, m, tw) && aligned16(C) &&
        (P == nullptr || (sc && aligned16(P)))) {
      mul_tc_store(N, m, m, C, P, sc, R, Cn, *tw, s);
      return;
    }
  }
  dim3 grid(ceil_div(N, GT), ceil_div(m, GT));
  k_rotate<T, TP><<<grid, 256, 0, s>>>(N, m, C, P, R, Cn, sc);
  TRM_CHECK_LAUNCH();
}

void rotate_split(int64_t N, int m, const double* C, const float* P,
                  const double* R, double* Cn, const IterScalars* sc,
                  cudaStream_t s, const float* C32, const TcWork* tw) {
  if (C32 && mul_tc_eligible(N, m, m, tw) && aligned16(C32) && aligned16(P)) {
    mul_tc_split64(N, m, C32, P, C, sc, R, Cn, *tw, s);
    return;
  }
  dim3 grid(ceil_div(N, GT), ceil_div(m, GT));
  k_rotate_split<<<grid, 256, 0, s>>>(N, m, C, P, R, Cn, sc);
  TRM_CHECK_LAUNCH();
}

void rotate_split_df(int64_t N, int m, const float* Ch, const float* Cl,
                     const float* P, const double* R, float* Cnh, float* Cnl,
                     const IterScalars* sc, cudaStream_t s, const TcWork* tw) {
  if (mul_tc_eligible(N, m, m, tw) && aligned16(Ch) && aligned16(P)) {
    mul_tc_splitdf(N, m, Ch, Cl, P, sc, R, Cnh, Cnl, *tw, s);
    return;
  }
  dim3 grid(ceil_div(N, GT), ceil_div(m, GT));
  k_rotate_split_df<<<grid, 256, 0, s>>>(N, m, Ch, Cl, P, R, Cnh, Cnl, sc);
  TRM_CHECK_LAUNCH();
}

void mult_df(int64_t N, int k, int n, const double* A, const double* M,
             double* Y, bool upper_tri, cudaStream_t s) {
  dim3 grid(ceil_div(N, GT), ceil_div(n, GT));
  k_mult_df<<<grid, 256, 0, s>>>(N, k, n, A, M, Y, upper_tri ? 1 : 0);
  TRM_CHECK_LAUNCH();
}

void mult(int64_t N, int k, int n, const double* A, const double* M, double* Y,
          cudaStream_t s) {
  dim3 grid(ceil_div(N, GT), ceil_div(n, GT));
  k_mult<<<grid, 256, 0, s>>>(N, k, n, A, M, Y);
  TRM_CHECK_LAUNCH();
}

void column_residuals(int64_t N, int m, const double* X, const double* C,
                      const double* lam, double* res, double* partials,
                      cudaStream_t s) {
  const int chunks = ceil_div(N, RCHUNK);
  k_resid<<<dim3(chunks, m), 256, 0, s>>>(N, m, X, C, lam, partials);
  TRM_CHECK_LAUNCH();
  k_colsum<<<1, 1024, 0, s>>>(partials, chunks, m, res, nullptr, 1);
  TRM_CHECK_LAUNCH();
}

void fix_signs(int64_t N, int m, double* C, double* X, double* work,
               cudaStream_t s) {
  const int chunks = ceil_div(N, RCHUNK);
  double* val = work;
  int64_t* idx = reinterpret_cast<int64_t*>(work + (size_t)chunks * m);
  double* sgn = work + (size_t)2 * chunks * m;
  k_colmax<<<dim3(chunks, m), 256, 0, s>>>(N, m, C, val, idx);
  TRM_CHECK_LAUNCH();
  k_sign_of_max<<<ceil_div(m, 128), 128, 0, s>>>(N, m, chunks, val, idx, C,
                                                 sgn);
  TRM_CHECK_LAUNCH();
  k_scale_cols<<<dim3(elem_grid_x(N), m), 256, 0, s>>>(N, C, X, sgn);
  TRM_CHECK_LAUNCH();
}

void to_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  k_to_f32<<<elem_grid_x(n), 256, 0, s>>>(x, y, n);
  TRM_CHECK_LAUNCH();
}
void to_f64(const float* x, double* y, int64_t n, cudaStream_t s) {
  k_to_f64<<<elem_grid_x(n), 256, 0, s>>>(x, y, n);
  TRM_CHECK_LAUNCH();
}

void random_block(int64_t N, int m, uint64_t seed, double* C, cudaStream_t s) {
  k_random<<<elem_grid_x(N * m), 256, 0, s>>>(N * m, seed, C);
  TRM_CHECK_LAUNCH();
}

#define TRM_INST(T)                                                          \
  template void energy_diag<T>(int64_t, int, const T*, const T*, double*,    \
                               IterScalars*, double*, cudaStream_t);         \
  template void xprime<T>(int64_t, int, const T*, T*, const double*, float*, \
                          float*, cudaStream_t, bool);                       \
  template void gradient<T>(int64_t, int, const T*, const T*, const double*, \
                            T*, const T*, const T*, const T*, IterScalars*,  \
                            double*, size_t, cudaStream_t, const TcWork*);   \
  template void update_p<T>(int64_t, int, const T*, T*, const T*,            \
                            const IterScalars*, cudaStream_t);
TRM_INST(float)
TRM_INST(double)
#undef TRM_INST
template void rotate<float, float>(int64_t, int, const float*, const float*,
                                   const double*, float*, const IterScalars*,
                                   cudaStream_t, const TcWork*);
template void rotate<double, double>(int64_t, int, const double*,
                                     const double*, const double*, double*,
                                     const IterScalars*, cudaStream_t,
                                     const TcWork*);

}  // namespace trm
