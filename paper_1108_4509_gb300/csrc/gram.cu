// Tall-skinny Gram products out = A^T [B_0 | B_1 | ...] with K = N rows
// (Fig. EGFIG step (6) H' = C^T X'; Fig. ONFIG step (1) S = C^T C; the
// line-search projections C^T P, P^T P, P^T H P, P^T G).
//
// Split-K over the N rows: CTA (s, t) multiplies rows [s*R, (s+1)*R) of its
// 64 x 64 output tile t, summing in the input precision, and writes the tile
// as FP64 partials; a second kernel adds the partials of all splits in a fixed
// order, so the result is bitwise reproducible.
#include "dfmath.cuh"
#include "ops.cuh"

namespace trm {

namespace {

constexpr int TM = 64;   // output tile rows (columns of A)
constexpr int TN = 64;   // output tile columns (columns of B)
constexpr int TK = 32;   // rows of A/B per shared-memory stage
constexpr int LDS = 68;  // padded shared row length (16-byte aligned)

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) {
    float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void ld(const double* p, double (&v)[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

template <typename T>
__global__ void __launch_bounds__(256)
    k_gram(int64_t N, int m, const T* __restrict__ A, Blocks<T> B,
           int64_t rows_per_split, int tiles_m, double* __restrict__ part) {
  __shared__ __align__(16) T As[TK][LDS];
  __shared__ __align__(16) T Bs[TK][LDS];
  const int n = B.total();
  const int split = blockIdx.x;
  const int tile = blockIdx.y;
  const int i0 = (tile % tiles_m) * TM;
  const int j0 = (tile / tiles_m) * TN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t rb = (int64_t)split * rows_per_split;
  const int64_t re = min(N, rb + rows_per_split);

  // Column base pointers for this thread's loads (fixed over the K loop).
  // Thread loads elements e = tid + 256 q, q = 0..7: kk = e % 32, col = e / 32.
  const T* pa[8];
  const T* pb[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + 256 * q;
    const int col = e / TK;
    const int ia = i0 + col;
    pa[q] = ia < m ? A + (int64_t)ia * N : nullptr;
    const int jb = j0 + col;
    if (jb < n) {
      const int seg = jb / B.cols;
      pb[q] = B.p[seg] + (int64_t)(jb - seg * B.cols) * N;
    } else {
      pb[q] = nullptr;
    }
  }
  const int kk_ld = tid % TK;

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;

  for (int64_t r0 = rb; r0 < re; r0 += TK) {
    const int64_t r = r0 + kk_ld;
    const bool rin = r < re;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int col = (tid + 256 * q) / TK;
      As[kk_ld][col] = (rin && pa[q]) ? pa[q][r] : (T)0;
      Bs[kk_ld][col] = (rin && pb[q]) ? pb[q][r] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
      Vec4<T>::ld(&As[kk][tx * 4], a);
      Vec4<T>::ld(&Bs[kk][ty * 4], b);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
  double* out = part + (size_t)split * m * n;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = i0 + tx * 4 + x;
    if (i >= m) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int j = j0 + ty * 4 + y;
      if (j < n) out[i + (size_t)j * m] = (double)acc[x][y];
    }
  }
}

// The FP64 Gram of the mixed ladder's FP64-class steps (re-orthonormalization
// and Rayleigh-Ritz) in double-float on the FP32 pipe: each FP64 value is
// split into (hi, lo) FP32 terms as it is staged, and every product is
// accumulated as hi*hi by a fused multiply-add TwoProduct plus the cross
// terms, into a pair sum by TwoSum (low parts added plainly, renormalised
// once per stage). Relative error about 2^-46 of sum |a||b| against
// FP64's 2^-53 (the all-FP64 path and trm_gram keep k_gram<double>); about
// three times the speed of FP64 on GB300, whose FP64 rate is 1/64 of FP32.
__global__ void __launch_bounds__(256)
    k_gram_df(int64_t N, int m, const double* __restrict__ A,
              Blocks<double> B, int64_t rows_per_split, int tiles_m,
              double* __restrict__ part) {
  __shared__ __align__(16) float Ah[TK][LDS], Al[TK][LDS];
  __shared__ __align__(16) float Bh[TK][LDS], Bl[TK][LDS];
  const int n = B.total();
  const int split = blockIdx.x;
  const int tile = blockIdx.y;
  const int i0 = (tile % tiles_m) * TM;
  const int j0 = (tile / tiles_m) * TN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t rb = (int64_t)split * rows_per_split;
  const int64_t re = min(N, rb + rows_per_split);
  const double* pa[8];
  const double* pb[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + 256 * q;
    const int col = e / TK;
    const int ia = i0 + col;
    pa[q] = ia < m ? A + (int64_t)ia * N : nullptr;
    const int jb = j0 + col;
    if (jb < n) {
      const int seg = jb / B.cols;
      pb[q] = B.p[seg] + (int64_t)(jb - seg * B.cols) * N;
    } else {
      pb[q] = nullptr;
    }
  }
  const int kk_ld = tid % TK;
  DfAcc acc[4][4];
  for (int64_t r0 = rb; r0 < re; r0 += TK) {
    const int64_t r = r0 + kk_ld;
    const bool rin = r < re;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int col = (tid + 256 * q) / TK;
      const F2 a = df_of((rin && pa[q]) ? pa[q][r] : 0.0);
      const F2 b = df_of((rin && pb[q]) ? pb[q][r] : 0.0);
      Ah[kk_ld][col] = a.h;
      Al[kk_ld][col] = a.l;
      Bh[kk_ld][col] = b.h;
      Bl[kk_ld][col] = b.l;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
      Vec4<float>::ld(&Ah[kk][tx * 4], ah);
      Vec4<float>::ld(&Al[kk][tx * 4], al);
      Vec4<float>::ld(&Bh[kk][ty * 4], bh);
      Vec4<float>::ld(&Bl[kk][ty * 4], bl);
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
  double* out = part + (size_t)split * m * n;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = i0 + tx * 4 + x;
    if (i >= m) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int j = j0 + ty * 4 + y;
      if (j < n) out[i + (size_t)j * m] = (double)acc[x][y].h + (double)acc[x][y].l;
    }
  }
}

// out[e] = sum over splits of part[k * count + e]. A CTA owns 32 consecutive
// outputs; its 8 warps take the splits k = g (mod 8) (coalesced rows of the
// partials) and the 8 sums are added in a fixed order.
__global__ void __launch_bounds__(256)
    k_sum_splits(const double* __restrict__ part, int splits, size_t count,
                 double* __restrict__ out, float* __restrict__ out32) {
  __shared__ double red[8][33];
  const int el = threadIdx.x & 31, g = threadIdx.x >> 5;
  const size_t e = (size_t)blockIdx.x * 32 + el;
  double s = 0.0;
  if (e < count) {
#pragma unroll 4
    for (int k = g; k < splits; k += 8) s += part[(size_t)k * count + e];
  }
  red[g][el] = s;
  __syncthreads();
  if (g == 0 && e < count) {
    double t = red[0][el];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][el];
    out[e] = t;
    if (out32) out32[e] = (float)t;
  }
}

// The same for partials stored as FP32 pairs (hi at [2 k count, ...), lo
// after it): the sums run in double-float on the FP32 pipe and each output
// is converted to FP64 once.
__global__ void __launch_bounds__(256)
    k_sum_splits_pairs(const float* __restrict__ part, int splits,
                       size_t count, double* __restrict__ out,
                       float* __restrict__ out32, SymSeg sym) {
  __shared__ float rh[8][33], rl[8][33];
  const int el = threadIdx.x & 31, g = threadIdx.x >> 5;
  const size_t e = (size_t)blockIdx.x * 32 + el;
  F2 acc = {0.f, 0.f};
  if (e < count) {
    size_t src = e;  // a mirrored entry of a symmetric segment reads (j, i)
    if (sym.seg >= 0) {
      const int i = (int)(e % sym.m), j = (int)(e / sym.m);
      const int seg = j / sym.seg_cols, jj = j - seg * sym.seg_cols;
      if (seg == sym.seg && i / sym.tile > jj / sym.tile)
        src = (size_t)jj + (size_t)(seg * sym.seg_cols + i) * sym.m;
    }
#pragma unroll 4
    for (int k = g; k < splits; k += 8)
      acc = df_add(acc, F2{part[2 * (size_t)k * count + src],
                           part[(2 * (size_t)k + 1) * count + src]});
  }
  rh[g][el] = acc.h;
  rl[g][el] = acc.l;
  __syncthreads();
  if (g == 0 && e < count) {
    F2 t = {rh[0][el], rl[0][el]};
#pragma unroll
    for (int q = 1; q < 8; ++q) t = df_add(t, F2{rh[q][el], rl[q][el]});
    out[e] = (double)t.h + (double)t.l;
    if (out32) out32[e] = t.h;  // the sum rounded to FP32
  }
}

void plan(int64_t N, int m, int n, int* splits, int64_t* rows) {
  const int tiles = ceil_div(m, TM) * ceil_div(n, TN);
  const int target = 4 * sm_count();
  int s = ceil_div(target, tiles);
  const int64_t max_s = (N + TK - 1) / TK;
  if (s > max_s) s = (int)max_s;
  if (s < 1) s = 1;
  int64_t r = (N + s - 1) / s;
  r = ((r + TK - 1) / TK) * TK;
  s = (int)((N + r - 1) / r);
  *splits = s;
  *rows = r;
}

}  // namespace

// Partials for either kernel a Gram of these sizes may run (the SIMT
// kernel's plan, or the tensor-core kernel's row slices for FP32 blocks).
size_t gram_partials_doubles(int64_t N, int m, int n) {
  int s;
  int64_t r;
  plan(N, m, n, &s, &r);
  return std::max((size_t)s * m * n, gram_tc_partials_doubles(N, m, n));
}

void sum_splits_pairs(const float* part, int splits, size_t count,
                      double* out, cudaStream_t s, float* out32, SymSeg sym) {
  k_sum_splits_pairs<<<ceil_div(count, 32), 256, 0, s>>>(part, splits, count,
                                                         out, out32, sym);
  TRM_CHECK_LAUNCH();
}

void sum_splits(const double* part, int splits, size_t count, double* out,
                cudaStream_t s) {
  k_sum_splits<<<ceil_div(count, 32), 256, 0, s>>>(part, splits, count, out,
                                                   nullptr);
  TRM_CHECK_LAUNCH();
}

template <typename T>
void gram(int64_t N, int m, const T* A, const Blocks<T>& B, double* out,
          double* partials, size_t partials_cap, cudaStream_t s, int* err,
          float* out32) {
  const int n = B.total();
  if (m <= 0 || n <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (gram_tc_eligible(N, m, A, B)) {  // tensor cores, FP32-class accuracy
      gram_tc(N, m, A, B, out, partials, partials_cap, err, s, out32);
      return;
    }
  }
  int splits;
  int64_t rows;
  plan(N, m, n, &splits, &rows);
  if ((size_t)splits * m * n > partials_cap)
    throw Error(-2, "gram: partials buffer too small");
  const int tiles_m = ceil_div(m, TM);
  dim3 grid(splits, tiles_m * ceil_div(n, TN));
  k_gram<T><<<grid, 256, 0, s>>>(N, m, A, B, rows, tiles_m, partials);
  TRM_CHECK_LAUNCH();
  const size_t count = (size_t)m * n;
  k_sum_splits<<<ceil_div(count, 32), 256, 0, s>>>(partials, splits, count,
                                                   out, out32);
  TRM_CHECK_LAUNCH();
}

template <typename T>
void gram_in_scratch(int64_t N, int m, const T* A, const Blocks<T>& B,
                     double* out, double* scratch, size_t scratch_doubles,
                     cudaStream_t s) {
  const int n = B.total();
  if (m <= 0 || n <= 0) return;
  if ((size_t)m * n > scratch_doubles)
    throw Error(-1, "gram: m*n exceeds the scratch capacity");
  int splits;
  int64_t rows;
  plan(N, m, n, &splits, &rows);
  const int64_t fit = (int64_t)(scratch_doubles / ((size_t)m * n));
  if (splits > fit) {  // fewer, longer row slices so the partials fit
    rows = (N + fit - 1) / fit;
    rows = ((rows + TK - 1) / TK) * TK;
    splits = (int)((N + rows - 1) / rows);
  }
  const int tiles_m = ceil_div(m, TM);
  dim3 grid(splits, tiles_m * ceil_div(n, TN));
  k_gram<T><<<grid, 256, 0, s>>>(N, m, A, B, rows, tiles_m, scratch);
  TRM_CHECK_LAUNCH();
  const size_t count = (size_t)m * n;
  k_sum_splits<<<ceil_div(count, 32), 256, 0, s>>>(scratch, splits, count,
                                                   out, nullptr);
  TRM_CHECK_LAUNCH();
}

template void gram_in_scratch<float>(int64_t, int, const float*,
                                     const Blocks<float>&, double*, double*,
                                     size_t, cudaStream_t);
template void gram_in_scratch<double>(int64_t, int, const double*,
                                      const Blocks<double>&, double*, double*,
                                      size_t, cudaStream_t);

void gram_df(int64_t N, int m, const double* A, const Blocks<double>& B,
             double* out, double* partials, size_t partials_cap,
             cudaStream_t s) {
  const int n = B.total();
  if (m <= 0 || n <= 0) return;
  int splits;
  int64_t rows;
  plan(N, m, n, &splits, &rows);
  if ((size_t)splits * m * n > partials_cap)
    throw Error(-2, "gram: partials buffer too small");
  const int tiles_m = ceil_div(m, TM);
  dim3 grid(splits, tiles_m * ceil_div(n, TN));
  k_gram_df<<<grid, 256, 0, s>>>(N, m, A, B, rows, tiles_m, partials);
  TRM_CHECK_LAUNCH();
  const size_t count = (size_t)m * n;
  k_sum_splits<<<ceil_div(count, 32), 256, 0, s>>>(partials, splits, count,
                                                   out, nullptr);
  TRM_CHECK_LAUNCH();
}

template void gram<float>(int64_t, int, const float*, const Blocks<float>&,
                          double*, double*, size_t, cudaStream_t, int*,
                          float*);
template void gram<double>(int64_t, int, const double*, const Blocks<double>&,
                           double*, double*, size_t, cudaStream_t, int*,
                           float*);

}  // namespace trm
