// H applied to a block of columns: X = H C (Fig. EGFIG, step (1)).
//
// Stencil operators: H = t (T_x (+) T_y (+) T_z) + diag(V) on a Dirichlet grid,
// x fastest. Every column is one grid function; a thread owns four consecutive
// x points of one (y, z) row and walks a few columns, so the grid-index work
// and the diagonal are shared across columns and every access is a 16-byte
// vector load (x neighbours come from the vectors left and right of it).
// CSR operators: one thread per row keeps the row's entries in registers and
// walks the columns of its column group.
#include "ops.cuh"

namespace trm {

namespace {

template <typename T>
struct V4 {
  T v[4];
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.v[0], v.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.v[2], v.v[3]);
}

template <typename T>
__device__ __forceinline__ const T* diag_ptr(const double* d64,
                                             const float* d32);
template <>
__device__ __forceinline__ const float* diag_ptr<float>(const double*,
                                                        const float* d32) {
  return d32;
}
template <>
__device__ __forceinline__ const double* diag_ptr<double>(const double* d64,
                                                          const float*) {
  return d64;
}

// Columns per CTA (grid.y walks column groups).
constexpr int kCpb = 4;

// Column dot products sum_i X_ic Y_ic fused into H X (Fig. EGFIG steps
// (2), (3) read exactly the block pair this kernel holds): every warp adds
// its lanes' products per column into red[q][warp]; after the column loop
// the CTA's 8 warp sums are added in a fixed order and written to
// dots[blockIdx.x * ncols + c].
template <typename T>
__device__ __forceinline__ void warp_dot(T d, double (*red)[8], int q) {
  d = warp_sum(d);
  if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = (double)d;
}
__device__ __forceinline__ void write_dots(double (*red)[8], double* dots,
                                           int cb, int ncols) {
  __syncthreads();
  if (threadIdx.x < kCpb && cb + (int)threadIdx.x < ncols) {
    double t = red[threadIdx.x][0];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += red[threadIdx.x][w];
    dots[(size_t)blockIdx.x * ncols + cb + threadIdx.x] = t;
  }
}

// Four x points per thread; requires nx % 4 == 0.
template <typename T, int R, bool DOTS>
__global__ void __launch_bounds__(256)
    k_stencil_v4(StencilOp st, int64_t N, const double* __restrict__ d64,
                 const float* __restrict__ d32, const T* __restrict__ X,
                 T* __restrict__ Y, int ncols, double* __restrict__ dots) {
  const int64_t nv = N >> 2;
  const int64_t v0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = v0 < nv;
  if (!DOTS && !valid) return;  // with DOTS every thread joins the sums
  const int64_t v = valid ? v0 : 0;
  __shared__ double red[kCpb][8];
  const int nxv = st.nx >> 2;
  const int xv = (int)(v % nxv);
  const int64_t yz = v / nxv;
  const int y = (int)(yz % st.ny);
  const int z = (int)(yz / st.ny);
  const int64_t i0 = v << 2;
  const int64_t sy = st.nx, sz = (int64_t)st.nx * st.ny;
  const bool xl = xv > 0, xr = xv + 1 < nxv;
  const bool ym1 = y >= 1, yp1 = y + 1 < st.ny;
  const bool zm1 = z >= 1, zp1 = z + 1 < st.nz;
  const bool ym2 = y >= 2, yp2 = y + 2 < st.ny;
  const bool zm2 = z >= 2, zp2 = z + 2 < st.nz;
  const V4<T> d = ld4(diag_ptr<T>(d64, d32) + i0);
  const T c1 = (T)st.c1, c2 = (T)st.c2;
  const int cb = blockIdx.y * kCpb;
  for (int q = 0; q < kCpb; ++q) {
    const int c = cb + q;
    if (c >= ncols) break;
    if (DOTS && !valid) {
      warp_dot((T)0, red, q);
      continue;
    }
    const T* x = X + (int64_t)c * N + i0;
    const V4<T> xc = ld4(x);
    V4<T> xlv = {{0, 0, 0, 0}}, xrv = {{0, 0, 0, 0}};
    if (xl) xlv = ld4(x - 4);
    if (xr) xrv = ld4(x + 4);
    T s1[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0};
    if (ym1) { V4<T> a = ld4(x - sy); for (int k = 0; k < 4; ++k) s1[k] += a.v[k]; }
    if (yp1) { V4<T> a = ld4(x + sy); for (int k = 0; k < 4; ++k) s1[k] += a.v[k]; }
    if (zm1) { V4<T> a = ld4(x - sz); for (int k = 0; k < 4; ++k) s1[k] += a.v[k]; }
    if (zp1) { V4<T> a = ld4(x + sz); for (int k = 0; k < 4; ++k) s1[k] += a.v[k]; }
    if (R == 2) {
      if (ym2) { V4<T> a = ld4(x - 2 * sy); for (int k = 0; k < 4; ++k) s2[k] += a.v[k]; }
      if (yp2) { V4<T> a = ld4(x + 2 * sy); for (int k = 0; k < 4; ++k) s2[k] += a.v[k]; }
      if (zm2) { V4<T> a = ld4(x - 2 * sz); for (int k = 0; k < 4; ++k) s2[k] += a.v[k]; }
      if (zp2) { V4<T> a = ld4(x + 2 * sz); for (int k = 0; k < 4; ++k) s2[k] += a.v[k]; }
    }
    // x neighbours: l1/r1 at distance 1, l2/r2 at distance 2
    const T l1[4] = {xlv.v[3], xc.v[0], xc.v[1], xc.v[2]};
    const T r1[4] = {xc.v[1], xc.v[2], xc.v[3], xrv.v[0]};
    V4<T> out;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T acc = d.v[k] * xc.v[k] + c1 * (s1[k] + l1[k] + r1[k]);
      if (R == 2) {
        const T l2 = k < 2 ? xlv.v[2 + k] : xc.v[k - 2];
        const T r2 = k > 1 ? xrv.v[k - 2] : xc.v[k + 2];
        acc += c2 * (s2[k] + l2 + r2);
      }
      out.v[k] = acc;
    }
    st4(Y + (int64_t)c * N + i0, out);
    if (DOTS)
      warp_dot(xc.v[0] * out.v[0] + xc.v[1] * out.v[1] +
                   xc.v[2] * out.v[2] + xc.v[3] * out.v[3],
               red, q);
  }
  if (DOTS) write_dots(red, dots, cb, ncols);
}

// One point per thread, any nx.
template <typename T, int R, bool DOTS>
__global__ void __launch_bounds__(256)
    k_stencil_1(StencilOp st, int64_t N, const double* __restrict__ d64,
                const float* __restrict__ d32, const T* __restrict__ X,
                T* __restrict__ Y, int ncols, double* __restrict__ dots) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i0 < N;
  if (!DOTS && !valid) return;
  const int64_t i = valid ? i0 : 0;
  __shared__ double red[kCpb][8];
  const int x = (int)(i % st.nx);
  const int64_t yz = i / st.nx;
  const int y = (int)(yz % st.ny);
  const int z = (int)(yz / st.ny);
  const int64_t sy = st.nx, sz = (int64_t)st.nx * st.ny;
  const T d = diag_ptr<T>(d64, d32)[i];
  const T c1 = (T)st.c1, c2 = (T)st.c2;
  const int cb = blockIdx.y * kCpb;
  for (int q = 0; q < kCpb; ++q) {
    const int c = cb + q;
    if (c >= ncols) break;
    if (DOTS && !valid) {
      warp_dot((T)0, red, q);
      continue;
    }
    const T* xp = X + (int64_t)c * N + i;
    T s1 = 0, s2 = 0;
    if (x >= 1) s1 += xp[-1];
    if (x + 1 < st.nx) s1 += xp[1];
    if (y >= 1) s1 += xp[-sy];
    if (y + 1 < st.ny) s1 += xp[sy];
    if (z >= 1) s1 += xp[-sz];
    if (z + 1 < st.nz) s1 += xp[sz];
    T acc = d * xp[0] + c1 * s1;
    if (R == 2) {
      if (x >= 2) s2 += xp[-2];
      if (x + 2 < st.nx) s2 += xp[2];
      if (y >= 2) s2 += xp[-2 * sy];
      if (y + 2 < st.ny) s2 += xp[2 * sy];
      if (z >= 2) s2 += xp[-2 * sz];
      if (z + 2 < st.nz) s2 += xp[2 * sz];
      acc += c2 * s2;
    }
    Y[(int64_t)c * N + i] = acc;
    if (DOTS) warp_dot(xp[0] * acc, red, q);
  }
  if (DOTS) write_dots(red, dots, cb, ncols);
}

constexpr int kCsrCache = 16;

template <typename T, typename TV, bool DOTS>
__global__ void __launch_bounds__(256)
    k_csr(int64_t N, const int32_t* __restrict__ rowptr,
          const int32_t* __restrict__ cols, const TV* __restrict__ vals,
          const T* __restrict__ X, T* __restrict__ Y, int ncols,
          double* __restrict__ dots) {
  const int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r0 < N;
  if (!DOTS && !valid) return;
  const int64_t r = valid ? r0 : 0;
  __shared__ double red[kCpb][8];
  const int b = valid ? rowptr[r] : 0, e = valid ? rowptr[r + 1] : 0;
  const int nnz = e - b;
  const int cb = blockIdx.y * kCpb;
  if (nnz <= kCsrCache) {
    int ci[kCsrCache];
    T cv[kCsrCache];
#pragma unroll
    for (int k = 0; k < kCsrCache; ++k) {
      ci[k] = k < nnz ? cols[b + k] : 0;
      cv[k] = k < nnz ? (T)vals[b + k] : (T)0;
    }
    for (int q = 0; q < kCpb; ++q) {
      const int c = cb + q;
      if (c >= ncols) break;
      T d = 0;
      if (valid) {
        const T* x = X + (int64_t)c * N;
        T acc = 0;
#pragma unroll
        for (int k = 0; k < kCsrCache; ++k)
          if (k < nnz) acc += cv[k] * __ldg(x + ci[k]);
        Y[(int64_t)c * N + r] = acc;
        d = x[r] * acc;
      }
      if (DOTS) warp_dot(d, red, q);
    }
  } else {
    for (int q = 0; q < kCpb; ++q) {
      const int c = cb + q;
      if (c >= ncols) break;
      T d = 0;
      if (valid) {
        const T* x = X + (int64_t)c * N;
        T acc = 0;
        for (int k = b; k < e; ++k) acc += (T)vals[k] * __ldg(x + cols[k]);
        Y[(int64_t)c * N + r] = acc;
        d = x[r] * acc;
      }
      if (DOTS) warp_dot(d, red, q);
    }
  }
  if (DOTS) write_dots(red, dots, cb, ncols);
}

template <typename T, bool DOTS>
int launch_apply(const Operator& op, const T* X, T* Y, int ncols, double* dots,
                 cudaStream_t s) {
  const int threads = 256;
  const int gy = ceil_div(ncols, kCpb);
  if (gy > 65535) throw Error(-1, "too many columns for one launch");
  dim3 grid;
  if (op.kind == 0) {
    const StencilOp& st = op.st;
    if (st.nx % 4 == 0) {
      grid = dim3(ceil_div(op.N / 4, threads), gy);
      if (st.radius == 1)
        k_stencil_v4<T, 1, DOTS><<<grid, threads, 0, s>>>(
            st, op.N, op.diag64, op.diag32, X, Y, ncols, dots);
      else
        k_stencil_v4<T, 2, DOTS><<<grid, threads, 0, s>>>(
            st, op.N, op.diag64, op.diag32, X, Y, ncols, dots);
    } else {
      grid = dim3(ceil_div(op.N, threads), gy);
      if (st.radius == 1)
        k_stencil_1<T, 1, DOTS><<<grid, threads, 0, s>>>(
            st, op.N, op.diag64, op.diag32, X, Y, ncols, dots);
      else
        k_stencil_1<T, 2, DOTS><<<grid, threads, 0, s>>>(
            st, op.N, op.diag64, op.diag32, X, Y, ncols, dots);
    }
  } else {
    grid = dim3(ceil_div(op.N, threads), gy);
    if (op.csr.vals64)
      k_csr<T, double, DOTS><<<grid, threads, 0, s>>>(
          op.N, op.csr.rowptr, op.csr.cols, op.csr.vals64, X, Y, ncols, dots);
    else
      k_csr<T, float, DOTS><<<grid, threads, 0, s>>>(
          op.N, op.csr.rowptr, op.csr.cols, op.csr.vals32, X, Y, ncols, dots);
  }
  TRM_CHECK_LAUNCH();
  return (int)grid.x;
}

__global__ void k_stencil_diag(int64_t N, double base,
                               const double* __restrict__ V, double* d64,
                               float* d32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double d = base + (V ? V[i] : 0.0);
  d64[i] = d;
  d32[i] = (float)d;
}

template <typename TV>
__global__ void k_csr_diag(int64_t N, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ cols,
                           const TV* __restrict__ vals, double* d64,
                           float* d32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double d = 0.0;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k)
    if (cols[k] == r) d += (double)vals[k];
  d64[r] = d;
  d32[r] = (float)d;
}

// Block-wise minima of x, then the reciprocal shift.
__global__ void k_min_partial(const double* __restrict__ x, int64_t n,
                              double* out) {
  __shared__ double sm[32];
  double v = 1e300;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v = fmin(v, x[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

__global__ void k_precond(const double* __restrict__ d, int64_t n,
                          const double* __restrict__ mins, int nmins,
                          double* m64, float* m32) {
  double mn = 1e300;
  for (int k = 0; k < nmins; ++k) mn = fmin(mn, mins[k]);
  const double sigma = mn - 1.0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = 1.0 / (d[i] - sigma);
  m64[i] = v;
  m32[i] = (float)v;
}

}  // namespace

void apply_h(const Operator& op, const float* X, float* Y, int ncols,
             cudaStream_t s) {
  if (ncols > 0) launch_apply<float, false>(op, X, Y, ncols, nullptr, s);
}
void apply_h(const Operator& op, const double* X, double* Y, int ncols,
             cudaStream_t s) {
  if (ncols > 0) launch_apply<double, false>(op, X, Y, ncols, nullptr, s);
}
int apply_h_dots(const Operator& op, const float* X, float* Y, int ncols,
                 double* dots, cudaStream_t s) {
  return ncols > 0 ? launch_apply<float, true>(op, X, Y, ncols, dots, s) : 0;
}
size_t apply_h_dots_doubles(const Operator& op, int ncols) {
  const int64_t pts = (op.kind == 0 && op.st.nx % 4 == 0) ? op.N / 4 : op.N;
  return (size_t)ceil_div(pts, 256) * ncols;
}

void stencil_diag(const StencilOp&, double base, const double* V,
                  double* diag64, float* diag32, int64_t N, cudaStream_t s) {
  k_stencil_diag<<<ceil_div(N, 256), 256, 0, s>>>(N, base, V, diag64, diag32);
  TRM_CHECK_LAUNCH();
}

void csr_diag(const Operator& op, double* diag64, float* diag32,
              cudaStream_t s) {
  if (op.csr.vals64)
    k_csr_diag<double><<<ceil_div(op.N, 256), 256, 0, s>>>(
        op.N, op.csr.rowptr, op.csr.cols, op.csr.vals64, diag64, diag32);
  else
    k_csr_diag<float><<<ceil_div(op.N, 256), 256, 0, s>>>(
        op.N, op.csr.rowptr, op.csr.cols, op.csr.vals32, diag64, diag32);
  TRM_CHECK_LAUNCH();
}

void diag_preconditioner(const double* diag64, int64_t N, double* minv64,
                         float* minv32, double* work, cudaStream_t s) {
  const int nb = 256;
  k_min_partial<<<nb, 256, 0, s>>>(diag64, N, work);
  TRM_CHECK_LAUNCH();
  k_precond<<<ceil_div(N, 256), 256, 0, s>>>(diag64, N, work, nb, minv64,
                                             minv32);
  TRM_CHECK_LAUNCH();
}

}  // namespace trm
