// Double-float ("FP32 pair") arithmetic for the FP64-accuracy steps of the
// MP2 phase (Sec. 2.2: H C, the energy terms H_D and X' = X - C diag(H_D)).
//
// GB300 runs FP64 at 1/64 of its FP32 rate, and the FP64 stencil was bound
// by that pipe. Here a value is held as hi + lo with hi = fl32(v) and
// lo = fl32(v - hi) (|lo| <= ulp(hi)/2, about 48 significant bits), and
// sums and products use the error-free transformations of Knuth (TwoSum)
// and Dekker/Kahan (TwoProduct with a fused multiply-add), so the results
// carry a relative error of a few units of 2^-48 of the magnitudes involved
// — far below what E_G at 1e-10 and residuals at 1e-10 need — while every
// operation runs on the FP32 pipe. No FP64 instruction is executed per
// element, except once per thread when an FP64 scalar is split.
#include "dfmath.cuh"
#include "ops.cuh"

namespace trm {

namespace {

// Neighbour-sum accumulator: the hi parts are added exactly (TwoSum), the
// lo parts and the rounding errors plainly; normalised once at the end.
struct Acc {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float vh, float vl) {
    const F2 t = two_sum(h, vh);
    h = t.h;
    l += t.l + vl;
  }
  __device__ __forceinline__ F2 get() const { return quick_two_sum(h, l); }
};

__global__ void k_split_df(int64_t n, const double* __restrict__ x,
                           float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const F2 v = df_of(x[i]);
    hi[i] = v.h;
    lo[i] = v.l;
  }
}

__global__ void k_join_df(int64_t n, const float* __restrict__ hi,
                          const float* __restrict__ lo,
                          double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (double)hi[i] + (double)lo[i];
}

constexpr int kCols = 4;  // columns per CTA (grid.y walks column groups)

// X = H C for the stencil operator, one grid point per thread.
template <int R>
__global__ void __launch_bounds__(256)
    k_stencil_df(StencilOp st, int64_t N, const float* __restrict__ dh,
                 const float* __restrict__ dl, const float* __restrict__ Ch,
                 const float* __restrict__ Cl, float* __restrict__ Xh,
                 float* __restrict__ Xl, int ncols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int x = (int)(i % st.nx);
  const int64_t yz = i / st.nx;
  const int y = (int)(yz % st.ny);
  const int z = (int)(yz / st.ny);
  const int64_t sy = st.nx, sz = (int64_t)st.nx * st.ny;
  const F2 d = {dh[i], dl[i]};
  const F2 c1 = {st.c1h, st.c1l}, c2 = {st.c2h, st.c2l};
  // neighbours present at this point (Dirichlet: absent ones are 0)
  const bool xm1 = x >= 1, xp1 = x + 1 < st.nx, ym1 = y >= 1,
             yp1 = y + 1 < st.ny, zm1 = z >= 1, zp1 = z + 1 < st.nz;
  const bool xm2 = x >= 2, xp2 = x + 2 < st.nx, ym2 = y >= 2,
             yp2 = y + 2 < st.ny, zm2 = z >= 2, zp2 = z + 2 < st.nz;
  const int cb = blockIdx.y * kCols;
  for (int q = 0; q < kCols; ++q) {
    const int c = cb + q;
    if (c >= ncols) break;
    const int64_t base = (int64_t)c * N + i;
    const float* ph = Ch + base;
    const float* pl = Cl + base;
    Acc s1, s2;
    if (xm1) s1.add(__ldg(ph - 1), __ldg(pl - 1));
    if (xp1) s1.add(__ldg(ph + 1), __ldg(pl + 1));
    if (ym1) s1.add(__ldg(ph - sy), __ldg(pl - sy));
    if (yp1) s1.add(__ldg(ph + sy), __ldg(pl + sy));
    if (zm1) s1.add(__ldg(ph - sz), __ldg(pl - sz));
    if (zp1) s1.add(__ldg(ph + sz), __ldg(pl + sz));
    if (R == 2) {
      if (xm2) s2.add(__ldg(ph - 2), __ldg(pl - 2));
      if (xp2) s2.add(__ldg(ph + 2), __ldg(pl + 2));
      if (ym2) s2.add(__ldg(ph - 2 * sy), __ldg(pl - 2 * sy));
      if (yp2) s2.add(__ldg(ph + 2 * sy), __ldg(pl + 2 * sy));
      if (zm2) s2.add(__ldg(ph - 2 * sz), __ldg(pl - 2 * sz));
      if (zp2) s2.add(__ldg(ph + 2 * sz), __ldg(pl + 2 * sz));
    }
    F2 r = df_mul(d, F2{__ldg(ph), __ldg(pl)});
    r = df_add(r, df_mul(c1, s1.get()));
    if (R == 2) r = df_add(r, df_mul(c2, s2.get()));
    Xh[base] = r.h;
    Xl[base] = r.l;
  }
}

// The same four grid points at a time (nx % 4 == 0): one thread owns points
// x0..x0+3 of a row, loads the centre, the neighbouring quads along x and the
// y/z neighbours as 16-byte (hi, lo) vectors, and takes the x neighbours
// from registers, which cuts loads and boundary logic per point fourfold.
//
// With DOTS the column dots H_D = c_j . (H c)_j of Fig. EGFIG step (2) are
// formed from the pairs in registers (the arithmetic of k_coldot_df per
// thread, double-float warp sums, one FP64 add per warp), so the MP2 step
// does not read C and X again: CTA b writes dots[b * ncols + column].
template <int R, bool DOTS>
__global__ void __launch_bounds__(256)
    k_stencil_df_v4(StencilOp st, int64_t N, const float* __restrict__ dh,
                    const float* __restrict__ dl, const float* __restrict__ Ch,
                    const float* __restrict__ Cl, float* __restrict__ Xh,
                    float* __restrict__ Xl, int ncols,
                    double* __restrict__ dots) {
  const int64_t v0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = v0 < (N >> 2);
  if (!DOTS && !valid) return;  // with DOTS every thread joins the sums
  const int64_t v = valid ? v0 : 0;
  __shared__ double red[kCols][8];
  F2 dacc[kCols];
#pragma unroll
  for (int q = 0; q < kCols; ++q) dacc[q] = F2{0.f, 0.f};
  const int nxv = st.nx >> 2;
  const int xv = (int)(v % nxv);
  const int64_t yz = v / nxv;
  const int y = (int)(yz % st.ny);
  const int z = (int)(yz / st.ny);
  const int64_t i0 = v << 2;
  const int64_t sy = st.nx, sz = (int64_t)st.nx * st.ny;
  const bool xl = xv > 0, xr = xv + 1 < nxv;
  const bool ym1 = y >= 1, yp1 = y + 1 < st.ny, zm1 = z >= 1,
             zp1 = z + 1 < st.nz;
  const bool ym2 = y >= 2, yp2 = y + 2 < st.ny, zm2 = z >= 2,
             zp2 = z + 2 < st.nz;
  const float4 d4h = *reinterpret_cast<const float4*>(dh + i0);
  const float4 d4l = *reinterpret_cast<const float4*>(dl + i0);
  const float dH[4] = {d4h.x, d4h.y, d4h.z, d4h.w};
  const float dL[4] = {d4l.x, d4l.y, d4l.z, d4l.w};
  const F2 c1 = {st.c1h, st.c1l}, c2 = {st.c2h, st.c2l};
  auto ld = [](const float* p) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    return t;
  };
  auto add4 = [](Acc (&a)[4], const float4& h, const float4& l) {
    a[0].add(h.x, l.x);
    a[1].add(h.y, l.y);
    a[2].add(h.z, l.z);
    a[3].add(h.w, l.w);
  };
  const int cb = blockIdx.y * kCols;
#pragma unroll
  for (int q = 0; q < kCols; ++q) {
    const int c = cb + q;
    if (c >= ncols || !valid) break;
    const int64_t base = (int64_t)c * N + i0;
    const float* ph = Ch + base;
    const float* pl = Cl + base;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ch = ld(ph), cl = ld(pl);
    const float4 lh = xl ? ld(ph - 4) : zero, ll = xl ? ld(pl - 4) : zero;
    const float4 rh = xr ? ld(ph + 4) : zero, rl = xr ? ld(pl + 4) : zero;
    Acc s1[4], s2[4];
    if (ym1) add4(s1, ld(ph - sy), ld(pl - sy));
    if (yp1) add4(s1, ld(ph + sy), ld(pl + sy));
    if (zm1) add4(s1, ld(ph - sz), ld(pl - sz));
    if (zp1) add4(s1, ld(ph + sz), ld(pl + sz));
    // x neighbours at distance 1: (l.w, c.x, c.y, c.z) and (c.y, c.z, c.w, r.x)
    s1[0].add(lh.w, ll.w); s1[0].add(ch.y, cl.y);
    s1[1].add(ch.x, cl.x); s1[1].add(ch.z, cl.z);
    s1[2].add(ch.y, cl.y); s1[2].add(ch.w, cl.w);
    s1[3].add(ch.z, cl.z); s1[3].add(rh.x, rl.x);
    if (R == 2) {
      if (ym2) add4(s2, ld(ph - 2 * sy), ld(pl - 2 * sy));
      if (yp2) add4(s2, ld(ph + 2 * sy), ld(pl + 2 * sy));
      if (zm2) add4(s2, ld(ph - 2 * sz), ld(pl - 2 * sz));
      if (zp2) add4(s2, ld(ph + 2 * sz), ld(pl + 2 * sz));
      // distance 2: (l.z, l.w, c.x, c.y) and (c.z, c.w, r.x, r.y)
      s2[0].add(lh.z, ll.z); s2[0].add(ch.z, cl.z);
      s2[1].add(lh.w, ll.w); s2[1].add(ch.w, cl.w);
      s2[2].add(ch.x, cl.x); s2[2].add(rh.x, rl.x);
      s2[3].add(ch.y, cl.y); s2[3].add(rh.y, rl.y);
    }
    const float cH[4] = {ch.x, ch.y, ch.z, ch.w};
    const float cL[4] = {cl.x, cl.y, cl.z, cl.w};
    float oh[4], ol[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      F2 r = df_mul(F2{dH[k], dL[k]}, F2{cH[k], cL[k]});
      r = df_add(r, df_mul(c1, s1[k].get()));
      if (R == 2) r = df_add(r, df_mul(c2, s2[k].get()));
      oh[k] = r.h;
      ol[k] = r.l;
    }
    *reinterpret_cast<float4*>(Xh + base) = make_float4(oh[0], oh[1], oh[2], oh[3]);
    *reinterpret_cast<float4*>(Xl + base) = make_float4(ol[0], ol[1], ol[2], ol[3]);
    if (DOTS) {
      F2 a = dacc[q];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        a = df_add(a, df_mul(F2{cH[k], cL[k]}, F2{oh[k], ol[k]}));
      dacc[q] = a;
    }
  }
  if (DOTS) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kCols; ++q) {
      F2 w = dacc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        w = df_add(w, F2{__shfl_xor_sync(0xffffffffu, w.h, o),
                         __shfl_xor_sync(0xffffffffu, w.l, o)});
      if (lane == 0) red[q][warp] = to_f64(w.h) + to_f64(w.l);
    }
    __syncthreads();
    if (threadIdx.x < kCols && cb + (int)threadIdx.x < ncols) {
      double t = red[threadIdx.x][0];
#pragma unroll
      for (int w = 1; w < 8; ++w) t += red[threadIdx.x][w];
      dots[(size_t)blockIdx.x * ncols + cb + threadIdx.x] = t;
    }
  }
}

// X = H C for a CSR operator (values split into hi + lo at creation).
__global__ void __launch_bounds__(256)
    k_csr_df(int64_t N, const int32_t* __restrict__ rowptr,
             const int32_t* __restrict__ cols, const float* __restrict__ vh,
             const float* __restrict__ vl, const float* __restrict__ Ch,
             const float* __restrict__ Cl, float* __restrict__ Xh,
             float* __restrict__ Xl, int ncols) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int b = rowptr[r], e = rowptr[r + 1];
  const int cb = blockIdx.y * kCols;
  for (int q = 0; q < kCols; ++q) {
    const int c = cb + q;
    if (c >= ncols) break;
    const int64_t off = (int64_t)c * N;
    F2 acc = {0.f, 0.f};
    for (int k = b; k < e; ++k) {
      const int64_t j = off + cols[k];
      acc = df_add(acc, df_mul(F2{vh[k], vl[k]}, F2{__ldg(Ch + j), __ldg(Cl + j)}));
    }
    Xh[off + r] = acc.h;
    Xl[off + r] = acc.l;
  }
}

constexpr int kRowChunk = 4096;  // rows per partial of the column dots

// dots[chunk * m + j] = sum_{i in chunk} C_ij X_ij (16-byte vectors when
// N % 4 == 0 and the blocks are 16-byte aligned)
__global__ void __launch_bounds__(256)
    k_coldot_df(int64_t N, int m, const float* __restrict__ Ch,
                const float* __restrict__ Cl, const float* __restrict__ Xh,
                const float* __restrict__ Xl, double* __restrict__ dots,
                int vec) {
  __shared__ double red[32];
  const int j = blockIdx.y;
  const int64_t rb = (int64_t)blockIdx.x * kRowChunk;
  const int64_t re = min(N, rb + kRowChunk);
  const int64_t off = (int64_t)j * N;
  F2 acc = {0.f, 0.f};
  if (vec) {
    const float4* ch = reinterpret_cast<const float4*>(Ch + off);
    const float4* cl = reinterpret_cast<const float4*>(Cl + off);
    const float4* xh = reinterpret_cast<const float4*>(Xh + off);
    const float4* xl = reinterpret_cast<const float4*>(Xl + off);
    for (int64_t i = (rb >> 2) + threadIdx.x; i < (re >> 2); i += blockDim.x) {
      const float4 a = ch[i], b = cl[i], c = xh[i], d = xl[i];
      acc = df_add(acc, df_mul(F2{a.x, b.x}, F2{c.x, d.x}));
      acc = df_add(acc, df_mul(F2{a.y, b.y}, F2{c.y, d.y}));
      acc = df_add(acc, df_mul(F2{a.z, b.z}, F2{c.z, d.z}));
      acc = df_add(acc, df_mul(F2{a.w, b.w}, F2{c.w, d.w}));
    }
  } else {
    for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x)
      acc = df_add(acc, df_mul(F2{Ch[off + i], Cl[off + i]},
                               F2{Xh[off + i], Xl[off + i]}));
  }
  double v[1] = {to_double(acc)};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) dots[(size_t)blockIdx.x * m + j] = v[0];
}

// X32 = fl32(X - C diag(H_D))
__global__ void k_xprime_df(int64_t N, const float* __restrict__ Ch,
                            const float* __restrict__ Cl,
                            const float* __restrict__ Xh,
                            const float* __restrict__ Xl,
                            const double* __restrict__ HD,
                            float* __restrict__ X32) {
  const int j = blockIdx.y;
  const F2 h = df_of(-HD[j]);
  const int64_t off = (int64_t)j * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const F2 t = df_mul(F2{Ch[off + i], Cl[off + i]}, h);
    X32[off + i] = df_add(F2{Xh[off + i], Xl[off + i]}, t).h;
  }
}

// The same on 16-byte vectors (N % 4 == 0, aligned blocks).
__global__ void k_xprime_df4(int64_t N, const float4* __restrict__ Ch,
                             const float4* __restrict__ Cl,
                             const float4* __restrict__ Xh,
                             const float4* __restrict__ Xl,
                             const double* __restrict__ HD,
                             float4* __restrict__ X32) {
  const int j = blockIdx.y;
  const F2 h = df_of(-HD[j]);
  const int64_t n4 = N >> 2, off = (int64_t)j * n4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = Ch[off + i], b = Cl[off + i], c = Xh[off + i],
                 d = Xl[off + i];
    float4 o;
    o.x = df_add(F2{c.x, d.x}, df_mul(F2{a.x, b.x}, h)).h;
    o.y = df_add(F2{c.y, d.y}, df_mul(F2{a.y, b.y}, h)).h;
    o.z = df_add(F2{c.z, d.z}, df_mul(F2{a.z, b.z}, h)).h;
    o.w = df_add(F2{c.w, d.w}, df_mul(F2{a.w, b.w}, h)).h;
    X32[off + i] = o;
  }
}

int grid_1d(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 8 * 4096 ? 8 * 4096 : g));
}

}  // namespace

void split_df(const double* x, float* hi, float* lo, int64_t n,
              cudaStream_t s) {
  k_split_df<<<grid_1d(n), 256, 0, s>>>(n, x, hi, lo);
  TRM_CHECK_LAUNCH();
}

void join_df(const float* hi, const float* lo, double* x, int64_t n,
             cudaStream_t s) {
  k_join_df<<<grid_1d(n), 256, 0, s>>>(n, hi, lo, x);
  TRM_CHECK_LAUNCH();
}

void apply_h_df(const Operator& op, const float* Ch, const float* Cl,
                float* Xh, float* Xl, int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  const int gy = ceil_div(ncols, kCols);
  if (gy > 65535) throw Error(-1, "too many columns for one launch");
  dim3 grid(ceil_div(op.N, 256), gy);
  const bool v4 = op.kind == 0 && op.st.nx % 4 == 0 && op.N % 4 == 0 &&
                  ((reinterpret_cast<uintptr_t>(Ch) | reinterpret_cast<uintptr_t>(Cl) |
                    reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl) |
                    reinterpret_cast<uintptr_t>(op.diag32) |
                    reinterpret_cast<uintptr_t>(op.diaglo)) & 15) == 0;
  if (v4) {
    dim3 g4(ceil_div(op.N / 4, 256), gy);
    if (op.st.radius == 1)
      k_stencil_df_v4<1, false><<<g4, 256, 0, s>>>(
          op.st, op.N, op.diag32, op.diaglo, Ch, Cl, Xh, Xl, ncols, nullptr);
    else
      k_stencil_df_v4<2, false><<<g4, 256, 0, s>>>(
          op.st, op.N, op.diag32, op.diaglo, Ch, Cl, Xh, Xl, ncols, nullptr);
  } else if (op.kind == 0) {
    if (op.st.radius == 1)
      k_stencil_df<1><<<grid, 256, 0, s>>>(op.st, op.N, op.diag32, op.diaglo,
                                           Ch, Cl, Xh, Xl, ncols);
    else
      k_stencil_df<2><<<grid, 256, 0, s>>>(op.st, op.N, op.diag32, op.diaglo,
                                           Ch, Cl, Xh, Xl, ncols);
  } else {
    k_csr_df<<<grid, 256, 0, s>>>(op.N, op.csr.rowptr, op.csr.cols,
                                  op.csr.valshi, op.csr.valslo, Ch, Cl, Xh,
                                  Xl, ncols);
  }
  TRM_CHECK_LAUNCH();
}

int apply_h_df_dots(const Operator& op, const float* Ch, const float* Cl,
                    float* Xh, float* Xl, int ncols, double* dots,
                    cudaStream_t s) {
  if (ncols <= 0) return 0;
  const bool v4 = op.kind == 0 && op.st.nx % 4 == 0 && op.N % 4 == 0 &&
                  ((reinterpret_cast<uintptr_t>(Ch) | reinterpret_cast<uintptr_t>(Cl) |
                    reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl) |
                    reinterpret_cast<uintptr_t>(op.diag32) |
                    reinterpret_cast<uintptr_t>(op.diaglo)) & 15) == 0;
  const int gy = ceil_div(ncols, kCols);
  if (!v4 || gy > 65535) return 0;  // the caller forms the dots separately
  dim3 g4(ceil_div(op.N / 4, 256), gy);
  if (op.st.radius == 1)
    k_stencil_df_v4<1, true><<<g4, 256, 0, s>>>(
        op.st, op.N, op.diag32, op.diaglo, Ch, Cl, Xh, Xl, ncols, dots);
  else
    k_stencil_df_v4<2, true><<<g4, 256, 0, s>>>(
        op.st, op.N, op.diag32, op.diaglo, Ch, Cl, Xh, Xl, ncols, dots);
  TRM_CHECK_LAUNCH();
  return (int)g4.x;  // partial dots per column
}

void energy_diag_df(int64_t N, int m, const float* Ch, const float* Cl,
                    const float* Xh, const float* Xl, double* HD,
                    IterScalars* sc, double* partials, cudaStream_t s) {
  const int chunks = ceil_div(N, kRowChunk);
  const int vec = N % 4 == 0 &&
                  ((reinterpret_cast<uintptr_t>(Ch) | reinterpret_cast<uintptr_t>(Cl) |
                    reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl)) &
                   15) == 0;
  k_coldot_df<<<dim3(chunks, m), 256, 0, s>>>(N, m, Ch, Cl, Xh, Xl, partials,
                                               vec);
  TRM_CHECK_LAUNCH();
  energy_from_dots(partials, chunks, m, HD, sc, s);
}

void xprime_df(int64_t N, int m, const float* Ch, const float* Cl,
               const float* Xh, const float* Xl, const double* HD, float* X32,
               cudaStream_t s) {
  int gx = ceil_div(N, 256 * 4);
  gx = gx < 1 ? 1 : (gx > 4096 ? 4096 : gx);
  if (N % 4 == 0 &&
      ((reinterpret_cast<uintptr_t>(Ch) | reinterpret_cast<uintptr_t>(Cl) |
        reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl) |
        reinterpret_cast<uintptr_t>(X32)) & 15) == 0) {
    k_xprime_df4<<<dim3(gx, m), 256, 0, s>>>(
        N, reinterpret_cast<const float4*>(Ch), reinterpret_cast<const float4*>(Cl),
        reinterpret_cast<const float4*>(Xh), reinterpret_cast<const float4*>(Xl),
        HD, reinterpret_cast<float4*>(X32));
    TRM_CHECK_LAUNCH();
    return;
  }
  k_xprime_df<<<dim3(gx, m), 256, 0, s>>>(N, Ch, Cl, Xh, Xl, HD, X32);
  TRM_CHECK_LAUNCH();
}

}  // namespace trm
