// m x m matrix work on the device: products, the line model along P,
// Cholesky factorisation and triangular inverse (Fig. ONFIG steps (2), (3)),
// and the symmetric eigenproblem of the closing Rayleigh-Ritz step
// (Sec. 2.1: "diagonalization of H ... will give the explicit eigenvalues").
// All matrices are column-major with leading dimension m and stored as FP64;
// the template parameter Tm is the arithmetic type.
#include <atomic>
#include <cstdlib>

#include "ops.cuh"

namespace trm {

namespace {

// ---------------------------------------------------------------------------
// Cm = alpha op(A) op(B) + beta Cm, 16 x 16 tiles, one output per thread.
// ---------------------------------------------------------------------------
template <typename Tc>
__global__ void __launch_bounds__(256)
    k_mm_gemm(int m, const double* __restrict__ A, int trA,
              const double* __restrict__ B, int trB, double* Cm,
              double alpha, double beta) {
  __shared__ Tc As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx;
  const int j = blockIdx.y * 16 + ty;
  Tc acc = 0;
  for (int k0 = 0; k0 < m; k0 += 16) {
    const int ka = k0 + ty;
    As[ty][tx] = (i < m && ka < m) ? (Tc)(trA ? A[ka + (int64_t)i * m]
                                              : A[i + (int64_t)ka * m])
                                   : (Tc)0;
    const int kb = k0 + tx;
    Bs[ty][tx] = (kb < m && j < m) ? (Tc)(trB ? B[j + (int64_t)kb * m]
                                              : B[kb + (int64_t)j * m])
                                   : (Tc)0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc += As[kk][tx] * Bs[ty][kk];
    __syncthreads();
  }
  if (i < m && j < m) {
    const int64_t o = i + (int64_t)j * m;
    Cm[o] = alpha * (double)acc + (beta != 0.0 ? beta * Cm[o] : 0.0);
  }
}

__global__ void k_zero_diag(int m, double* A, float* A32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    A[i + (int64_t)i * m] = 0.0;
    if (A32) A32[i + (int64_t)i * m] = 0.f;
  }
}

// A0 = sym(H') + diag(H_D): the projected matrix C^T H C when C^T C = I
// (H_D may be null: plain symmetrisation).
__global__ void k_make_A0(int m, const double* __restrict__ Hp,
                          const double* __restrict__ HD, double* A0) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int i = (int)(e % m), j = (int)(e / m);
  double v = 0.5 * (Hp[i + (int64_t)j * m] + Hp[j + (int64_t)i * m]);
  if (i == j && HD) v += HD[i];
  A0[e] = v;
}

// ---------------------------------------------------------------------------
// Line model along P. With R = H C - C A0 = -G/2, the block pencil C + a P
// (C^T C = I) has S(a) = I + a S1 + a^2 Q and A(a) - S(a) A0 = a D1 + a^2 D2,
//   S1 = B + B^T,  D1 = A0 B - B A0 - (W + W^T)/2,  D2 = P^T H P - Q A0,
// with B = C^T P, Q = P^T P, W = P^T G. Every term is formed from small
// quantities, so E(a) - E(0) = tr(S(a)^{-1} (a D1 + a^2 D2)) keeps its
// relative accuracy close to convergence. To second order
//   E(a) - E(0) = a tr(D1) + a^2 (tr(D2) - tr(S1 D1)).
// ---------------------------------------------------------------------------

// The step along P: minimiser of the parabola a tr(D1) + a^2 (tr(D2) -
// tr(S1 D1)), bounded so that the RMS column change a ||P||_F / sqrt(m)
// stays below 1; a restart is requested when P is not a descent direction.
__device__ void line_alpha_block(int m, const double* __restrict__ part,
                                 int nparts, IterScalars* sc, double* red) {
  double v[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] += part[(size_t)p * 4 + q];
  block_sum<4>(v, red);
  if (threadIdx.x == 0) {
    const double g0 = v[0];
    const double c2 = v[1] - v[2];
    const double qn = v[3];
    double alpha = 0.0;
    const double cap = qn > 0.0 ? sqrt((double)m / qn) : 0.0;
    if (g0 < 0.0 && qn > 0.0) {
      if (c2 > 0.0)
        alpha = -g0 / (2.0 * c2);
      else
        alpha = sc->alpha_prev > 0.0 ? 2.0 * sc->alpha_prev : 0.5 * cap;
      if (alpha > cap) alpha = cap;
    } else {
      sc->restart = 1;  // not a descent direction: restart CG next time
    }
    sc->alpha = alpha;
    sc->alpha_prev = alpha > 0.0 ? alpha : sc->alpha_prev;
    sc->c2 = c2;
    sc->dE = alpha * g0 + alpha * alpha * c2;
  }
}

// ---------------------------------------------------------------------------
// Cholesky S = L L^T and L^{-1}, blocked in 32-column panels, one CTA of 256
// threads. Writes Linv (lower) and R = L^{-T} (upper).
//
// m is padded to mp, a multiple of 32, with the identity, which changes
// neither factor. Per panel p: (a) the eight warps factor the diagonal block
// column by column (right-looking), four columns per warp in registers: the
// owner of a column takes its pivot by a shuffle and publishes the column
// through shared memory, and each warp updates its own columns; (b) every row
// below solves x L_pp^T = a (registers, reciprocal pivots from (a));
// (c) all threads update the lower trailing triangle with 4 x 4 register
// tiles. The inverse: (d) warp p inverts diagonal block p by forward
// substitution, one column of the inverse per lane in registers, rows of L
// read as broadcasts; (e) row-block by row-block,
// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj through a 32 x mp temporary. The
// working copy has leading dimension mp + 1. Linv may be null (only R is
// written then). Every pivot chain step is a dependent sequence, so the
// phases avoid shuffles and global loads inside it.
//
// S is read from memory, or (Bm != null) formed on the fly as
// S = I + a (B + B^T) + a^2 Q with a = sc->alpha (the line step's overlap).
//
// With dev = true the factorisation runs in deviation form for S = I + E:
// L = I + F and L^{-1} = I + Y with the identity kept exact and only the
// small E, F, Y held in Tm. Pivot: d = E_cc - sum_k F_ck^2 and
// f_cc = d / (1 + sqrt(1 + d)); off the diagonal L and F coincide; inverse
// diagonal y_cc = -f_cc / (1 + f_cc). When S - I is small, FP32 arithmetic
// here yields L to FP64 accuracy relative to I.
// ---------------------------------------------------------------------------
// Reciprocal square root and reciprocal of the pivot chain by Newton's
// method from the hardware approximations (rsqrt, reciprocal): one step in
// FP32, two from the FP32 seed in FP64. Arguments are positive normal numbers (the pivot
// tests come first); the results are within a few ulp, and the chain stays
// free of the slow-path calls of the IEEE operations.
__device__ __forceinline__ float piv_rcp(float t) {
  const float r = __fdividef(1.0f, t);
  return fmaf(r, fmaf(-t, r, 1.0f), r);
}
__device__ __forceinline__ double piv_rcp(double t) {
  double r = (double)__fdividef(1.0f, (float)t);
  r = fma(r, fma(-t, r, 1.0), r);
  return fma(r, fma(-t, r, 1.0), r);
}
// 1 / sqrt(t): the hardware reciprocal square root refined by Newton's step
// r <- r (3 - t r^2) / 2, once in FP32, twice (from the FP32 seed) in FP64.
__device__ __forceinline__ float piv_rsqrt(float t) {
  const float r = rsqrtf(t);
  return r * fmaf(-0.5f * t * r, r, 1.5f);
}
__device__ __forceinline__ double piv_rsqrt(double t) {
  double r = (double)rsqrtf((float)t);
  r = r * fma(-0.5 * t * r, r, 1.5);
  return r * fma(-0.5 * t * r, r, 1.5);
}

// Cholesky of a 32 x 32 diagonal block on one warp (Fig. ONFIG step (2)
// restricted to the block). Lane r holds row r of the block in w (w[j] =
// entry (r, j), meaningful for j <= r) and ends with row r of L (of F in
// deviation form, L = I + F); rd[c] = 1 / L_cc. The pivot of column c comes
// from lane c by a shuffle and the entries L_jc (j > c) of the rank-1 update
// from lanes j, so the 32 steps need no barrier. Entries above the diagonal
// are updated too and never read. thr: the pivot floor of column `lane`
// (plain form). Returns true when a pivot was not positive (singular S).
// Used by the blocked factorisation's diagonal kernel; the single-CTA
// kernel keeps its eight-warp column steps, which measured faster there
// (10.5K against 12.3K cycles per 32-column panel at m = 128: one warp
// issues all 31 - c shuffles of a step by itself).
template <typename Tm, bool dev>
__device__ __forceinline__ bool diag_factor_warp(Tm (&w)[32], Tm thr, Tm* rd) {
  const int lane = threadIdx.x & 31;
  bool b = false;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    Tm d = __shfl_sync(0xffffffffu, w[c], c);
    Tm rl;
    if (dev) {
      if (!(d > (Tm)-0.999)) {  // pivot 1 + d not positive
        b = true;
        d = (Tm)0;
      }
      rl = piv_rsqrt((Tm)1 + d);
    } else {
      if (!(d > __shfl_sync(0xffffffffu, thr, c))) {
        b = true;
        d = (Tm)1;
      }
      rl = piv_rsqrt(d);
    }
    const Tm l = lane > c ? w[c] * rl : w[c];  // L_rc for r > c
    if (lane == 0) rd[c] = rl;
    // L_cc (deviation form: L_cc - 1 = d / (1 + sqrt(1 + d)), with
    // sqrt(1 + d) = (1 + d) rl, which keeps small d accurate)
    w[c] = lane == c ? (dev ? d * piv_rcp((Tm)1 + ((Tm)1 + d) * rl) : d * rl)
                     : l;
#pragma unroll
    for (int j = c + 1; j < 32; ++j) w[j] -= l * __shfl_sync(0xffffffffu, l, j);
  }
  return b;
}

// X = L^{-1} of a 32 x 32 lower-triangular diagonal block (Fig. ONFIG step
// (3) restricted to the block): L in shared memory at B[i + k ldb], rd[i] =
// 1 / L_ii. Lane j forms column j of X in x by forward substitution,
// x_ij = (delta_ij - sum_{k=j}^{i-1} L_ik x_kj) / L_ii, with the column in
// registers and the rows of L read as broadcasts (x_kj = 0 for k < j, so
// the sums run over all k < i). Deviation form (L = I + F, X = I + Y):
// y_jj = -f_jj / (1 + f_jj), y_ij = -(f_ij + sum_k f_ik y_kj) / (1 + f_ii).
template <typename Tm, bool dev>
__device__ __forceinline__ void diag_inverse_warp(const Tm* B, int ldb,
                                                  const Tm* rd, Tm (&x)[32]) {
  const int j = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    Tm s0 = (dev && i > j) ? B[i + j * ldb] : (Tm)0, s1 = 0;
#pragma unroll
    for (int k = 0; k < i; ++k) {
      if (k & 1) s1 += B[i + k * ldb] * x[k];
      else s0 += B[i + k * ldb] * x[k];
    }
    const Tm r = rd[i];
    x[i] = i == j ? (dev ? -B[i + i * ldb] * r : r)
                  : (i > j ? -(s0 + s1) * r : (Tm)0);
  }
}

// 256 threads: the register-resident rows of the diagonal-block steps need
// more than the 128 registers a 512-thread CTA allows (they spilled, and
// the sequential pivot chain paid for it); the parallel phases lose less.
template <typename Tm>
constexpr int chol_threads() { return 256; }

// SM: the working copy lives in shared memory (a compile-time choice, so its
// accesses compile to shared-memory instructions), else in gwork.
template <typename Tm, bool dev, bool SM>
__global__ void __launch_bounds__(chol_threads<Tm>(), 1)
    k_chol_inv(int m, const double* __restrict__ S, const double* __restrict__ Bm,
               const double* __restrict__ Q, const float* __restrict__ Bf,
               const float* __restrict__ Qf, double* __restrict__ Linv,
               double* __restrict__ R, IterScalars* sc, Tm* gwork,
               const double* __restrict__ lpart, int nlpart) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  __shared__ Tm rdiag[1024];  // 1 / L_cc, all columns (mp <= 1024)
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int mp = (m + 31) & ~31, ld = mp + 1, P = mp >> 5;
  Tm* a = SM ? reinterpret_cast<Tm*>(smraw) : gwork;
  Tm* tb = a + (size_t)mp * ld;  // 32 x mp, leading dimension 33
  const Tm one = dev ? (Tm)1 : (Tm)0;
  const Tm eps = sizeof(Tm) == 4 ? (Tm)1.2e-7 : (Tm)2.3e-16;
  if (lpart) {  // the line step first (it sets sc->alpha)
    __shared__ double lred[4 * 32];
    line_alpha_block(m, lpart, nlpart, sc, lred);
    __syncthreads();
  }
  if (Bm || Bf) {
    // half of a (B + B^T) + a^2/2 (Q + Q^T) from each triangle, read in
    // column order (four loads of each matrix in flight per thread), then
    // the lower triangle adds its mirror. With FP32 copies of B and Q (Bf,
    // Qf) the FP32 factorisation does no FP64 work here.
    const double al = sc->alpha;
    const double hq = 0.5 * al * al;
    const float alf = (float)al, hqf = (float)hq;
    for (int k = warp; k < mp; k += nw)
      for (int i0 = lane; i0 < mp; i0 += 128) {
        Tm t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          const bool in = i < m && k < m;
          if (Bf)
            t[u] = in ? (Tm)(alf * Bf[i + k * m] + hqf * Qf[i + k * m]) : (Tm)0;
          else
            t[u] = in ? (Tm)(al * Bm[i + k * m] + hq * Q[i + k * m]) : (Tm)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i0 + 32 * u < mp) a[(i0 + 32 * u) + k * ld] = t[u];
      }
    __syncthreads();
    for (int k = warp; k < mp; k += nw)
      for (int i = k + lane; i < mp; i += 32)
        a[i + k * ld] = a[i + k * ld] + a[k + i * ld] +
                        ((!dev && i == k) ? (Tm)1 : (Tm)0);
  } else {
    for (int k = warp; k < mp; k += nw)
      for (int i = k + lane; i < mp; i += 32) {
        double v;
        if (i < m && k < m)
          v = S[i + k * m] - (dev && i == k ? 1.0 : 0.0);
        else
          v = (!dev && i == k) ? 1.0 : 0.0;
        a[i + k * ld] = (Tm)v;
      }
  }
  if (tid == 0) bad = 0;
  __syncthreads();

  for (int p = 0; p < P; ++p) {
    const int c0 = 32 * p;
    // (a) diagonal block on all eight warps: warp w keeps columns w, w + 8,
    // w + 16 and w + 24 of the block in registers (lane r = row c0 + r).
    // For column c the owning warp forms the pivot and publishes the column
    // through shared memory (two buffers, so one barrier per column); every
    // warp then updates its own later columns. Lanes above the diagonal
    // update too: those entries are never read.
    {
      __shared__ Tm colbuf[2][32];
      const int r = c0 + lane;
      Tm v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = a[r + (c0 + warp + 8 * q) * ld];
      bool b = false;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int q = c >> 3;
        if (warp == (c & 7)) {
          Tm d = __shfl_sync(0xffffffffu, v[q], c);
          // 1 / L_cc is all the column needs: rsqrt(1 + d) (rsqrt(d)) on the
          // pivot chain; L_cc itself is formed after the column is out
          Tm rl;
          if (dev) {
            if (!(d > (Tm)-0.999)) {  // pivot 1 + d not positive: singular S
              b = true;
              d = (Tm)0;
            }
            rl = piv_rsqrt((Tm)1 + d);
          } else {
            // a pivot that has lost all but 4m roundings of its original
            // diagonal entry marks a (numerically) singular S
            const int cc = c0 + c;
            const double sjj =
                (Bm || Bf || cc >= m) ? 1.0 : fabs(S[cc + cc * m]);
            if (!(d > (Tm)(4 * m) * eps * (Tm)sjj)) {
              b = true;
              d = (Tm)1;
            }
            rl = piv_rsqrt(d);
          }
          if (lane > c) v[q] *= rl;
          colbuf[c & 1][lane] = v[q];  // the diagonal entry is not read
          if (lane == 0) rdiag[c0 + c] = rl;
          // L_cc (deviation form: L_cc - 1 = d / (1 + sqrt(1 + d)), with
          // sqrt(1 + d) = (1 + d) rl, which keeps small d accurate)
          if (lane == c)
            v[q] = dev ? d * piv_rcp((Tm)1 + ((Tm)1 + d) * rl) : d * rl;
        }
        __syncthreads();
        const Tm lrc = colbuf[c & 1][lane];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          if (warp + 8 * qq > c) v[qq] -= lrc * colbuf[c & 1][warp + 8 * qq];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) a[r + (c0 + warp + 8 * q) * ld] = v[q];
      if (lane == 0 && b) bad = 1;
    }
    __syncthreads();
    // (b) rows below the block: x L_pp^T = a
    for (int r = c0 + 32 + tid; r < mp; r += nt) {
      Tm x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = a[r + (c0 + c) * ld];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        Tm s0 = x[c], s1 = 0;
#pragma unroll
        for (int k = 0; k < 31; k += 2) {
          if (k < c) s0 -= x[k] * a[(c0 + c) + (c0 + k) * ld];
          if (k + 1 < c) s1 -= x[k + 1] * a[(c0 + c) + (c0 + k + 1) * ld];
        }
        x[c] = (s0 + s1) * rdiag[c0 + c];
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) a[r + (c0 + c) * ld] = x[c];
    }
    __syncthreads();
    // (c) lower trailing triangle, 4 x 4 tiles
    const int base = c0 + 32;
    const int T = (mp - base) >> 2;
    const int ntile = T * (T + 1) / 2;
    for (int t = tid; t < ntile; t += nt) {
      int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
      while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
      while (ti * (ti + 1) / 2 > t) --ti;
      const int tj = t - ti * (ti + 1) / 2;
      const int r0 = base + 4 * ti, s0 = base + 4 * tj;
      Tm acc[4][4] = {};
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        Tm lr[4], ls[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          lr[u] = a[(r0 + u) + (c0 + k) * ld];
          ls[u] = a[(s0 + u) + (c0 + k) * ld];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += lr[u] * ls[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (r0 + u >= s0 + v) a[(r0 + u) + (s0 + v) * ld] -= acc[u][v];
    }
    __syncthreads();
  }

  // (d) inverse X = L_pp^{-1} of each diagonal block, one warp per block,
  // in place, row by row: lane j forms X_ij = (delta_ij - sum_{k=j}^{i-1}
  // L_ik X_kj) / L_ii from row i of L and its own column of X (rolled loops:
  // code run once per launch would stall on instruction fetch). In
  // deviation form (L = I + F, X = I + Y) the same recurrence reads
  // y_jj = -f_jj / (1 + f_jj) and, for i > j,
  // y_ij = -(f_ij + sum_{k=j}^{i-1} f_ik y_kj) / (1 + f_ii).
  for (int pb = warp; pb < P; pb += nw) {
    Tm* B = a + 32 * pb + (size_t)(32 * pb) * ld;  // block (i, k) at B[i + k ld]
    const Tm* rd = rdiag + 32 * pb;
    const int j = lane;
    for (int i = 0; i < 32; ++i) {
      Tm s0 = (dev && i > j) ? B[i + j * ld] : (Tm)0, s1 = 0;
      int k = j;
#pragma unroll 2
      for (; k + 1 < i; k += 2) {
        s0 += B[i + k * ld] * B[k + j * ld];
        s1 += B[i + (k + 1) * ld] * B[(k + 1) + j * ld];
      }
      if (k < i) s0 += B[i + k * ld] * B[k + j * ld];
      Tm x = 0;
      if (i == j) x = dev ? -B[i + i * ld] * rd[i] : rd[i];
      else if (i > j) x = -(s0 + s1) * rd[i];
      __syncwarp();  // row i of L is read by every lane before it is replaced
      if (i >= j) B[i + j * ld] = x;
      __syncwarp();
    }
  }
  __syncthreads();
  // (e) off-diagonal blocks, row-block by row-block: T = L_{i,0:i} X_{0:i,0:i}
  // (32 x ri, through tb), then X_{i,0:i} = -X_ii T; 4 x 4 register tiles.
  // Only the lower triangle of the working copy is read.
  for (int i = 1; i < P; ++i) {
    const int ri = 32 * i;
    const int nblk = 2 * ri;  // 8 row groups x ri/4 column groups
    for (int bq = tid; bq < nblk; bq += nt) {
      const int r0 = 4 * (bq & 7), cb = 4 * (bq >> 3);
      Tm acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)  // identity part of X (deviation form)
          acc[u][v] = dev ? a[(ri + r0 + u) + (cb + v) * ld] : (Tm)0;
#pragma unroll 4
      for (int col = cb; col < ri; ++col) {
        Tm lr[4], xc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) lr[u] = a[(ri + r0 + u) + col * ld];
#pragma unroll
        for (int v = 0; v < 4; ++v)
          xc[v] = col >= cb + v ? a[col + (cb + v) * ld] : (Tm)0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += lr[u] * xc[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) tb[(r0 + u) + (cb + v) * 33] = acc[u][v];
    }
    __syncthreads();
    for (int bq = tid; bq < nblk; bq += nt) {
      const int r0 = 4 * (bq & 7), cb = 4 * (bq >> 3);
      Tm acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          acc[u][v] = dev ? tb[(r0 + u) + (cb + v) * 33] : (Tm)0;
#pragma unroll 4
      for (int q = 0; q <= r0 + 3; ++q) {
        Tm xr[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          xr[u] = q <= r0 + u ? a[(ri + r0 + u) + (ri + q) * ld] : (Tm)0;
#pragma unroll
        for (int v = 0; v < 4; ++v) tv[v] = tb[q + (cb + v) * 33];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += xr[u] * tv[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) a[(ri + r0 + u) + (cb + v) * ld] = -acc[u][v];
    }
    __syncthreads();
  }
  const int isbad = bad;
  // Linv(i, k) column by column, then R(k, i) = Linv(i, k) column by column
  // (FP64 work only where it is needed: a conversion per lower-triangle
  // entry, the identity added on the diagonal alone)
  // (four entries per thread in flight; an FP64 conversion per
  // lower-triangle entry, the identity added on the diagonal alone)
  auto entry = [&](int i, int k) -> double {
    double v = 0.0;
    if (isbad) {
      if (i == k) v = 1.0;
    } else if (i >= k) {
      v = (double)a[i + k * ld];
      if (dev && i == k) v += 1.0;
    }
    return v;
  };
  for (int o = 0; o < (Linv ? 2 : 1); ++o) {
    double* out = o ? Linv : R;
    for (int k = warp; k < m; k += nw)  // column k of Linv, row k of R
      for (int i0 = lane; i0 < m; i0 += 128) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          v[u] = i < m ? (o ? entry(i, k) : entry(k, i)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          if (i < m) out[i + k * m] = v[u];
        }
      }
  }
  if (tid == 0 && isbad && sc) sc->status |= 1;
}

// ---------------------------------------------------------------------------
// Blocked Cholesky S = L L^T and L^{-1} on many CTAs, for large m (Fig. ONFIG
// steps (2), (3)): the same arithmetic as k_chol_inv, spread over launches.
// The padded working copy W (mp x mp, leading dimension mp, lower triangle)
// is factorised right-looking over 32-column panels: per panel p, one CTA
// factors the diagonal block and inverts it (k_cb_diag); then every lower
// tile (I, J) of the trailing matrix, on its own CTA, solves its two panel
// blocks against the diagonal block's inverse, L_Ip = A_Ip X_pp^T, and
// subtracts L_Ip L_Jp^T (k_cb_update); the diagonal tile's CTA stores L_Ip.
// L^{-1} = X follows by recursive doubling: for a diagonal block split as
// [A 0; B C], its inverse is [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}], so with the
// 32 x 32 inverses from k_cb_diag, levels of block size 32, 64, ... each form
// T = B A^{-1}, then X_CA = -C^{-1} T, for all blocks of the level at once
// (k_cb_inv). Deviation form (dev) as in k_chol_inv: W holds S - I, L = I + F
// and X = I + Y with the identities implicit, so FP32 arithmetic keeps L to
// FP64 accuracy relative to I when S is close to I.
// ---------------------------------------------------------------------------
constexpr int CB = 32;

// The line step alpha from the line-term partials (one CTA).
__global__ void k_cb_alpha(int m, const double* __restrict__ lpart, int nlpart,
                           IterScalars* sc) {
  __shared__ double lred[4 * 32];
  line_alpha_block(m, lpart, nlpart, sc, lred);
}

// W <- lower triangle of S, or of S(a) = I + a (B + B^T) + a^2 Q (Q
// symmetric), minus I in deviation form; the padding is the identity (zero
// in deviation form). Clears the failure flag.
template <typename Tm, bool dev>
__global__ void k_cb_form(int m, int mp, const double* __restrict__ S,
                          const double* __restrict__ Bm,
                          const double* __restrict__ Q,
                          const float* __restrict__ Bf,
                          const float* __restrict__ Qf,
                          const IterScalars* __restrict__ sc, Tm* __restrict__ W,
                          int* bad) {
  const int64_t total = (int64_t)mp * mp;
  if (blockIdx.x == 0 && threadIdx.x == 0) *bad = 0;
  const double al = (Bm || Bf) ? sc->alpha : 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), k = (int)(e / mp);
    if (i < k) continue;  // the upper triangle is never read
    double v;
    if (i < m && k < m) {
      // a (B + B^T) + a^2 (Q + Q^T) / 2, as k_chol_inv forms it
      if (Bf)
        v = (double)((float)al * (Bf[i + k * m] + Bf[k + i * m]) +
                     (float)(0.5 * al * al) * (Qf[i + k * m] + Qf[k + i * m]));
      else if (Bm)
        v = al * (Bm[i + (int64_t)k * m] + Bm[k + (int64_t)i * m]) +
            0.5 * al * al * (Q[i + (int64_t)k * m] + Q[k + (int64_t)i * m]);
      else
        v = S[i + (int64_t)k * m] - (dev && i == k ? 1.0 : 0.0);
      if ((Bm || Bf) && !dev && i == k) v += 1.0;
    } else {
      v = (!dev && i == k) ? 1.0 : 0.0;
    }
    W[e] = (Tm)v;
  }
}

// Factor and invert the 32 x 32 diagonal block of panel p: warp 0 runs
// diag_factor_warp and diag_inverse_warp; all 256 threads write the inverse.
// Writes the block of L (F in deviation form; zeros above the diagonal) and
// of X = L^{-1} (Y in deviation form).
template <typename Tm, bool dev>
__global__ void __launch_bounds__(256, 1)
    k_cb_diag(int m, int mp, int p, const double* __restrict__ S,
              bool from_S, const Tm* __restrict__ W, Tm* __restrict__ L,
              Tm* __restrict__ X, int* bad) {
  __shared__ Tm B[32 * 33];  // the block, column-major, leading dimension 33
  __shared__ Tm rd[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = CB * p, r = c0 + lane;
  const Tm eps = sizeof(Tm) == 4 ? (Tm)1.2e-7 : (Tm)2.3e-16;
  if (warp == 0) {
    Tm w[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) w[j] = W[r + (size_t)(c0 + j) * mp];
    Tm thr = (Tm)0;
    if (!dev) {
      const double sjj = (!from_S || r >= m) ? 1.0 : fabs(S[r + (int64_t)r * m]);
      thr = (Tm)(4 * m) * eps * (Tm)sjj;
    }
    const bool b = diag_factor_warp<Tm, dev>(w, thr, rd);
    // the block of L (lower, zeros above) to global and to shared memory
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const Tm x = lane >= j ? w[j] : (Tm)0;
      L[r + (size_t)(c0 + j) * mp] = x;
      B[lane + 33 * j] = x;
    }
    if (lane == 0 && b) atomicOr(bad, 1);
    __syncwarp();
    Tm x[32];
    diag_inverse_warp<Tm, dev>(B, 33, rd, x);
    __syncwarp();  // every lane has read L before the block is replaced
#pragma unroll
    for (int i = 0; i < 32; ++i) B[i + 33 * lane] = x[i];
  }
  __syncthreads();
  for (int e = tid; e < 32 * 32; e += 256) {
    const int i = e & 31, j = e >> 5;
    X[(c0 + i) + (size_t)(c0 + j) * mp] = i >= j ? B[i + 33 * j] : (Tm)0;
  }
}

// Trailing update of panel p: CTA t takes the lower tile (I, J), p < J <= I,
// of the trailing matrix. L_I = A_I X_pp^T (deviation form: A_I + A_I Y_pp^T)
// for the panel blocks of rows I and J, then W_IJ -= L_I L_J^T; the CTA of
// the diagonal tile writes L_I into L.
template <typename Tm, bool dev>
__global__ void __launch_bounds__(256)
    k_cb_update(int mp, int p, Tm* __restrict__ W, Tm* __restrict__ L,
                const Tm* __restrict__ X) {
  __shared__ Tm Xp[32][33], AI[32][33], AJ[32][33], LI[32][33], LJ[32][33];
  const int tid = threadIdx.x;
  const int P = mp / CB;
  // tile t -> (I, J), J <= I, counted over rows I = p + 1 .. P - 1
  const int t = blockIdx.x;
  int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  const int I = p + 1 + a, J = p + 1 + (t - a * (a + 1) / 2);
  if (I >= P) return;
  const int c0 = CB * p, i0 = CB * I, j0 = CB * J;
  for (int e = tid; e < 32 * 32; e += 256) {
    const int i = e & 31, k = e >> 5;
    Xp[i][k] = X[(c0 + i) + (size_t)(c0 + k) * mp];
    AI[i][k] = W[(i0 + i) + (size_t)(c0 + k) * mp];
    AJ[i][k] = W[(j0 + i) + (size_t)(c0 + k) * mp];
  }
  __syncthreads();
  const int r = tid & 31, cb = (tid >> 5) * 4;
  // L_I (and L_J) rows: L[r][c] = sum_{k <= c} A[r][k] X[c][k] (+ A[r][c])
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = cb + u;
    Tm sI = dev ? AI[r][c] : (Tm)0, sJ = dev ? AJ[r][c] : (Tm)0;
    for (int k = 0; k <= c; ++k) {
      sI += AI[r][k] * Xp[c][k];
      sJ += AJ[r][k] * Xp[c][k];
    }
    LI[r][c] = sI;
    LJ[r][c] = sJ;
  }
  __syncthreads();
  if (I == J)
    for (int e = tid; e < 32 * 32; e += 256) {
      const int i = e & 31, k = e >> 5;
      L[(i0 + i) + (size_t)(c0 + k) * mp] = LI[i][k];
    }
  // W_IJ -= L_I L_J^T: thread (r, cb..cb+3)
  Tm acc[4] = {0, 0, 0, 0};
#pragma unroll 8
  for (int k = 0; k < 32; ++k) {
    const Tm li = LI[r][k];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += li * LJ[cb + u][k];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const size_t o = (i0 + r) + (size_t)(j0 + cb + u) * mp;
    W[o] -= acc[u];
  }
}

// One level of the recursive inverse, block size s: pair q has A = rows and
// columns [2 q s, 2 q s + s) and C = [2 q s + s, 2 q s + 2 s) (cut at mp);
// phase 0: T_CA = L_CA X_A (deviation form: F_CA + F_CA Y_A), phase 1:
// X_CA = -X_C T_CA (deviation form: -(T + Y_C T)). One CTA per 32 x 32 tile
// of C x A (blockIdx.y), pairs along blockIdx.x.
template <typename Tm, bool dev>
__global__ void __launch_bounds__(256)
    k_cb_inv(int mp, int s, int phase, const Tm* __restrict__ L,
             Tm* __restrict__ X, Tm* __restrict__ T) {
  __shared__ Tm Ls[32][33], Rs[32][33];
  const int tid = threadIdx.x;
  const int a0 = 2 * s * blockIdx.x, c0 = a0 + s;
  if (c0 >= mp) return;
  const int nc = min(s, mp - c0);           // rows of C (multiple of 32)
  const int tiles_a = s / CB;
  const int ti = blockIdx.y / tiles_a, tj = blockIdx.y % tiles_a;
  if (CB * ti >= nc) return;
  const int gi = c0 + CB * ti, gj = a0 + CB * tj;  // output tile origin
  const int r = tid & 31, cb = (tid >> 5) * 4;
  Tm acc[4] = {0, 0, 0, 0};
  // phase 0: sum over k in A of L[gi.., k] X[k, gj..] (X_A lower: k >= gj)
  // phase 1: sum over k in C of X[gi.., k] T[k, gj..] (X_C lower: k <= gi+31)
  const int kb = phase == 0 ? gj : c0;
  const int ke = phase == 0 ? a0 + s : gi + CB;
  for (int k0 = kb; k0 < ke; k0 += CB) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int i = e & 31, k = e >> 5;
      if (phase == 0) {
        Ls[i][k] = L[(gi + i) + (size_t)(k0 + k) * mp];
        Rs[k][i] = X[(k0 + k) + (size_t)(gj + i) * mp];   // Rs[k][col]
      } else {
        Ls[i][k] = X[(gi + i) + (size_t)(k0 + k) * mp];
        Rs[k][i] = T[(k0 + k) + (size_t)(gj + i) * mp];
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const Tm l = Ls[r][k];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += l * Rs[k][cb + u];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const size_t o = (gi + r) + (size_t)(gj + cb + u) * mp;
    if (phase == 0)
      T[o] = acc[u] + (dev ? L[o] : (Tm)0);
    else
      X[o] = -(acc[u] + (dev ? T[o] : (Tm)0));
  }
}

// R = L^{-T} (upper) and Linv = L^{-1} (lower) in FP64 from X; identities
// and status bit 1 when a pivot failed.
template <typename Tm, bool dev>
__global__ void k_cb_out(int m, int mp, const Tm* __restrict__ X,
                         double* __restrict__ Linv, double* __restrict__ R,
                         const int* bad, IterScalars* sc) {
  const int isbad = *bad;
  const int64_t total = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), k = (int)(e / m);  // Linv(i, k) = R(k, i)
    double v = 0.0;
    if (isbad) {
      if (i == k) v = 1.0;
    } else if (i >= k) {
      v = (double)X[i + (size_t)k * mp];
      if (dev && i == k) v += 1.0;
    }
    if (Linv) Linv[e] = v;
    R[k + (int64_t)i * m] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && isbad && sc) sc->status |= 1;
}

// ---------------------------------------------------------------------------
// Line-model terms over 32 x 32 tiles of the (i, j) index space, one CTA of
// 1024 threads per tile, partial sums to part[tile * 4 + q]:
//   q = 0: tr(D1) = -tr(W)
//   q = 1: tr(D2) = tr(P^T H P) - sum_ij Q_ij A0_ij
//   q = 2: tr(S1 D1) = sum_ij A0_ij (B B^T - B^T B)_ij
//                      - 1/2 sum_ij S1_ij (W_ij + W_ji)
//   q = 3: tr(Q)
// with A0 = sym(H') + diag(H_D), S1 = B + B^T; tr(S1 (A0 B - B A0)) reduces
// to tr(A0 (B B^T - B^T B)) by cyclic invariance, so no m x m product is
// stored.
// ---------------------------------------------------------------------------
template <typename Tm, typename Tin>
__global__ void __launch_bounds__(1024)
    k_line_terms(int m, const Tin* __restrict__ Hp,
                 const double* __restrict__ HD, const Tin* __restrict__ Bm,
                 const Tin* __restrict__ Q, const double* __restrict__ hpd,
                 int hpd_stride, const double* __restrict__ tr_parts,
                 int n_tr_parts, const Tin* __restrict__ W,
                 double* __restrict__ part,
                 float* __restrict__ Bf, float* __restrict__ Qf) {
  __shared__ Tm t0[32][33], t1[32][33], t2[32][33], t3[32][33];
  __shared__ double red[4 * 32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int I0 = blockIdx.x * 32, J0 = blockIdx.y * 32;
  const int i = I0 + tx, j = J0 + ty;
  // blockIdx.z splits the k range of M = B B^T - B^T B; every other term is
  // added by the first split only (the sums are linear in M)
  const int ks = blockIdx.z, KS = gridDim.z;
  Tm M = 0;
  for (int k0 = 32 * ks; k0 < m; k0 += 32 * KS) {
    t0[tx][ty] = (I0 + tx < m && k0 + ty < m) ? (Tm)Bm[(I0 + tx) + (k0 + ty) * m] : (Tm)0;
    t1[tx][ty] = (J0 + tx < m && k0 + ty < m) ? (Tm)Bm[(J0 + tx) + (k0 + ty) * m] : (Tm)0;
    t2[tx][ty] = (k0 + tx < m && I0 + ty < m) ? (Tm)Bm[(k0 + tx) + (I0 + ty) * m] : (Tm)0;
    t3[tx][ty] = (k0 + tx < m && J0 + ty < m) ? (Tm)Bm[(k0 + tx) + (J0 + ty) * m] : (Tm)0;
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk)
      M += t0[tx][kk] * t1[ty][kk] - t2[kk][tx] * t3[kk][ty];
    __syncthreads();
  }
  // transposed tiles (J, I) of H', B, W for the (j, i) entries
  t0[tx][ty] = (J0 + tx < m && I0 + ty < m) ? (Tm)Hp[(J0 + tx) + (I0 + ty) * m] : (Tm)0;
  t1[tx][ty] = (J0 + tx < m && I0 + ty < m) ? (Tm)Bm[(J0 + tx) + (I0 + ty) * m] : (Tm)0;
  t2[tx][ty] = (J0 + tx < m && I0 + ty < m) ? (Tm)W[(J0 + tx) + (I0 + ty) * m] : (Tm)0;
  __syncthreads();
  Tm v0 = 0, v1 = 0, v2 = 0, v3 = 0;
  if (i < m && j < m) {
    const int e = i + j * m;
    const Tm a0 = (Tm)0.5 * ((Tm)Hp[e] + t0[ty][tx]) + (i == j ? (Tm)HD[i] : (Tm)0);
    v2 = a0 * M;
    if (ks == 0) {
      const Tm bij = (Tm)Bm[e], qij = (Tm)Q[e];
      if (Bf) {  // FP32 copies for the factorisation that follows
        Bf[e] = (float)bij;
        Qf[e] = (float)qij;
      }
      const Tm s1 = bij + t1[ty][tx];
      const Tm wij = (Tm)W[e], wji = t2[ty][tx];
      v2 -= (Tm)0.5 * s1 * (wij + wji);
      v1 = -qij * a0;
      if (i == j) {
        v0 = -wij;
        if (hpd) v1 += (Tm)hpd[(size_t)i * hpd_stride];
        v3 = (Tm)Q[e];
      }
    }
  }
  double v[4] = {(double)v0, (double)v1, (double)v2, (double)v3};
  if (tr_parts && ks == 0) {
    // tr(P^T H P) as the sum of the stencil's partial column dots, each
    // first-split CTA adding a fixed share
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    const int ncta = gridDim.x * gridDim.y;
    for (int k = cta * blockDim.x + threadIdx.x; k < n_tr_parts;
         k += ncta * blockDim.x)
      v[1] += tr_parts[k];
  }
  block_sum<4>(v, red);
  if (threadIdx.x == 0) {
    const size_t b =
        ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) part[b * 4 + q] = v[q];
  }
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi with the round-robin ordering: in each round m/2 disjoint
// (p, q) pairs are annihilated at once (columns, then rows, then Z). One CTA;
// A lives in shared memory (leading dimension m + 1) when it fits, else in
// the global work copy; Z accumulates in global memory, where its column
// updates are contiguous. T is the arithmetic type. Z starts from Z0 (FP64,
// may be null for the identity), so Z = Z0 J. A rotation is skipped when
// |a_pq| <= rot_tol (|a_pp| + |a_qq|) + abs_c ||A||_F (the second term sits
// above the rounding noise of the arithmetic type, so the sweeps end); they
// stop when one applied no rotation or the off-diagonal part is below
// conv_tol of the whole (squared Frobenius norms).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024)
    k_jacobi(int m, const double* __restrict__ Ain, T* __restrict__ Ag,
             T* __restrict__ Zw, const double* __restrict__ Z0,
             double* __restrict__ w, double* __restrict__ Z, int* info,
             int max_sweeps, T rot_tol, T abs_c, T conv_tol, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T cs[512], sn[512];
  __shared__ int pp[512], qq[512];
  __shared__ double red[2 * 32];
  __shared__ int done, rotated;
  __shared__ T abs_tol;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int ld = use_smem ? m + 1 : m;
  T* A = use_smem ? reinterpret_cast<T*>(smraw) : Ag;
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32) A[r + c * ld] = (T)Ain[r + c * m];
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32)
      Zw[r + c * m] = Z0 ? (T)Z0[r + c * m] : (r == c ? (T)1 : (T)0);
  const int M = m + (m & 1);
  const int np = M / 2;
  int sweeps = 0;
  if (tid == 0) rotated = 1;
  __syncthreads();
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double v[2] = {0.0, 0.0};
    for (int c = warp; c < m; c += nw)
      for (int r = lane; r < m; r += 32) {
        const double x = (double)A[r + c * ld];
        if (r == c)
          v[1] += x * x;
        else
          v[0] += x * x;
      }
    block_sum<2>(v, red);
    if (tid == 0) {
      done = (v[0] <= (double)conv_tol * (v[0] + v[1])) || !rotated ||
             sweep == max_sweeps;
      if (sweep == 0) abs_tol = (T)((double)abs_c * sqrt(v[0] + v[1]));
      rotated = 0;  // before the barrier: the rounds below may set it
    }
    __syncthreads();
    if (done) break;
    sweeps = sweep + 1;
    for (int r = 0; r < M - 1; ++r) {
      for (int k = tid; k < np; k += nt) {
        const int a0 = (k == 0) ? 0 : 1 + ((k - 1 + r) % (M - 1));
        const int kb = M - 1 - k;
        const int b0 = 1 + ((kb - 1 + r) % (M - 1));
        const int p = min(a0, b0), q = max(a0, b0);
        T c = 1, s = 0;
        if (q < m) {
          const T apq = A[p + q * ld];
          const T app = A[p + p * ld];
          const T aqq = A[q + q * ld];
          if (apq != (T)0 &&
              fabs(apq) > rot_tol * (fabs(app) + fabs(aqq)) + abs_tol) {
            const T th = (aqq - app) / ((T)2 * apq);
            T t;
            if (fabs(th) > (T)1e18)
              t = (T)0.5 / th;
            else
              t = (th >= (T)0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + (T)1));
            c = (T)1 / sqrt(t * t + (T)1);
            s = t * c;
            rotated = 1;
          }
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = min(q, m - 1);
      }
      __syncthreads();
      for (int k = warp; k < np; k += nw) {  // A <- A J (columns p, q)
        const T s = sn[k];
        if (s == (T)0) continue;
        const T c = cs[k];
        T* ap = A + pp[k] * ld;
        T* aq = A + qq[k] * ld;
        for (int i0 = lane; i0 < m; i0 += 128) {
          T x[4], y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + 32 * u;
            x[u] = i < m ? ap[i] : (T)0;
            y[u] = i < m ? aq[i] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + 32 * u;
            if (i < m) {
              ap[i] = c * x[u] - s * y[u];
              aq[i] = s * x[u] + c * y[u];
            }
          }
        }
      }
      __syncthreads();
      for (int k = warp; k < np; k += nw) {  // A <- J^T A (rows), Z <- Z J
        const T s = sn[k];
        if (s == (T)0) continue;
        const T c = cs[k];
        const int p = pp[k], q = qq[k];
        T* zp = Zw + p * m;
        T* zq = Zw + q * m;
        for (int j0 = lane; j0 < m; j0 += 128) {
          T x[4], y[4], u_[4], t_[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jc = j0 + 32 * u;
            x[u] = jc < m ? A[p + jc * ld] : (T)0;
            y[u] = jc < m ? A[q + jc * ld] : (T)0;
            u_[u] = jc < m ? zp[jc] : (T)0;
            t_[u] = jc < m ? zq[jc] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jc = j0 + 32 * u;
            if (jc < m) {
              A[p + jc * ld] = c * x[u] - s * y[u];
              A[q + jc * ld] = s * x[u] + c * y[u];
              zp[jc] = c * u_[u] - s * t_[u];
              zq[jc] = s * u_[u] + c * t_[u];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  // ascending order (stable on ties)
  for (int i = tid; i < m; i += nt) {
    const T wi = A[i + i * ld];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const T wj = A[j + j * ld];
      rank += (wj < wi) || (wj == wi && j < i);
    }
    w[rank] = (double)wi;
    for (int r = 0; r < m; ++r) Z[r + rank * m] = (double)Zw[r + i * m];
  }
  if (tid == 0 && info) *info = done ? sweeps : -1;
}

// ---------------------------------------------------------------------------
// One correction of an approximate eigenvector matrix X of a symmetric A, by
// the refinement of Ogita and Aishima (2018), derived to first order from
// (I + E)^T (X^T X) (I + E) = I and (I + E)^T (X^T A X) (I + E) diagonal:
// with R = I - X^T X and S = X^T A X,
//   lambda_i = s_ii / (1 - r_ii),
//   e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if the two are
//          further apart than delta = 2 (||S - diag(lambda)|| + ||A|| ||R||),
//   e_ij = r_ij / 2 otherwise, and also where the first-order step would
//          exceed 0.01 (inside a cluster only orthonormality is restored;
//          the closing FP64 Jacobi separates the cluster),
// and X <- X + X E. Frobenius norms stand for the 2-norms (a larger delta)
// and max |lambda_i| for ||A||. One CTA; G = X^T X, S = X^T A X in, E out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    k_refine_eig(int m, const double* __restrict__ G,
                 const double* __restrict__ S, double* __restrict__ E) {
  __shared__ double lam[1024];
  __shared__ double red[2 * 32];
  __shared__ unsigned long long amax;  // max |lambda| (bits of a double >= 0)
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) amax = 0ull;
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    lam[i] = S[i + (size_t)i * m] / G[i + (size_t)i * m];
    // non-negative doubles order like their bit patterns
    atomicMax(&amax, (unsigned long long)__double_as_longlong(fabs(lam[i])));
  }
  __syncthreads();
  double v[2] = {0.0, 0.0};  // ||S - D||^2, ||R||^2
  for (size_t e = tid; e < (size_t)m * m; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double r = (i == j ? 1.0 : 0.0) - G[e];
    const double d = S[e] - (i == j ? lam[i] : 0.0);
    v[0] += d * d;
    v[1] += r * r;
  }
  block_sum<2>(v, red);
  const double anorm = __longlong_as_double((long long)amax);
  const double delta = 2.0 * (sqrt(v[0]) + anorm * sqrt(v[1]));
  for (size_t e = tid; e < (size_t)m * m; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double r = (i == j ? 1.0 : 0.0) - G[e];
    const double dl = lam[j] - lam[i];
    const double num = S[e] + lam[j] * r;
    E[e] = (i != j && fabs(dl) > delta && fabs(num) <= 0.01 * fabs(dl))
               ? num / dl
               : 0.5 * r;
  }
}

}  // namespace

void mm_gemm(int m, const double* A, bool trA, const double* B, bool trB,
             double* Cm, double alpha, double beta, cudaStream_t s,
             bool fp32) {
  dim3 grid(ceil_div(m, 16), ceil_div(m, 16));
  if (fp32)
    k_mm_gemm<float><<<grid, 256, 0, s>>>(m, A, trA, B, trB, Cm, alpha, beta);
  else
    k_mm_gemm<double><<<grid, 256, 0, s>>>(m, A, trA, B, trB, Cm, alpha, beta);
  TRM_CHECK_LAUNCH();
}

void zero_diag(int m, double* A, cudaStream_t s, float* A32) {
  k_zero_diag<<<ceil_div(m, 256), 256, 0, s>>>(m, A, A32);
  TRM_CHECK_LAUNCH();
}

void make_A0(int m, const double* Hp, const double* HD, double* A0,
             cudaStream_t s) {
  k_make_A0<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, Hp, HD, A0);
  TRM_CHECK_LAUNCH();
}


// From this m on the factorisation runs blocked on many CTAs; the
// environment variable TRM_CHOL_BLOCKED_FROM, read once per process,
// overrides the default.
static int chol_blocked_from() {
  static const int v = [] {
    const char* e = std::getenv("TRM_CHOL_BLOCKED_FROM");
    const int d = 256;
    if (!e || !*e) return d;
    const long x = std::strtol(e, nullptr, 10);
    return x > 0 && x <= 4096 ? (int)x : d;
  }();
  return v;
}

// elements of the padded working copy plus the inverse's temporary (one
// CTA), or of W, L, X, T and the failure flag (blocked)
size_t chol_work_elems(int m) {
  const size_t mp = (size_t)((m + 31) & ~31);
  if (m >= chol_blocked_from()) return 4 * mp * mp + 8;
  return mp * (mp + 1) + 33 * mp;
}

template <typename Tm, bool dev>
static void chol_blocked(int m, const double* S, const double* Bm,
                         const double* Q, const float* Bf, const float* Qf,
                         double* Linv, double* R, IterScalars* sc,
                         double* gwork, cudaStream_t s, const double* lpart,
                         int nlpart) {
  const int mp = (m + 31) & ~31, P = mp / CB;
  const size_t mp2 = (size_t)mp * mp;
  Tm* W = reinterpret_cast<Tm*>(gwork);
  Tm* L = W + mp2;
  Tm* X = L + mp2;
  Tm* T = X + mp2;
  int* bad = reinterpret_cast<int*>(T + mp2);
  if (lpart) {
    k_cb_alpha<<<1, 256, 0, s>>>(m, lpart, nlpart, sc);
    TRM_CHECK_LAUNCH();
  }
  const int fb = (int)std::min<size_t>(ceil_div(mp2, (size_t)256), 1024);
  k_cb_form<Tm, dev><<<fb, 256, 0, s>>>(m, mp, S, Bm, Q, Bf, Qf, sc, W, bad);
  TRM_CHECK_LAUNCH();
  const bool from_S = S != nullptr && !Bm && !Bf;
  for (int p = 0; p < P; ++p) {
    k_cb_diag<Tm, dev><<<1, 256, 0, s>>>(m, mp, p, S, from_S, W, L, X, bad);
    TRM_CHECK_LAUNCH();
    const int t = P - p - 1;
    if (t > 0) {
      k_cb_update<Tm, dev><<<t * (t + 1) / 2, 256, 0, s>>>(mp, p, W, L, X);
      TRM_CHECK_LAUNCH();
    }
  }
  for (int sz = CB; sz < mp; sz *= 2) {
    const dim3 g(ceil_div(mp, 2 * sz), (sz / CB) * (sz / CB));
    k_cb_inv<Tm, dev><<<g, 256, 0, s>>>(mp, sz, 0, L, X, T);
    TRM_CHECK_LAUNCH();
    k_cb_inv<Tm, dev><<<g, 256, 0, s>>>(mp, sz, 1, L, X, T);
    TRM_CHECK_LAUNCH();
  }
  const int ob = (int)std::min<size_t>(ceil_div((size_t)m * m, (size_t)256), 1024);
  k_cb_out<Tm, dev><<<ob, 256, 0, s>>>(m, mp, X, Linv, R, bad, sc);
  TRM_CHECK_LAUNCH();
}

template <typename Tm, bool dev>
static void chol_launch(int m, const double* S, const double* Bm,
                        const double* Q, const float* Bf, const float* Qf,
                        double* Linv, double* R, IterScalars* sc,
                        double* gwork, cudaStream_t s,
                        const double* lpart = nullptr, int nlpart = 0) {
  if (m > 1024) throw Error(-1, "chol_inv: m > 1024");
  if (m >= chol_blocked_from()) {
    chol_blocked<Tm, dev>(m, S, Bm, Q, Bf, Qf, Linv, R, sc, gwork, s, lpart,
                          nlpart);
    return;
  }
  const size_t bytes = chol_work_elems(m) * sizeof(Tm);
  const bool smem = bytes <= 200 * 1024;
  if (smem) {
    static std::atomic<int> done[64] = {};  // per device; any thread may launch
    int dv = 0;
    cudaGetDevice(&dv);
    if (dv < 0 || dv >= 64 || !done[dv].load(std::memory_order_relaxed)) {
      TRM_CUDA(cudaFuncSetAttribute(k_chol_inv<Tm, dev, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
      if (dv >= 0 && dv < 64) done[dv].store(1, std::memory_order_relaxed);
    }
  }
  if (smem)
    k_chol_inv<Tm, dev, true><<<1, chol_threads<Tm>(), bytes, s>>>(
        m, S, Bm, Q, Bf, Qf, Linv, R, sc, nullptr, lpart, nlpart);
  else
    k_chol_inv<Tm, dev, false><<<1, chol_threads<Tm>(), 0, s>>>(
        m, S, Bm, Q, Bf, Qf, Linv, R, sc, reinterpret_cast<Tm*>(gwork), lpart,
        nlpart);
  TRM_CHECK_LAUNCH();
}

template <typename Tm>
void chol_inv(int m, const double* S, double* Linv, double* R, IterScalars* sc,
              double* gwork, cudaStream_t s) {
  chol_launch<Tm, false>(m, S, nullptr, nullptr, nullptr, nullptr, Linv, R,
                         sc, gwork, s);
}

template <typename Tm>
void chol_inv_dev(int m, const double* S, double* Linv, double* R,
                  IterScalars* sc, double* gwork, cudaStream_t s) {
  chol_launch<Tm, true>(m, S, nullptr, nullptr, nullptr, nullptr, Linv, R,
                        sc, gwork, s);
}

// k-splits of the line terms: about 64 CTAs when the m x m tiles are few
// (partials: 4 doubles per CTA, at most 4 ceil(m/32)^2 * 4 in all)
static int line_ksplit(int m) {
  const int t = ceil_div(m, 32);
  const int ks = std::min(std::min(t, 4), std::max(1, 64 / (t * t)));
  return std::max(1, ks);
}

template <typename Tm>
void line_factor(int m, const double* Hp, const double* HD, const double* Bm,
                 const double* Q, const double* hpd, int hpd_stride,
                 const double* tr_parts, int n_tr_parts, const double* W,
                 double* Linv, double* R, IterScalars* sc, double* gwork,
                 double* part, bool dev, cudaStream_t s) {
  const int t = ceil_div(m, 32);
  const int ksplit = line_ksplit(m);
  // FP32 factorisations take B and Q as FP32 copies written by the line
  // terms, placed after the factorisation's own FP32 working copy in gwork
  // (gwork holds max(2 m^2, chol_work_elems(m)) doubles)
  float* Bf = nullptr;
  float* Qf = nullptr;
  if (sizeof(Tm) == 4) {
    Bf = reinterpret_cast<float*>(gwork) + chol_work_elems(m);
    Qf = Bf + (size_t)m * m;
  }
  k_line_terms<Tm, double><<<dim3(t, t, ksplit), 1024, 0, s>>>(
      m, Hp, HD, Bm, Q, hpd, hpd_stride, tr_parts, n_tr_parts, W, part, Bf,
      Qf);
  TRM_CHECK_LAUNCH();
  // the factorisation kernel takes the line step from the partials first
  if (dev)
    chol_launch<Tm, true>(m, nullptr, Bm, Q, Bf, Qf, Linv, R, sc, gwork, s,
                          part, t * t * ksplit);
  else
    chol_launch<Tm, false>(m, nullptr, Bm, Q, Bf, Qf, Linv, R, sc, gwork, s,
                           part, t * t * ksplit);
}

// The FP32 path with the m x m inputs already in FP32 (copies the Gram sums
// write): no FP64 conversion in the line terms or the factorisation.
void line_factor32(int m, const float* Hp, const double* HD, const float* Bm,
                   const float* Q, const double* hpd, int hpd_stride,
                   const double* tr_parts, int n_tr_parts, const float* W,
                   double* Linv, double* R, IterScalars* sc, double* gwork,
                   double* part, cudaStream_t s) {
  const int t = ceil_div(m, 32);
  const int ksplit = line_ksplit(m);
  k_line_terms<float, float><<<dim3(t, t, ksplit), 1024, 0, s>>>(
      m, Hp, HD, Bm, Q, hpd, hpd_stride, tr_parts, n_tr_parts, W, part,
      nullptr, nullptr);
  TRM_CHECK_LAUNCH();
  chol_launch<float, true>(m, nullptr, nullptr, nullptr, Bm, Q, Linv, R, sc,
                           gwork, s, part, t * t * ksplit);
}

template void chol_inv_dev<float>(int, const double*, double*, double*,
                                  IterScalars*, double*, cudaStream_t);
template void chol_inv_dev<double>(int, const double*, double*, double*,
                                   IterScalars*, double*, cudaStream_t);
template void line_factor<float>(int, const double*, const double*,
                                 const double*, const double*, const double*,
                                 int, const double*, int, const double*,
                                 double*, double*, IterScalars*, double*,
                                 double*, bool, cudaStream_t);
template void line_factor<double>(int, const double*, const double*,
                                  const double*, const double*, const double*,
                                  int, const double*, int, const double*,
                                  double*, double*, IterScalars*, double*,
                                  double*, bool, cudaStream_t);

template <typename T>
static void jacobi_launch(int m, const double* A, const double* Z0, double* w,
                          double* Z, T* Aw, T* Zw, int* info, int max_sweeps,
                          T rot_tol, T abs_c, T conv_tol, cudaStream_t s) {
  const size_t bytes = (size_t)m * (m + 1) * sizeof(T);
  const bool smem = bytes <= 200 * 1024;
  if (smem) {
    static std::atomic<int> done[64] = {};  // per device; any thread may launch
    int dv = 0;
    cudaGetDevice(&dv);
    if (dv < 0 || dv >= 64 || !done[dv].load(std::memory_order_relaxed)) {
      TRM_CUDA(cudaFuncSetAttribute(k_jacobi<T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
      if (dv >= 0 && dv < 64) done[dv].store(1, std::memory_order_relaxed);
    }
  }
  k_jacobi<T><<<1, 1024, smem ? bytes : 0, s>>>(m, A, Aw, Zw, Z0, w, Z, info,
                                                max_sweeps, rot_tol, abs_c,
                                                conv_tol, smem ? 1 : 0);
  TRM_CHECK_LAUNCH();
}

size_t sym_eig_work_doubles(int m) { return (size_t)8 * m * m; }

// FP32 Jacobi sweeps (the FP64 pipe is 1/64 of the FP32 one); then twice:
// one FP64 refinement of the eigenvectors by matrix products on many CTAs,
// and four Newton-Schulz steps X <- X (3 I - X^T X) / 2 (the refinement is
// first order: where it splits close pairs it leaves X non-orthonormal by
// the square of its step, and X^T A X would then not be similar to A; the
// quadratically convergent steps bring that to FP64 rounding from up to
// ~0.1); then FP64 Jacobi on X^T A X, nearly diagonal, which rotates
// only the pairs still coupled above FP64 product noise (clusters) and
// accumulates onto X.
void sym_eig(int m, const double* A, double* w, double* Z, double* work,
             int* info, cudaStream_t s) {
  if (m > 1024) throw Error(-1, "sym_eig: m > 1024");
  const size_t mm = (size_t)m * m;
  double* X = work;
  double* T = work + mm;
  double* Sx = work + 2 * mm;
  double* G = work + 3 * mm;
  double* E = work + 4 * mm;
  double* Xn = work + 5 * mm;
  double* jw = work + 6 * mm;  // Jacobi work copies (2 m^2 of its type)
  // FP32 sweeps until no coupling above 4e-7 of its pair's diagonal plus
  // 1e-6 ||A||_F is left
  jacobi_launch<float>(m, A, nullptr, w, X, reinterpret_cast<float*>(jw),
                       reinterpret_cast<float*>(jw) + mm, info, 20, 4e-7f,
                       1e-6f, 0.0f, s);
  for (int it = 0; it < 2; ++it) {
    mm_gemm(m, A, false, X, false, T, 1.0, 0.0, s, false);   // A X
    mm_gemm(m, X, true, T, false, Sx, 1.0, 0.0, s, false);   // X^T A X
    mm_gemm(m, X, true, X, false, G, 1.0, 0.0, s, false);    // X^T X
    k_refine_eig<<<1, 1024, 0, s>>>(m, G, Sx, E);
    TRM_CHECK_LAUNCH();
    TRM_CUDA(cudaMemcpyAsync(Xn, X, mm * 8, cudaMemcpyDeviceToDevice, s));
    mm_gemm(m, X, false, E, false, Xn, 1.0, 1.0, s, false);  // X + X E
    std::swap(X, Xn);
    for (int ns = 0; ns < 4; ++ns) {
      mm_gemm(m, X, true, X, false, G, 1.0, 0.0, s, false);  // X^T X
      TRM_CUDA(cudaMemcpyAsync(Xn, X, mm * 8, cudaMemcpyDeviceToDevice, s));
      mm_gemm(m, X, false, G, false, Xn, -0.5, 1.5, s, false);  // 1.5 X - X G / 2
      std::swap(X, Xn);
    }
  }
  mm_gemm(m, A, false, X, false, T, 1.0, 0.0, s, false);
  mm_gemm(m, X, true, T, false, Sx, 1.0, 0.0, s, false);
  jacobi_launch<double>(m, Sx, X, w, Z, jw, jw + mm, info, 8, 1e-13, 1e-15,
                        0.0, s);
}

template void chol_inv<float>(int, const double*, double*, double*,
                              IterScalars*, double*, cudaStream_t);
template void chol_inv<double>(int, const double*, double*, double*,
                               IterScalars*, double*, cudaStream_t);

}  // namespace trm
