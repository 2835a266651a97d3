// m x m matrix work on the device: products, the line model along P,
// Cholesky factorisation and triangular inverse (Fig. ONFIG steps (2), (3)),
// and the symmetric eigenproblem of the closing Rayleigh-Ritz step
// (Sec. 2.1: "diagonalization of H ... will give the explicit eigenvalues").
// All matrices are column-major with leading dimension m and stored as FP64;
// the template parameter Tm is the arithmetic type.
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

__global__ void k_zero_diag(int m, double* A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) A[i + (int64_t)i * m] = 0.0;
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
//   E(a) - E(0) = a tr(D1) + a^2 (tr(D2) - tr(S1 D1)),
// and the step is the minimiser of that parabola, bounded so that the RMS
// column change a ||P||_F / sqrt(m) stays below 1.
// ---------------------------------------------------------------------------
template <typename Tm>
__global__ void __launch_bounds__(1024)
    k_line_step(int m, const double* __restrict__ A0,
                const double* __restrict__ Bm, const double* __restrict__ Q,
                const double* __restrict__ HPP, const double* __restrict__ W,
                const double* __restrict__ T1, const double* __restrict__ T2,
                double* __restrict__ S, IterScalars* sc) {
  __shared__ double red[4 * 32];
  __shared__ double alpha_sh;
  Tm trD1 = 0, trD2 = 0, trS1D1 = 0, trQ = 0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = threadIdx.x >> 5; j < m; j += nw)
  for (int i = lane; i < m; i += 32) {
    const int e = i + j * m;
    const int et = j + i * m;  // (j, i)
    const Tm s1 = (Tm)Bm[e] + (Tm)Bm[et];   // S1_ij
    // D1_ji = T1_ji - T2_ji - (W_ji + W_ij)/2
    const Tm d1ji = (Tm)T1[et] - (Tm)T2[et] - (Tm)0.5 * ((Tm)W[et] + (Tm)W[e]);
    trS1D1 += s1 * d1ji;
    trD2 -= (Tm)Q[e] * (Tm)A0[e];
    if (i == j) {
      trD1 -= (Tm)W[e];
      trD2 += (Tm)HPP[e];
      trQ += (Tm)Q[e];
    }
  }
  double v[4] = {(double)trD1, (double)trD2, (double)trS1D1, (double)trQ};
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
    alpha_sh = alpha;
  }
  __syncthreads();
  const double a = alpha_sh;
  for (int j = threadIdx.x >> 5; j < m; j += nw)
  for (int i = lane; i < m; i += 32) {
    const int e = i + j * m;
    const int et = j + i * m;
    const double s1 = Bm[e] + Bm[et];
    const double q = 0.5 * (Q[e] + Q[et]);
    S[e] = (i == j ? 1.0 : 0.0) + a * s1 + a * a * q;
  }
}

// ---------------------------------------------------------------------------
// Cholesky S = L L^T (right-looking, lower) and L^{-1} in place (backward
// column sweep: col j of L^{-1} below the diagonal is -(L22^{-1} l) / l_jj).
// Writes Linv (lower) and R = L^{-T} (upper). One CTA of 1024 threads; the
// working copy has leading dimension m + 1 so that a warp walking along a
// row touches 32 distinct banks.
//
// With dev = true the matrix is S = I + E and the factorisation runs in
// deviation form: L = I + F and L^{-1} = I + Y with the identity kept exact
// and only the small E, F, Y held in Tm. Pivot j: d = E_jj - sum_k F_jk^2,
// f_jj = d / (1 + sqrt(1 + d)); below it F_ij = (E_ij - sum_k F_ik F_jk) /
// (1 + f_jj). Inverse: y_jj = -f_jj / (1 + f_jj), and the column below is
// -(1 + y_jj) (x + Y22 x) with x = F[j+1:, j]. When S - I is small, FP32
// arithmetic here yields L to FP64 accuracy relative to I.
// ---------------------------------------------------------------------------
template <typename Tm, bool dev>
__global__ void __launch_bounds__(1024)
    k_chol_inv(int m, const double* __restrict__ S, double* __restrict__ Linv,
               double* __restrict__ R, IterScalars* sc, Tm* gwork,
               int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  __shared__ Tm tmp[1024];
  Tm* a = use_smem ? reinterpret_cast<Tm*>(smraw) : gwork;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int ld = m + 1;
  const Tm eps = sizeof(Tm) == 4 ? (Tm)1.2e-7 : (Tm)2.3e-16;
  for (int k = warp; k < m; k += nw)
    for (int i = lane; i < m; i += 32)
      a[i + k * ld] = (Tm)(S[i + k * m] - (dev && i == k ? 1.0 : 0.0));
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      Tm d = a[j + j * ld];
      if (dev) {
        if (!(d > (Tm)-0.999)) {  // pivot 1 + d not positive: singular S
          bad = 1;
          d = (Tm)0;
        }
        a[j + j * ld] = d / ((Tm)1 + sqrt((Tm)1 + d));
      } else {
        // a pivot that has lost all but 4m roundings of its original
        // diagonal entry marks a (numerically) singular S
        const Tm floor_j = (Tm)(4 * m) * eps * (Tm)fabs(S[j + j * m]);
        if (!(d > floor_j)) {
          bad = 1;
          d = (Tm)1;
        }
        a[j + j * ld] = sqrt(d);
      }
    }
    __syncthreads();
    const Tm ljj = (dev ? (Tm)1 : (Tm)0) + a[j + j * ld];
    for (int i = j + 1 + tid; i < m; i += nt) a[i + j * ld] /= ljj;
    __syncthreads();
    // trailing update of the lower triangle: a warp per column, lanes down
    for (int k = j + 1 + warp; k < m; k += nw) {
      const Tm lkj = a[k + j * ld];
      for (int i = k + lane; i < m; i += 32) a[i + k * ld] -= a[i + j * ld] * lkj;
    }
    __syncthreads();
  }
  for (int j = m - 1; j >= 0; --j) {
    if (tid == 0) {
      const Tm f = a[j + j * ld];
      a[j + j * ld] = dev ? -f / ((Tm)1 + f) : (Tm)1 / f;
    }
    for (int i = j + 1 + tid; i < m; i += nt) tmp[i] = a[i + j * ld];
    __syncthreads();
    const Tm scale = dev ? -((Tm)1 + a[j + j * ld]) : -a[j + j * ld];
    // row i of the already inverted trailing block times the column below
    // the pivot: one warp per row, lanes along k
    for (int i = j + 1 + warp; i < m; i += nw) {
      Tm y = 0;
      for (int k = j + 1 + lane; k <= i; k += 32) y += a[i + k * ld] * tmp[k];
      y = warp_sum(y);
      if (lane == 0) a[i + j * ld] = scale * ((dev ? tmp[i] : (Tm)0) + y);
    }
    __syncthreads();
  }
  const int isbad = bad;
  for (int k = warp; k < m; k += nw) {
    for (int i = lane; i < m; i += 32) {
      double v;
      if (isbad)
        v = (i == k) ? 1.0 : 0.0;
      else
        v = (dev && i == k ? 1.0 : 0.0) + (i >= k ? (double)a[i + k * ld] : 0.0);
      Linv[i + k * m] = v;  // Linv(i, k)
      R[k + i * m] = v;     // R(k, i) = Linv(i, k)
    }
  }
  if (tid == 0 && isbad && sc) sc->status |= 1;
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi with the round-robin ordering: in each round m/2 disjoint
// (p, q) pairs are annihilated at once (columns, then rows, then Z).
// A (work, overwritten) and Zw are in global memory; one CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    k_jacobi(int m, double* __restrict__ A, double* __restrict__ Zw,
             double* __restrict__ w, double* __restrict__ Z, int* info,
             int max_sweeps) {
  __shared__ double cs[512], sn[512];
  __shared__ int pp[512], qq[512];
  __shared__ double red[2 * 32];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, nw = nt >> 5;
  for (int c = tid >> 5; c < m; c += nw)
    for (int r = lane; r < m; r += 32) Zw[r + c * m] = (r == c) ? 1.0 : 0.0;
  const int M = m + (m & 1);
  const int np = M / 2;
  int sweeps = 0;
  __syncthreads();
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double v[2] = {0.0, 0.0};
    for (int c = tid >> 5; c < m; c += nw)
      for (int r = lane; r < m; r += 32) {
        const double x = A[r + c * m];
        if (r == c)
          v[1] += x * x;
        else
          v[0] += x * x;
      }
    block_sum<2>(v, red);
    if (tid == 0) done = (v[0] <= 1e-30 * (v[0] + v[1])) || sweep == max_sweeps;
    __syncthreads();
    if (done) break;
    sweeps = sweep + 1;
    for (int r = 0; r < M - 1; ++r) {
      for (int k = tid; k < np; k += nt) {
        const int a0 = (k == 0) ? 0 : 1 + ((k - 1 + r) % (M - 1));
        const int kb = M - 1 - k;
        const int b0 = 1 + ((kb - 1 + r) % (M - 1));
        const int p = min(a0, b0), q = max(a0, b0);
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p + (int64_t)q * m];
          const double app = A[p + (int64_t)p * m];
          const double aqq = A[q + (int64_t)q * m];
          if (fabs(apq) > 1e-300 &&
              fabs(apq) > 1e-18 * (fabs(app) + fabs(aqq))) {
            const double th = (aqq - app) / (2.0 * apq);
            double t;
            if (fabs(th) > 1e150)
              t = 0.5 / th;
            else
              t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = min(q, m - 1);
      }
      __syncthreads();
      for (int k = tid >> 5; k < np; k += nw) {  // A <- A J
        const double s = sn[k];
        if (s == 0.0) continue;
        const double c = cs[k];
        double* ap = A + pp[k] * m;
        double* aq = A + qq[k] * m;
        for (int i = lane; i < m; i += 32) {
          const double x = ap[i], y = aq[i];
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
        }
      }
      __syncthreads();
      for (int k = tid >> 5; k < np; k += nw) {  // A <- J^T A, Z <- Z J
        const double s = sn[k];
        if (s == 0.0) continue;
        const double c = cs[k];
        const int p = pp[k], q = qq[k];
        for (int jc = lane; jc < m; jc += 32) {
          const double x = A[p + jc * m], y = A[q + jc * m];
          A[p + jc * m] = c * x - s * y;
          A[q + jc * m] = s * x + c * y;
        }
        double* zp = Zw + p * m;
        double* zq = Zw + q * m;
        for (int jc = lane; jc < m; jc += 32) {
          const double u = zp[jc], t = zq[jc];
          zp[jc] = c * u - s * t;
          zq[jc] = s * u + c * t;
        }
      }
      __syncthreads();
    }
  }
  // ascending order (stable on ties)
  for (int i = tid; i < m; i += nt) {
    const double wi = A[i + (int64_t)i * m];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double wj = A[j + (int64_t)j * m];
      rank += (wj < wi) || (wj == wi && j < i);
    }
    w[rank] = wi;
    for (int r = 0; r < m; ++r) Z[r + (int64_t)rank * m] = Zw[r + (int64_t)i * m];
  }
  if (tid == 0 && info) *info = done ? sweeps : -1;
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

void zero_diag(int m, double* A, cudaStream_t s) {
  k_zero_diag<<<ceil_div(m, 256), 256, 0, s>>>(m, A);
  TRM_CHECK_LAUNCH();
}

void make_A0(int m, const double* Hp, const double* HD, double* A0,
             cudaStream_t s) {
  k_make_A0<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, Hp, HD, A0);
  TRM_CHECK_LAUNCH();
}

template <typename Tm>
void line_step(int m, const double* A0, const double* Bm, const double* Q,
               const double* HPP, const double* W, const double* T1,
               const double* T2, double* S, IterScalars* sc, cudaStream_t s) {
  k_line_step<Tm><<<1, 1024, 0, s>>>(m, A0, Bm, Q, HPP, W, T1, T2, S, sc);
  TRM_CHECK_LAUNCH();
}

template <typename Tm, bool dev>
static void chol_launch(int m, const double* S, double* Linv, double* R,
                        IterScalars* sc, double* gwork, cudaStream_t s) {
  if (m > 1024) throw Error(-1, "chol_inv: m > 1024");
  const size_t bytes = (size_t)m * (m + 1) * sizeof(Tm);
  const bool smem = bytes <= 200 * 1024;
  if (smem) {
    TRM_CUDA(cudaFuncSetAttribute(k_chol_inv<Tm, dev>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes));
  }
  k_chol_inv<Tm, dev><<<1, 1024, smem ? bytes : 0, s>>>(
      m, S, Linv, R, sc, reinterpret_cast<Tm*>(gwork), smem ? 1 : 0);
  TRM_CHECK_LAUNCH();
}

template <typename Tm>
void chol_inv(int m, const double* S, double* Linv, double* R, IterScalars* sc,
              double* gwork, cudaStream_t s) {
  chol_launch<Tm, false>(m, S, Linv, R, sc, gwork, s);
}

template <typename Tm>
void chol_inv_dev(int m, const double* S, double* Linv, double* R,
                  IterScalars* sc, double* gwork, cudaStream_t s) {
  chol_launch<Tm, true>(m, S, Linv, R, sc, gwork, s);
}

template void chol_inv_dev<float>(int, const double*, double*, double*,
                                  IterScalars*, double*, cudaStream_t);
template void chol_inv_dev<double>(int, const double*, double*, double*,
                                   IterScalars*, double*, cudaStream_t);

void sym_eig(int m, const double* A, double* w, double* Z, double* work,
             int* info, cudaStream_t s) {
  if (m > 1024) throw Error(-1, "sym_eig: m > 1024");
  double* Aw = work;
  double* Zw = work + (size_t)m * m;
  TRM_CUDA(cudaMemcpyAsync(Aw, A, sizeof(double) * m * m,
                           cudaMemcpyDeviceToDevice, s));
  k_jacobi<<<1, 1024, 0, s>>>(m, Aw, Zw, w, Z, info, 40);
  TRM_CHECK_LAUNCH();
}

template void line_step<float>(int, const double*, const double*,
                               const double*, const double*, const double*,
                               const double*, const double*, double*,
                               IterScalars*, cudaStream_t);
template void line_step<double>(int, const double*, const double*,
                                const double*, const double*, const double*,
                                const double*, const double*, double*,
                                IterScalars*, cudaStream_t);
template void chol_inv<float>(int, const double*, double*, double*,
                              IterScalars*, double*, cudaStream_t);
template void chol_inv<double>(int, const double*, double*, double*,
                               IterScalars*, double*, cudaStream_t);

}  // namespace trm
