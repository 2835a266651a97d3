// Internal launcher declarations of the block-step kernels.
#pragma once

#include "common.cuh"

namespace trm {

// ---------------------------------------------------------------------------
// H operators (Eq. BASICEQ: sparse symmetric H with O(N) nonzeros)
// ---------------------------------------------------------------------------
struct StencilOp {
  int nx = 1, ny = 1, nz = 1;
  int radius = 1;            // 1: 3-point rule per axis, 2: 5-point rule
  double c1 = 0.0, c2 = 0.0; // coefficients of the +-1 and +-2 neighbours
  float c1h = 0.f, c1l = 0.f, c2h = 0.f, c2l = 0.f;  // the same as FP32 pairs
};

struct CsrOp {
  const int32_t* rowptr = nullptr;
  const int32_t* cols = nullptr;
  const float* vals32 = nullptr;
  const double* vals64 = nullptr;
  const float* valshi = nullptr;  // values as FP32 pairs (hi + lo)
  const float* valslo = nullptr;
  int max_row_nnz = 0;
};

struct Operator {
  int kind = 0;  // 0 stencil, 1 csr
  int64_t N = 0;
  StencilOp st;
  CsrOp csr;
  const double* diag64 = nullptr;  // H_ii
  const float* diag32 = nullptr;   // fl32(H_ii), the hi part of the pair
  const float* diaglo = nullptr;   // H_ii - fl32(H_ii)
  const double* minv64 = nullptr;  // diagonal preconditioner M_ii
  const float* minv32 = nullptr;
  int* err = nullptr;  // device status word: bit 2 when a bounded wait gave up
};

void apply_h(const Operator& op, const float* X, float* Y, int ncols,
             cudaStream_t s);
void apply_h(const Operator& op, const double* X, double* Y, int ncols,
             cudaStream_t s);
// FP32 Y = H X with the column dot products sum_i X_ic Y_ic of each CTA in
// dots[chunk * ncols + c] (apply_h_dots_doubles entries); returns the number
// of chunks (energy_from_dots adds them up). Y may be null: then only the
// dots are formed (the line model needs tr(P^T H P), not H P). (In FP64 the products would
// load the FP64 pipe the stencil is already bound by; energy_diag reads the
// two blocks instead.)
int apply_h_dots(const Operator& op, const float* X, float* Y, int ncols,
                 double* dots, cudaStream_t s);
size_t apply_h_dots_doubles(const Operator& op, int ncols);

// ---------------------------------------------------------------------------
// Double-float (FP32 pair, ~48-bit) arithmetic for the FP64-accuracy steps
// of MP2; a block is two arrays (hi, lo) of N x m floats.
// ---------------------------------------------------------------------------
void split_df(const double* x, float* hi, float* lo, int64_t n,
              cudaStream_t s);
void join_df(const float* hi, const float* lo, double* x, int64_t n,
             cudaStream_t s);
// X = H C in double-float (needs Operator::diaglo, and valshi/valslo for CSR)
void apply_h_df(const Operator& op, const float* Ch, const float* Cl,
                float* Xh, float* Xl, int ncols, cudaStream_t s);
// The same with the column dots sum_i C_ij X_ij of each CTA in
// dots[chunk * ncols + j] (apply_h_dots_doubles entries; energy_from_dots
// adds them up); returns the number of chunks, or 0 when this operator or
// these buffers take the unfused kernels (then nothing is launched).
int apply_h_df_dots(const Operator& op, const float* Ch, const float* Cl,
                    float* Xh, float* Xl, int ncols, double* dots,
                    cudaStream_t s);
// H_D[j] = sum_i C_ij X_ij, E = sum_j H_D[j] into sc->E
void energy_diag_df(int64_t N, int m, const float* Ch, const float* Cl,
                    const float* Xh, const float* Xl, double* HD,
                    IterScalars* sc, double* partials, cudaStream_t s);
// X32 = fl32(X - C diag(H_D))
void xprime_df(int64_t N, int m, const float* Ch, const float* Cl,
               const float* Xh, const float* Xl, const double* HD, float* X32,
               cudaStream_t s);

// diag[i] = t*w0*ndim + V[i] for a stencil operator
void stencil_diag(const StencilOp& st, double t_w0_ndim, const double* V,
                  double* diag64, float* diag32, int64_t N, cudaStream_t s);
// diag[i] = H_ii from a CSR matrix
void csr_diag(const Operator& op, double* diag64, float* diag32,
              cudaStream_t s);
// M_ii = 1 / (H_ii - sigma), sigma = min_k H_kk - 1; work: >= 1024 doubles
// Generalized problem: M_ii = 1 / (H_ii - sigma S_ii) with
// sigma = min_k H_kk / S_kk - 1 (S_ii > 0), so M is SPD; work: >= 256 doubles.
void diag_preconditioner_gen(const double* diagH, const double* diagS,
                             int64_t N, double* minv64, float* minv32,
                             double* work, cudaStream_t s);
void diag_preconditioner(const double* diag64, int64_t N, double* minv64,
                         float* minv32, double* work, cudaStream_t s);

// ---------------------------------------------------------------------------
// Gram products out = A^T [B_0 | B_1 | ...] (FP64 m x n, column-major)
// ---------------------------------------------------------------------------
template <typename T>
struct Blocks {
  const T* p[4] = {nullptr, nullptr, nullptr, nullptr};
  int cols = 0;   // columns per segment
  int count = 0;  // segments
  __host__ __device__ int total() const { return cols * count; }
};

size_t gram_partials_doubles(int64_t N, int m, int n);
// FP32 inputs go to the tensor-core kernel when gram_tc_eligible; err (device
// int, may be null) receives bit 2 if one of its bounded waits gave up;
// out32 (may be null) receives the result rounded to FP32 as well.
template <typename T>
void gram(int64_t N, int m, const T* A, const Blocks<T>& B, double* out,
          double* partials, size_t partials_cap, cudaStream_t s,
          int* err = nullptr, float* out32 = nullptr);
void sum_splits(const double* part, int splits, size_t count, double* out,
                cudaStream_t s);
// A^T B of FP64 blocks in double-float on the FP32 pipe (about 2^-46
// relative to sum |a||b|; see k_gram_df), for the mixed ladder's FP64-class
// steps.
void gram_df(int64_t N, int m, const double* A, const Blocks<double>& B,
             double* out, double* partials, size_t partials_cap,
             cudaStream_t s);
// A symmetric m x m output segment of which only the tiles on or above the
// diagonal were computed (seg < 0: none): an entry (i, j) of segment seg
// whose tile lies below the diagonal (i / tile > j / tile) takes the sum of
// entry (j, i).
struct SymSeg {
  int seg = -1;
  int m = 0, seg_cols = 0, tile = 0;
};
// the same for partials stored as FP32 pairs (hi, then lo, per split)
void sum_splits_pairs(const float* part, int splits, size_t count,
                      double* out, cudaStream_t s, float* out32 = nullptr,
                      SymSeg sym = SymSeg{});
// tcgen05 Gram of FP32 blocks (two-term TF32 split, three products, FP32
// accumulation in tensor memory): needs N % 4 == 0, m >= 32, A and every B
// segment 16-byte aligned (TMA), at most 4 B segments (each padded to whole
// 128-column tiles, its columns past the segment's width read as zeros).
bool gram_tc_eligible(int64_t N, int m, const float* A, const Blocks<float>& B);
// Segment k of the output is A_k^T B_k (A.count == B.count, or one A for all
// segments); up to four segments.
bool gram_tc_pairs_eligible(int64_t N, int m, const Blocks<float>& A,
                            const Blocks<float>& B);
// Doubles of split partials gram_tc / gram_tc_pairs need for an m x n result
// (skipped_tiles: tiles of a symmetric segment that are mirrored, not run).
size_t gram_tc_partials_doubles(int64_t N, int m, int n, int skipped_tiles = 0);
// sym_seg >= 0: that segment is symmetric (m x m); only its tiles on or
// above the diagonal are computed and the rest mirrored (Fig. DIVFIG).
// max_splits > 0 caps the row slices (a fixed partials buffer).
void gram_tc_pairs(int64_t N, int m, const Blocks<float>& A,
                   const Blocks<float>& B, double* out, double* partials,
                   size_t cap, int* err, cudaStream_t s,
                   float* out32 = nullptr, int sym_seg = -1,
                   int max_splits = 0);
void gram_tc(int64_t N, int m, const float* A, const Blocks<float>& B,
             double* out, double* partials, size_t cap, int* err,
             cudaStream_t s, float* out32 = nullptr, int max_splits = 0);

// Same product with the split partials in a caller-given scratch of
// scratch_doubles doubles (fewer row slices when it is small); m*n must fit.
template <typename T>
void gram_in_scratch(int64_t N, int m, const T* A, const Blocks<T>& B,
                     double* out, double* scratch, size_t scratch_doubles,
                     cudaStream_t s);

// ---------------------------------------------------------------------------
// Tall-skinny products and fused row-local updates
// ---------------------------------------------------------------------------
// H_D[j] = sum_i C_ij X_ij (FP64), E = sum_j H_D[j] into sc->E
template <typename T>
void energy_diag(int64_t N, int m, const T* C, const T* X, double* HD,
                 IterScalars* sc, double* partials, cudaStream_t s);
// H_D[j] = sum over chunks of dots (from apply_h_dots), E into sc->E
void energy_from_dots(const double* dots, int chunks, int m, double* HD,
                      IterScalars* sc, cudaStream_t s);
// X' = X - C diag(H_D), in place on X unless write_x is false; optional
// FP32 copies (MP2 phase)
template <typename T>
void xprime(int64_t N, int m, const T* C, T* X, const double* HD,
            float* C32, float* Xp32, cudaStream_t s, bool write_x = true);
// Workspace of the tensor-core block products Y M: the TF32 split of the
// small matrix M (mul_tc_work_floats floats) and the device error word of the
// bounded waits. A null TcWork (or member) selects the SIMT kernels.
struct TcWork {
  float* msplit = nullptr;
  size_t msplit_floats = 0;
  int* err = nullptr;
};
size_t mul_tc_work_floats(int k, int n);
// Y: N x k FP32 block, M: k x n; N % 4 == 0, N >= 128, k, n >= 32, 16-byte
// aligned blocks (checked by the callers).
bool mul_tc_eligible(int64_t N, int k, int n, const TcWork* tw);
// number of partial-sum records mul_tc_grad writes
int mul_tc_parts(int64_t N, int n);
// out = (A + alpha P) M (P may be null; alpha = sc->alpha) for an upper
// triangular M (the rotation's L^{-T}): column j of the product takes only
// the rows k <= j of M, whole 32-row K blocks of zeros are skipped. The
// split updates below make the same assumption of their R.
void mul_tc_store(int64_t N, int k, int n, const float* A, const float* P,
                  const IterScalars* sc, const double* M, float* out,
                  const TcWork& tw, cudaStream_t s);
// G = -2 (X' - C H') with the four Polak-Ribiere partial sums per CTA in
// part; the last CTA to finish forms the CG scalars in sc (cg_scalars).
// Returns the number of records.
int mul_tc_grad(int64_t N, int m, const float* C, const double* Hp,
                const float* Xp, float* G, const float* Gprev,
                const float* Pprev, const float* minv, double* part,
                IterScalars* sc, const TcWork& tw, cudaStream_t s);
// Cn = (C64 + alpha P) diag(R) + (C32 + alpha P) (R - diag(R))
void mul_tc_split64(int64_t N, int m, const float* C32, const float* P,
                    const double* C64, const IterScalars* sc, const double* R,
                    double* Cn, const TcWork& tw, cudaStream_t s);
// The same with C and Cn as FP32 pairs (C32 = Ch): Y = C + alpha P and
// Y diag(R) in double-float, plus the tensor-core product
void mul_tc_splitdf(int64_t N, int m, const float* Ch, const float* Cl,
                    const float* P, const IterScalars* sc, const double* R,
                    float* Cnh, float* Cnl, const TcWork& tw, cudaStream_t s);

// G = -2 (X' - C H') with the Polak-Ribiere partial sums; G_prev/P_prev may
// be null (first iteration). Then the device scalar update of gamma, r.
// FP32 blocks use the tensor cores when tw allows.
template <typename T>
void gradient(int64_t N, int m, const T* C, const T* Xp, const double* Hp,
              T* G, const T* Gprev, const T* Pprev, const T* minv,
              IterScalars* sc, double* partials, size_t partials_cap,
              cudaStream_t s, const TcWork* tw = nullptr);
// P = M G + gamma P (gamma from sc)
template <typename T>
void update_p(int64_t N, int m, const T* G, T* P, const T* minv,
              const IterScalars* sc, cudaStream_t s);
// Cn = (C + alpha P) R, R upper triangular m x m FP64 (alpha from sc, or 0
// when P is null)
template <typename T, typename TP>
void rotate(int64_t N, int m, const T* C, const TP* P, const double* R,
            T* Cn, const IterScalars* sc, cudaStream_t s,
            const TcWork* tw = nullptr);
// MP1 (ii): Cn = Y L_D + fl32(Y) L', Y = C + alpha P; R = L^{-T} FP64.
// With C32 = fl32(C) and tw, fl32(Y) is formed as C32 + alpha P in FP32 and
// the product runs on the tensor cores.
void rotate_split(int64_t N, int m, const double* C, const float* P,
                  const double* R, double* Cn, const IterScalars* sc,
                  cudaStream_t s, const float* C32 = nullptr,
                  const TcWork* tw = nullptr);
// The split update with C and Cn as FP32 pairs (hi, lo): the FP32 operand
// is Ch + alpha P, Y diag(R) is formed in double-float
void rotate_split_df(int64_t N, int m, const float* Ch, const float* Cl,
                     const float* P, const double* R, float* Cnh, float* Cnl,
                     const IterScalars* sc, cudaStream_t s,
                     const TcWork* tw = nullptr);
// out = a X + b Y elementwise over n FP64 values (out may alias X or Y)
void lin_comb(int64_t n, double a, const double* X, double b, const double* Y,
              double* out, cudaStream_t s);
// Y = A M for A: N x k (FP64), M: k x n FP64
void mult(int64_t N, int k, int n, const double* A, const double* M,
          double* Y, cudaStream_t s);
// The same in double-float on the FP32 pipe (about 2^-46 relative; the
// mixed ladder's FP64-class steps); upper_tri: M is upper triangular (k = n)
void mult_df(int64_t N, int k, int n, const double* A, const double* M,
             double* Y, bool upper_tri, cudaStream_t s);
// per-column 2-norms of X - C diag(lambda) into res (FP64 device m)
void column_residuals(int64_t N, int m, const double* X, const double* C,
                      const double* lam, double* res, double* partials,
                      cudaStream_t s);
// flip each column's sign so its largest-magnitude entry is positive,
// applied to C and X together
void fix_signs(int64_t N, int m, double* C, double* X, double* work,
               cudaStream_t s);
void to_f32(const double* x, float* y, int64_t n, cudaStream_t s);
void to_f64(const float* x, double* y, int64_t n, cudaStream_t s);
void random_block(int64_t N, int m, uint64_t seed, double* C, cudaStream_t s);

// ---------------------------------------------------------------------------
// m x m FP64 matrices on the device
// ---------------------------------------------------------------------------
// Cm = alpha op(A) op(B) + beta Cm (all m x m FP64, column-major)
// (fp32: products and sums in FP32, inputs and outputs FP64)
void mm_gemm(int m, const double* A, bool trA, const double* B, bool trB,
             double* Cm, double alpha, double beta, cudaStream_t s,
             bool fp32 = false);
// A0 = sym(H') + diag(H_D)
void make_A0(int m, const double* Hp, const double* HD, double* A0,
             cudaStream_t s);
// The line step along P and the factor of the new overlap: the line-model
// terms from H' (diag zeroed), H_D, B = C^T P, Q = P^T P, the trace of
// P^T H P and W = P^T G give alpha (into sc); then S = I + a (B + B^T) +
// a^2 Q is factorised (in deviation form when dev) into Linv (may be null)
// and R = L^{-T}. The trace comes from the diagonal hpd[j * hpd_stride] (the
// matrix P^T H P with stride m + 1), or, when hpd is null, as the sum of the
// n_tr_parts partial column dots in tr_parts (the stencil applied to P).
// part: >= 16 * ceil(m/32)^2 doubles; gwork: max(2 m^2, chol_work_elems(m))
// doubles (FP32 factorisations keep FP32 copies of B and Q there).
template <typename Tm>
void line_factor(int m, const double* Hp, const double* HD, const double* Bm,
                 const double* Q, const double* hpd, int hpd_stride,
                 const double* tr_parts, int n_tr_parts, const double* W,
                 double* Linv, double* R, IterScalars* sc, double* gwork,
                 double* part, bool dev, cudaStream_t s);
// line_factor<float> with the m x m inputs given in FP32 (Gram copies)
void line_factor32(int m, const float* Hp, const double* HD, const float* Bm,
                   const float* Q, const double* hpd, int hpd_stride,
                   const double* tr_parts, int n_tr_parts, const float* W,
                   double* Linv, double* R, IterScalars* sc, double* gwork,
                   double* part, cudaStream_t s);
// Elements (of the arithmetic type) of the factorisation workspace gwork.
size_t chol_work_elems(int m);
// S = L L^T (lower); writes Linv = L^{-1} (unless null) and R = L^{-T}. Non-PD sets
// sc->status bit 1 and returns identities. gwork: chol_work_elems(m)
// doubles (used when the working copy does not fit in shared memory).
template <typename Tm>
void chol_inv(int m, const double* S, double* Linv, double* R,
              IterScalars* sc, double* gwork, cudaStream_t s);
// The same for S close to I, in deviation form (L = I + F, L^{-1} = I + Y):
// FP32 arithmetic on the small parts gives FP64 accuracy relative to I.
template <typename Tm>
void chol_inv_dev(int m, const double* S, double* Linv, double* R,
                  IterScalars* sc, double* gwork, cudaStream_t s);
// set diagonal of an m x m matrix (and of its FP32 copy A32, may be null)
// to zero
void zero_diag(int m, double* A, cudaStream_t s, float* A32 = nullptr);
// symmetric eigenproblem A = Z diag(w) Z^T to FP64 accuracy (FP32 cyclic
// Jacobi, FP64 refinement of the eigenvectors, FP64 Jacobi on the refined
// projection), w ascending; work: sym_eig_work_doubles(m); info (device
// int): sweeps of the closing FP64 Jacobi, or -1
size_t sym_eig_work_doubles(int m);
void sym_eig(int m, const double* A, double* w, double* Z, double* work,
             int* info, cudaStream_t s);
// U = M (M^T M)^{-1/2}, the orthogonal factor of the polar decomposition
// of M (m x m FP64): the orthogonal U minimising ||A U - B||_F when
// M = A^T B. M^T M = Z diag(w) Z^T by sym_eig; an eigenvalue at or below
// 1e-12 of the largest sets *status bit 1. work: polar_work_doubles(m);
// info as sym_eig's.
size_t polar_work_doubles(int m);
void polar_factor(int m, const double* M, double* U, double* work, int* status,
                  int* info, cudaStream_t s);

}  // namespace trm
