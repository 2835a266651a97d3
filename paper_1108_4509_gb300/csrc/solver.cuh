// Host-side solver state and the per-iteration block step (internal).
#pragma once

#include <vector>

#include "../../include/trm.h"
#include "ops.cuh"

namespace trm {

// Per-class timing of the library's launches with CUDA events on the solver's
// stream, plus the algorithmic flops and bytes of each launch, for roofline
// reporting. Off unless enabled; event pairs are resolved after a solve.
// Each class is one kernel family, so that a kernel's DRAM counters apply
// to its class alone: spmm_df and rotate_df are MP2's double-float H C and
// split rotation, apart from the FP64 and FP32 launches of the same steps.
enum KClass {
  KC_SPMM32, KC_SPMM64, KC_GRAM32, KC_GRAM64, KC_GRAD32, KC_GRAD64,
  KC_ROT32, KC_ROT64, KC_ROWOPS, KC_SMALL, KC_EIG, KC_SPMMDF, KC_ROTDF,
  KC_COUNT
};
extern const char* const kClassNames[KC_COUNT];

class Profiler {
 public:
  ~Profiler();
  bool on = false;
  void begin(int k, cudaStream_t s);
  void end(int k, double flops, double bytes, cudaStream_t s);
  void resolve();  // the stream must be idle
  void reset();
  // The next begin() records a fresh event (work other than kernel
  // launches, e.g. a copy, was enqueued since the last end()).
  void cut() { last_ = nullptr; }
  double ms[KC_COUNT] = {};
  long long launches[KC_COUNT] = {};
  double flops[KC_COUNT] = {};
  double bytes[KC_COUNT] = {};

 private:
  // b_taken: b is also the next record's a (and is released with it).
  struct Rec {
    int k;
    cudaEvent_t a, b;
    double flops, bytes;
    bool b_taken;
  };
  cudaEvent_t get();
  std::vector<Rec> pending_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t open_ = nullptr;
  bool open_shared_ = false;
  cudaEvent_t last_ = nullptr;  // end event of the last record
  long long last_launch_ = -1;  // thread launch count at that end
  cudaStream_t last_s_ = nullptr;
};

// Device memory owned by one solver; freed in the destructor.
// Device memory owned by one solver, stream-ordered: allocated from and
// returned to the device's memory pool on the solver's stream, so creating
// and destroying solvers never synchronises the device (cudaFree does), and
// concurrent solves on other streams keep running.
class DevArena {
 public:
  ~DevArena();
  void set_stream(cudaStream_t s) { s_ = s; }
  void* alloc(size_t bytes);
  size_t bytes() const { return total_; }

 private:
  std::vector<void*> ptrs_;
  size_t total_ = 0;
  cudaStream_t s_ = nullptr;
};

class Solver {
 public:
  Solver(int64_t N, int m, double tol, const trm_options& opt);
  ~Solver();
  static size_t footprint(int64_t N, int m);
  static size_t part_capacity(int64_t N, int m);
  size_t device_bytes() const { return mem_.bytes(); }

  void init_stencil(int nx, int ny, int nz, int order, double h,
                    const double* V_host);
  void init_csr(const int32_t* rowptr, const int32_t* cols, const void* vals,
                int vals_fp64);
  // Generalized problem H e = lambda S e: the SPD overlap S as CSR (FP64),
  // host arrays, validated by the caller. The iteration then keeps
  // C^T S C = I and carries Y = S C along with C (FP64 mode only).
  void init_overlap(const int32_t* rowptr, const int32_t* cols,
                    const double* vals);
  bool generalized() const { return has_S_; }
  int precision() const { return opt_.precision; }

  // Fig. TMFIG to convergence, then Rayleigh-Ritz. Returns a trm_status.
  int solve(double* lambda, double* E_G, double* C_out, int C_on_device,
            const double* C0_host, trm_stats* stats);

  // Step operations used by the C ABI.
  void apply(int din, const void* in, int dout, void* out, int ncols);
  void energy_gradient(const double* C, double* E, double* HD, double* Hprime,
                       void* G, int G_dtype, int zero_diag);
  void set_block(const double* C_dev);
  void get_block(double* C_dev);
  void iterate(int mode, int restart, double* E, double* rms, double* alpha);
  void rayleigh_ritz(double* C_dev, double* lambda_host, double* res_host);

  int64_t N() const { return N_; }
  // entries of the pinned ring of per-iteration scalars
  static constexpr int kRingSize = 64;
  // The scalars of every iteration of the last solve, in order, with the
  // phase the iteration ran in (0 full SP, 1 MP2, 2 FP64).
  struct IterRecord {
    IterScalars v;
    int phase;
  };
  const std::vector<IterRecord>& history() const { return history_; }
  Profiler prof;
  cudaStream_t stream() const { return s_; }
  std::string last_error;

 private:
  template <typename T, typename Tm>
  void iter_uniform(T*& C, T*& Cn, T* X, T*& G, T*& Gp, T* P, T* HP);
  void iter_mp2();
  void gram64(const double* A, const Blocks<double>& b, double* out);
  void mult64(const double* A, const double* M, double* Y);
  // The line-search Grams as one tensor-core launch [C P P]^T [P P G]
  // (C^T P, P^T P upper tiles mirrored, P^T G), with the diagonal of
  // P^T H P taken as column dots of the stencil applied to P (hpd_), when
  // the FP32 blocks are eligible.
  template <typename T>
  bool line_grams_fusable(const T* C, const T* P, const T* G) const;
  template <typename T>
  void line_grams_fused(const T* C, const T* P, const T* G);
  // CUDA graphs of block iterations. An iteration is a fixed kernel
  // sequence given the phase and the block pointers it swaps, so a graph is
  // keyed by both and remembers the pointers it leaves behind. The first
  // run of a key is plain (one-time setup such as kernel attributes stays
  // out of the capture), the second is captured, later ones replay it.
  static constexpr int kStatePtrs = 8;
  struct IterGraph {
    int phase;
    void* pre[kStatePtrs];
    void* post[kStatePtrs];
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<IterGraph> graphs_;
  void iter_state(void** st) const;
  void set_iter_state(void* const* st);
  template <typename F>
  void run_iteration(int phase, F&& body);
  void c64_to_df();
  void df_to_c64();
  void orth_fp64(double*& C, double*& Cn);
  template <typename T>
  void orth_uniform(T*& C, T*& Cn);
  void rr_rotate_fp64();  // C64 <- C64 Z diagonalising C^T H C
  // Final FP64 Rayleigh-Ritz on C64: writes lam_dev, res_dev, Cfin (=C64b)
  void final_rr(double* C, double* Cfin, double* Xfin);
  void set_restart();
  void read_scalars(IterScalars* out);

  int64_t N_;
  int m_;
  double tol_;
  trm_options opt_;
  cudaStream_t s_;
  Operator op_;
  DevArena mem_;
  int order_ = 0;
  // operator data
  double* diag64_ = nullptr;
  float* diag32_ = nullptr;
  float* diaglo_ = nullptr;
  double* minv64_ = nullptr;
  float* minv32_ = nullptr;
  // blocks (G, P, HP sized for FP64 and reused as FP32)
  double *C64_ = nullptr, *C64n_ = nullptr, *X64_ = nullptr;
  float *C32_ = nullptr, *C32n_ = nullptr, *X32_ = nullptr;
  float *Cdf_ = nullptr, *Cdfn_ = nullptr, *Xdf_ = nullptr;  // FP32 pairs
  void *Gb_[2] = {nullptr, nullptr}, *Pb_ = nullptr, *HPb_ = nullptr;
  // m x m (FP64)
  double *HD_, *hpdots_, *Hp_, *A0_, *Bm_, *PG_, *T1_, *T2_, *S_, *Linv_, *R_, *mmw_,
      *eigws_,
      *eigw_, *Z_, *lam_, *res_;
  int* info_;
  // FP32 copies of H', B = C^T P and P^T [P HP G] (the Gram sums write them)
  float *Hp32_ = nullptr, *Bm32_ = nullptr, *PG32_ = nullptr;
  double* part_;
  size_t part_cap_;
  IterScalars* sc_;
  TcWork tw_;  // tensor-core product workspace (error word in sc_->status)
  IterScalars* ring_ = nullptr;  // pinned host ring of per-iteration scalars
  std::vector<cudaEvent_t> ev_;
  int state_ = 0;  // 0: C64 current, 1: C32 current
  std::vector<IterRecord> history_;
  int ring_phase_[kRingSize] = {};  // phase of each ring entry's iteration
  // generalized problem: S as an operator, Y = S C (and its swap buffer),
  // S P of the line search, diag(S)
  Operator sop_;
  bool has_S_ = false;
  double *Y64_ = nullptr, *Y64n_ = nullptr, *SP64_ = nullptr;
  double* sdiag64_ = nullptr;
  float* sdiag32_ = nullptr;
  // the full-SP phase of the mixed ladder: Y = S C, its swap buffer and S P
  // in FP32 (S's values rounded to FP32 in sop_.csr.vals32)
  float *Y32_ = nullptr, *Y32n_ = nullptr, *SP32_ = nullptr;
};

}  // namespace trm
