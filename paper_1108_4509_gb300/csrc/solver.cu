// The trace-minimization loop of Fig. TMFIG on the device, with the precision
// modes of Sec. 2.2, driven from the host. Each iteration is a fixed sequence
// of kernels on one stream with no host synchronisation; the host reads the
// iteration's scalars (energy, residual, step) from a pinned ring a few
// iterations late and decides on convergence and on phase changes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "solver.cuh"

namespace trm {

namespace {

constexpr int kRing = Solver::kRingSize;

__global__ void k_set_restart(IterScalars* sc) {
  sc->restart = 1;
  sc->status = 0;
}

double neumaier_sum(const double* x, int n) {
  double s = 0.0, c = 0.0;
  for (int i = 0; i < n; ++i) {
    const double t = s + x[i];
    if (std::fabs(s) >= std::fabs(x[i]))
      c += (s - t) + x[i];
    else
      c += (x[i] - t) + s;
    s = t;
  }
  return s + c;
}

}  // namespace

int sm_count() {
  static std::atomic<int> cached{0};  // solves may run on several threads
  int n = cached.load(std::memory_order_relaxed);
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {
std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;  // launches issued by this host thread
thread_local long long* t_capture = nullptr;  // kernels of a graph being captured
}  // namespace

void count_launch() {
  if (t_capture) {  // captured into a graph: counted when the graph runs
    ++*t_capture;
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
void capture_launches(long long* sink) { t_capture = sink; }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }

const char* const kClassNames[KC_COUNT] = {
    "spmm_f32", "spmm_f64", "gram_f32", "gram_f64", "grad_f32", "grad_f64",
    "rotate_f32", "rotate_f64", "rowops", "small_mm", "eig", "spmm_df",
    "rotate_df"};

Profiler::~Profiler() {
  for (auto& r : pending_) {
    cudaEventDestroy(r.a);
    if (!r.b_taken) cudaEventDestroy(r.b);
  }
  for (auto e : pool_) cudaEventDestroy(e);
}

cudaEvent_t Profiler::get() {
  if (!pool_.empty()) {
    cudaEvent_t e = pool_.back();
    pool_.pop_back();
    return e;
  }
  cudaEvent_t e;
  TRM_CUDA(cudaEventCreate(&e));
  return e;
}

// Consecutive timed launches share one event: the end of one record is the
// start of the next when no other kernel was launched on the thread and
// nothing else was enqueued (cut()) in between, which halves the events
// recorded in the timed region.
void Profiler::begin(int, cudaStream_t s) {
  if (!on) return;
  if (last_ && s == last_s_ && thread_launch_count() == last_launch_ &&
      !pending_.empty() && pending_.back().b == last_) {
    pending_.back().b_taken = true;
    open_ = last_;
    open_shared_ = true;
  } else {
    open_ = get();
    open_shared_ = false;
    TRM_CUDA(cudaEventRecord(open_, s));
  }
  last_ = nullptr;
}

void Profiler::end(int k, double fl, double by, cudaStream_t s) {
  if (!on || !open_) return;
  cudaEvent_t b = get();
  TRM_CUDA(cudaEventRecord(b, s));
  pending_.push_back({k, open_, b, fl, by, false});
  open_ = nullptr;
  last_ = b;
  last_launch_ = thread_launch_count();
  last_s_ = s;
}

void Profiler::resolve() {
  size_t done = 0;
  for (auto& r : pending_) {
    if (cudaEventQuery(r.b) != cudaSuccess) break;
    float t = 0.f;
    TRM_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.k] += t;
    launches[r.k] += 1;
    flops[r.k] += r.flops;
    bytes[r.k] += r.bytes;
    // a record releases its start event (its own, or the previous record's
    // end, which it took over) and its end unless the next record took it
    pool_.push_back(r.a);
    if (!r.b_taken) pool_.push_back(r.b);
    ++done;
  }
  cudaGetLastError();
  pending_.erase(pending_.begin(), pending_.begin() + done);
  if (pending_.empty()) last_ = nullptr;
}

void Profiler::reset() {
  for (int k = 0; k < KC_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    flops[k] = bytes[k] = 0.0;
  }
}

// Pinned rings of per-iteration scalars, reused across solvers: a page-locked
// allocation (and its release) would serialise the streams of concurrent
// solves. Rings are kept for the life of the process (a few hundred bytes).
namespace {
std::mutex g_ring_mu;
std::vector<IterScalars*> g_rings;
}  // namespace

IterScalars* ring_acquire() {
  {
    std::lock_guard<std::mutex> lock(g_ring_mu);
    if (!g_rings.empty()) {
      IterScalars* r = g_rings.back();
      g_rings.pop_back();
      return r;
    }
  }
  IterScalars* r = nullptr;
  TRM_CUDA(cudaHostAlloc(&r, sizeof(IterScalars) * kRing,
                         cudaHostAllocDefault));
  return r;
}

void ring_release(IterScalars* r) {
  std::lock_guard<std::mutex> lock(g_ring_mu);
  g_rings.push_back(r);
}

DevArena::~DevArena() {
  for (void* p : ptrs_) cudaFreeAsync(p, s_);
}

namespace {
// The device's default pool keeps freed memory for reuse (no release to the
// driver at synchronisation), so repeated solver creation allocates without
// system calls. Set once per device.
void keep_pool_memory() {
  static std::atomic<int> done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (done[dev].exchange(1)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}
}  // namespace

void* DevArena::alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync(&p, bytes, s_);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(-2, "device allocation of " + std::to_string(bytes) +
                        " bytes failed: " + cudaGetErrorString(e));
  }
  ptrs_.push_back(p);
  total_ += bytes;
  return p;
}

// Doubles of the shared partial-sum buffer: the largest of the split-K Gram
// partials, the gradient's per-CTA sums and the column reductions.
size_t Solver::part_capacity(int64_t N, int m) {
  const size_t chunks = (size_t)ceil_div(N, 4096);
  const int tm = ceil_div(m, 128);  // the fused line Gram mirrors P^T P's
  return std::max<size_t>(          // tm (tm - 1) / 2 lower tiles
      {gram_partials_doubles(N, m, 4 * m), gram_partials_doubles(N, m, 3 * m),
       gram_partials_doubles(N, m, m),
       gram_tc_partials_doubles(N, m, 3 * m, tm * (tm - 1) / 2),
       (size_t)4 * ceil_div(N, 64) * ceil_div(m, 64), 3 * chunks * m + m,
       (size_t)ceil_div(N, 256) * m, (size_t)4096});
}

// Device bytes the constructor (and a stencil's potential) allocates; used
// to admit requests by footprint.
size_t Solver::footprint(int64_t N, int m) {
  const size_t nm = (size_t)N * m, mm = (size_t)m * m;
  size_t b = nm * (3 * 8 + 3 * 4 + 3 * 8 + 4 * 8);  // blocks
  b += mm * 8 * 13 + std::max(2 * mm, chol_work_elems(m)) * 8 + 4 * m * 8;
  b += std::max<size_t>(1, (size_t)ceil_div(N, 256) * m) * 8;  // P's dots
  b += sym_eig_work_doubles(m) * 8 + 5 * mm * 4;
  b += part_capacity(N, m) * 8 + sizeof(IterScalars) + 16;
  b += mul_tc_work_floats(m, m) * 4;
  b += (size_t)N * (8 + 4 + 4 + 8 + 4 + 8);  // diagonals, M, V
  return b + (64u << 10);                    // allocation granularity
}

Solver::Solver(int64_t N, int m, double tol, const trm_options& opt)
    : N_(N), m_(m), tol_(tol), opt_(opt) {
  s_ = reinterpret_cast<cudaStream_t>(opt.stream);
  mem_.set_stream(s_);
  const size_t nm = (size_t)N * m;
  const size_t mm = (size_t)m * m;
  auto d = [&](size_t n) { return static_cast<double*>(mem_.alloc(n * 8)); };
  auto f = [&](size_t n) { return static_cast<float*>(mem_.alloc(n * 4)); };
  C64_ = d(nm);
  C64n_ = d(nm);
  X64_ = d(nm);
  C32_ = f(nm);
  C32n_ = f(nm);
  X32_ = f(nm);
  Cdf_ = f(2 * nm);  // MP2 blocks as FP32 pairs: hi at [0, nm), lo after
  Cdfn_ = f(2 * nm);
  Xdf_ = f(2 * nm);
  Gb_[0] = d(nm);
  Gb_[1] = d(nm);
  Pb_ = d(nm);
  HPb_ = d(nm);
  for (void* p : {Gb_[0], Gb_[1], Pb_, HPb_})
    TRM_CUDA(cudaMemsetAsync(p, 0, nm * 8, s_));
  HD_ = d(m);
  // partial column dots of the stencil applied to P (their sum is
  // tr(P^T H P)), kept apart from part_, which the Grams then reuse
  hpdots_ = d(std::max<size_t>(1, (size_t)ceil_div(N, 256) * m));
  Hp_ = d(mm);
  A0_ = d(mm);
  Bm_ = d(4 * mm);  // C^T P, then P^T [P HP G] (unfused) or P^T [P G] (fused)
  PG_ = Bm_ + mm;
  // (also the line terms' partials: 4 doubles per CTA, at most
  // 4 * 4 ceil(m/32)^2 + 256 doubles, more than m^2 when m is small)
  T1_ = d(std::max(mm, (size_t)16 * ceil_div(m, 32) * ceil_div(m, 32) + 256));
  T2_ = d(mm);
  S_ = d(mm);
  Linv_ = d(mm);
  R_ = d(mm);
  Z_ = d(mm);
  mmw_ = d(std::max(2 * mm, chol_work_elems(m)));
  eigws_ = d(sym_eig_work_doubles(m));
  Hp32_ = f(mm);
  Bm32_ = f(4 * mm);
  PG32_ = Bm32_ + mm;
  eigw_ = d(m);
  lam_ = d(m);
  res_ = d(m);
  info_ = static_cast<int*>(mem_.alloc(16));
  part_cap_ = part_capacity(N, m);
  part_ = d(part_cap_);
  sc_ = static_cast<IterScalars*>(mem_.alloc(sizeof(IterScalars)));
  TRM_CUDA(cudaMemsetAsync(sc_, 0, sizeof(IterScalars), s_));
  op_.err = &sc_->status;
  tw_.msplit_floats = mul_tc_work_floats(m, m);
  tw_.msplit = f(tw_.msplit_floats);
  tw_.err = &sc_->status;
  diag64_ = d(N);
  diag32_ = f(N);
  diaglo_ = f(N);
  minv64_ = d(N);
  minv32_ = f(N);
  ring_ = ring_acquire();
  ev_.resize(kRing);
  for (auto& e : ev_) TRM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  set_restart();
}

Solver::~Solver() {
  if (s_) cudaStreamSynchronize(s_);
  else cudaDeviceSynchronize();
  for (auto& g : graphs_)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& e : ev_) cudaEventDestroy(e);
  if (ring_) ring_release(ring_);
}

void Solver::init_stencil(int nx, int ny, int nz, int order, double h,
                          const double* V_host) {
  order_ = order;
  const double t = 0.5 / (h * h);
  double w0, w1, w2;
  if (order == 2) {
    w0 = 2.0; w1 = -1.0; w2 = 0.0;
  } else {
    w0 = 2.5; w1 = -4.0 / 3.0; w2 = 1.0 / 12.0;
  }
  const int ndim = (nx > 1) + (ny > 1) + (nz > 1);
  op_.kind = 0;
  op_.N = N_;
  op_.st.nx = nx;
  op_.st.ny = ny;
  op_.st.nz = nz;
  op_.st.radius = order == 2 ? 1 : 2;
  op_.st.c1 = t * w1;
  op_.st.c2 = t * w2;
  op_.st.c1h = (float)op_.st.c1;
  op_.st.c1l = (float)(op_.st.c1 - (double)op_.st.c1h);
  op_.st.c2h = (float)op_.st.c2;
  op_.st.c2l = (float)(op_.st.c2 - (double)op_.st.c2h);
  double* Vd = nullptr;
  if (V_host) {
    Vd = static_cast<double*>(mem_.alloc((size_t)N_ * 8));
    TRM_CUDA(cudaMemcpyAsync(Vd, V_host, (size_t)N_ * 8,
                             cudaMemcpyHostToDevice, s_));
  }
  stencil_diag(op_.st, t * w0 * ndim, Vd, diag64_, diag32_, N_, s_);
  split_df(diag64_, diag32_, diaglo_, N_, s_);
  op_.diag64 = diag64_;
  op_.diag32 = diag32_;
  op_.diaglo = diaglo_;
  if (opt_.precond) {
    diag_preconditioner(diag64_, N_, minv64_, minv32_, part_, s_);
    op_.minv64 = minv64_;
    op_.minv32 = minv32_;
  }
  TRM_CUDA(cudaStreamSynchronize(s_));
}

void Solver::init_csr(const int32_t* rowptr, const int32_t* cols,
                      const void* vals, int vals_fp64) {
  const int64_t nnz = rowptr[N_];
  auto* rp = static_cast<int32_t*>(mem_.alloc((size_t)(N_ + 1) * 4));
  auto* ci = static_cast<int32_t*>(mem_.alloc((size_t)nnz * 4));
  TRM_CUDA(cudaMemcpyAsync(rp, rowptr, (size_t)(N_ + 1) * 4,
                           cudaMemcpyHostToDevice, s_));
  TRM_CUDA(cudaMemcpyAsync(ci, cols, (size_t)nnz * 4, cudaMemcpyHostToDevice,
                           s_));
  op_.kind = 1;
  op_.N = N_;
  op_.csr.rowptr = rp;
  op_.csr.cols = ci;
  int mx = 0;
  for (int64_t r = 0; r < N_; ++r) mx = std::max(mx, rowptr[r + 1] - rowptr[r]);
  op_.csr.max_row_nnz = mx;
  if (vals_fp64) {
    auto* v = static_cast<double*>(mem_.alloc((size_t)nnz * 8));
    TRM_CUDA(cudaMemcpyAsync(v, vals, (size_t)nnz * 8, cudaMemcpyHostToDevice,
                             s_));
    op_.csr.vals64 = v;
    auto* vh = static_cast<float*>(mem_.alloc((size_t)nnz * 4));
    auto* vl = static_cast<float*>(mem_.alloc((size_t)nnz * 4));
    split_df(v, vh, vl, nnz, s_);
    op_.csr.valshi = vh;
    op_.csr.valslo = vl;
    op_.csr.vals32 = vh;  // fl32(v): the FP32 products take it directly
  } else {
    auto* v = static_cast<float*>(mem_.alloc((size_t)nnz * 4));
    TRM_CUDA(cudaMemcpyAsync(v, vals, (size_t)nnz * 4, cudaMemcpyHostToDevice,
                             s_));
    op_.csr.vals32 = v;
    auto* vl = static_cast<float*>(mem_.alloc((size_t)nnz * 4));
    TRM_CUDA(cudaMemsetAsync(vl, 0, (size_t)nnz * 4, s_));
    op_.csr.valshi = v;
    op_.csr.valslo = vl;
  }
  csr_diag(op_, diag64_, diag32_, s_);
  split_df(diag64_, diag32_, diaglo_, N_, s_);
  op_.diag64 = diag64_;
  op_.diag32 = diag32_;
  op_.diaglo = diaglo_;
  if (opt_.precond) {
    diag_preconditioner(diag64_, N_, minv64_, minv32_, part_, s_);
    op_.minv64 = minv64_;
    op_.minv32 = minv32_;
  }
  TRM_CUDA(cudaStreamSynchronize(s_));
}

void Solver::init_overlap(const int32_t* rowptr, const int32_t* cols,
                          const double* vals) {
  const int64_t nnz = rowptr[N_];
  auto* rp = static_cast<int32_t*>(mem_.alloc((size_t)(N_ + 1) * 4));
  auto* ci = static_cast<int32_t*>(mem_.alloc((size_t)nnz * 4));
  auto* v = static_cast<double*>(mem_.alloc((size_t)nnz * 8));
  TRM_CUDA(cudaMemcpyAsync(rp, rowptr, (size_t)(N_ + 1) * 4,
                           cudaMemcpyHostToDevice, s_));
  TRM_CUDA(cudaMemcpyAsync(ci, cols, (size_t)nnz * 4, cudaMemcpyHostToDevice,
                           s_));
  TRM_CUDA(cudaMemcpyAsync(v, vals, (size_t)nnz * 8, cudaMemcpyHostToDevice,
                           s_));
  sop_ = Operator{};
  sop_.kind = 1;
  sop_.N = N_;
  sop_.csr.rowptr = rp;
  sop_.csr.cols = ci;
  sop_.csr.vals64 = v;
  if (opt_.precision != TRM_FP64) {  // the full-SP phase applies S in FP32
    std::vector<float> v32(nnz);
    for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)vals[k];
    auto* vf = static_cast<float*>(mem_.alloc((size_t)nnz * 4));
    TRM_CUDA(cudaMemcpyAsync(vf, v32.data(), (size_t)nnz * 4,
                             cudaMemcpyHostToDevice, s_));
    TRM_CUDA(cudaStreamSynchronize(s_));  // v32 leaves scope
    sop_.csr.vals32 = vf;
    if (!Y32_) {
      const size_t nm = (size_t)N_ * m_;
      Y32_ = static_cast<float*>(mem_.alloc(nm * 4));
      Y32n_ = static_cast<float*>(mem_.alloc(nm * 4));
      SP32_ = static_cast<float*>(mem_.alloc(nm * 4));
    }
  }
  int mx = 0;
  for (int64_t r = 0; r < N_; ++r) mx = std::max(mx, rowptr[r + 1] - rowptr[r]);
  sop_.csr.max_row_nnz = mx;
  sop_.err = &sc_->status;
  if (!Y64_) {
    const size_t nm = (size_t)N_ * m_;
    Y64_ = static_cast<double*>(mem_.alloc(nm * 8));
    Y64n_ = static_cast<double*>(mem_.alloc(nm * 8));
    SP64_ = static_cast<double*>(mem_.alloc(nm * 8));
    sdiag64_ = static_cast<double*>(mem_.alloc((size_t)N_ * 8));
    sdiag32_ = static_cast<float*>(mem_.alloc((size_t)N_ * 4));
  }
  csr_diag(sop_, sdiag64_, sdiag32_, s_);
  sop_.diag64 = sdiag64_;
  sop_.diag32 = sdiag32_;
  if (opt_.precond) {  // M = diag(1 / (H_ii - sigma S_ii))
    diag_preconditioner_gen(diag64_, sdiag64_, N_, minv64_, minv32_, part_,
                            s_);
    op_.minv64 = minv64_;
    op_.minv32 = minv32_;
  }
  has_S_ = true;
  TRM_CUDA(cudaStreamSynchronize(s_));
}

// Algorithmic flops and bytes of one H application to ncols columns of
// element size es: every stored nonzero is one multiply-add; the block is read
// and written once and the operator data (diagonal or CSR) read once.
static void spmm_cost(const Operator& op, int ncols, int es, double* fl,
                      double* by) {
  const double N = (double)op.N;
  double nnz_row;
  if (op.kind == 0) {
    const int ndim = (op.st.nx > 1) + (op.st.ny > 1) + (op.st.nz > 1);
    nnz_row = 1.0 + 2.0 * op.st.radius * ndim;
    *by = 2.0 * es * N * ncols + 8.0 * N;
  } else {
    nnz_row = 0.0;  // filled below
    *by = 2.0 * es * N * ncols;
  }
  if (op.kind == 1) {
    // nnz is not stored on the device side; the row-length bound is used
    nnz_row = op.csr.max_row_nnz;
    const int vs = op.csr.vals64 ? 8 : 4;
    *by += N * nnz_row * (4.0 + vs) + 4.0 * (N + 1);
  }
  *fl = 2.0 * nnz_row * N * ncols;
}

#define TRM_PROF(k, fl, by, call) \
  do {                            \
    prof.begin((k), s_);          \
    call;                         \
    prof.end((k), (fl), (by), s_); \
  } while (0)

void Solver::set_restart() {
  k_set_restart<<<1, 1, 0, s_>>>(sc_);
  TRM_CHECK_LAUNCH();
}

void Solver::read_scalars(IterScalars* out) {
  TRM_CUDA(cudaMemcpyAsync(&ring_[0], sc_, sizeof(IterScalars),
                           cudaMemcpyDeviceToHost, s_));
  TRM_CUDA(cudaStreamSynchronize(s_));
  *out = ring_[0];
}

// ---------------------------------------------------------------------------
// One iteration with every block in precision T and the m x m line model and
// factorisation in Tm (full DP: double/double; full SP: float/float).
// ---------------------------------------------------------------------------
// The line-search Grams C^T P, P^T P and P^T G as one tensor-core launch
// [C P P]^T [P P G] (one m x 3m result: Bm_, then PG_ = [P^T P, P^T G]).
// P^T P is symmetric, so only its tiles on and above the diagonal are
// computed and the rest are mirrored (the blocked symmetric product of
// Sec. 2.1, Fig. DIVFIG); of P^T H P the line model needs only the
// diagonal, which the stencil applied to P delivers as column dots, so HP
// is not read here at all.
// ---------------------------------------------------------------------------
template <typename T>
bool Solver::line_grams_fusable(const T* C, const T* P, const T* G) const {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    Blocks<float> a, b;
    a.p[0] = C;
    a.p[1] = a.p[2] = P;
    b.p[0] = b.p[1] = P;
    b.p[2] = G;
    a.cols = b.cols = m_;
    a.count = b.count = 3;
    return gram_tc_pairs_eligible(N_, m_, a, b);
  }
}

template <typename T>
void Solver::line_grams_fused(const T* C, const T* P, const T* G) {
  if constexpr (sizeof(T) == 4) {
    Blocks<float> a, b;
    a.p[0] = C;
    a.p[1] = a.p[2] = P;
    b.p[0] = b.p[1] = P;
    b.p[2] = G;
    a.cols = b.cols = m_;
    a.count = b.count = 3;
    const double nm = (double)N_ * m_, m2N = nm * m_;
    // algorithmic: 2 m^2 N per product, m^2 N for the symmetric one
    TRM_PROF(KC_GRAM32, 5 * m2N, 12 * nm,
             gram_tc_pairs(N_, m_, a, b, Bm_, part_, part_cap_, &sc_->status,
                           s_, Bm32_, /*sym_seg=*/1));
  }
}

template <typename T, typename Tm>
void Solver::iter_uniform(T*& C, T*& Cn, T* X, T*& G, T*& Gp, T* P, T* HP) {
  const T* minv = nullptr;
  if (opt_.precond) {
    if constexpr (sizeof(T) == 4)
      minv = minv32_;
    else
      minv = minv64_;
  }
  const size_t mm = (size_t)m_ * m_;
  const double es = sizeof(T), Nd = (double)N_, md = m_;
  const double nm = Nd * md, m2N = nm * md;
  const int ksp = sizeof(T) == 4 ? KC_SPMM32 : KC_SPMM64;
  const int kgr = sizeof(T) == 4 ? KC_GRAM32 : KC_GRAM64;
  const int kgd = sizeof(T) == 4 ? KC_GRAD32 : KC_GRAD64;
  const int krt = sizeof(T) == 4 ? KC_ROT32 : KC_ROT64;
  double sfl, sby;
  spmm_cost(op_, m_, (int)es, &sfl, &sby);
  // Generalized problem (FP64 only): C^T S C = I, and Y = S C takes C's
  // place where the constraint enters, X' = X - Y H_D and G = -2 (X' - Y H');
  // the line search projects with S P, and Y is rotated along with C.
  const T* Yc = C;
  T* SPt = P;
  bool gen = false;
  if constexpr (sizeof(T) == 8) {
    if (has_S_) {
      Yc = Y64_;
      SPt = SP64_;
      gen = true;
    }
  } else {  // the mixed ladder's full-SP phase
    if (has_S_) {
      Yc = Y32_;
      SPt = SP32_;
      gen = true;
    }
  }
  if constexpr (sizeof(T) == 4) {  // (1) with the column dots of (2) fused in
    int chunks = 0;
    TRM_PROF(ksp, sfl, sby, chunks = apply_h_dots(op_, C, X, m_, part_, s_));
    TRM_PROF(KC_ROWOPS, 2.0 * m_ * chunks, 8.0 * m_ * chunks,
             energy_from_dots(part_, chunks, m_, HD_, sc_, s_));      // (2), (3)
  } else {
    TRM_PROF(ksp, sfl, sby, apply_h(op_, C, X, m_, s_));             // (1)
    TRM_PROF(KC_ROWOPS, 2 * nm, 2 * es * nm,
             energy_diag<T>(N_, m_, C, X, HD_, sc_, part_, s_));      // (2), (3)
  }
  TRM_PROF(KC_ROWOPS, 2 * nm, 3 * es * nm,
           xprime<T>(N_, m_, Yc, X, HD_, nullptr, nullptr, s_));      // (5)
  Blocks<T> bx;
  bx.p[0] = X;
  bx.cols = m_;
  bx.count = 1;
  // FP32 phases also get FP32 copies of the m x m Gram results
  float* const hp32 = sizeof(T) == 4 ? Hp32_ : nullptr;
  float* const bm32 = sizeof(T) == 4 ? Bm32_ : nullptr;
  float* const pg32 = sizeof(T) == 4 ? PG32_ : nullptr;
  TRM_PROF(kgr, 2 * m2N, 2 * es * nm,
           gram<T>(N_, m_, C, bx, Hp_, part_, part_cap_, s_, &sc_->status,
                   hp32));                                            // (6)
  if (sizeof(T) == 4) zero_diag(m_, Hp_, s_, hp32);
  TRM_PROF(kgd, 2 * m2N, 5 * es * nm,
           gradient<T>(N_, m_, Yc, X, Hp_, G, Gp, P, minv, sc_, part_,
                       part_cap_, s_, &tw_));                         // (7)
  TRM_PROF(KC_ROWOPS, 2 * nm, 3 * es * nm,
           update_p<T>(N_, m_, G, P, minv, sc_, s_));                 // P
  const bool fused = !gen && line_grams_fusable<T>(C, P, G);
  int hp_chunks = 0;  // > 0: tr(P^T H P) from the stencil's column dots
  if constexpr (sizeof(T) == 4) {
    // the fused line Grams need only tr(P^T H P): the stencil forms its
    // column dots and writes no H P
    if (fused)
      TRM_PROF(ksp, sfl, sby - es * nm,
               hp_chunks = apply_h_dots(op_, P, nullptr, m_, hpdots_, s_));
  }
  if (!hp_chunks) TRM_PROF(ksp, sfl, sby, apply_h(op_, P, HP, m_, s_));  // H P
  if (gen) {
    double ffl, fby;
    spmm_cost(sop_, m_, (int)es, &ffl, &fby);
    TRM_PROF(ksp, ffl, fby, apply_h(sop_, P, SPt, m_, s_));          // S P
  }
  // where the trace of P^T H P and W = P^T G come from
  const double* hpd = nullptr;
  const double* trp = hp_chunks ? hpdots_ : nullptr;
  const int ntrp = hp_chunks * m_;
  size_t woff = mm;
  if (fused) {
    line_grams_fused<T>(C, P, G);
  } else {
    hpd = PG_ + mm;  // the diagonal of P^T H P, stride m + 1
    woff = 2 * mm;
    Blocks<T> bp;
    bp.p[0] = P;
    bp.cols = m_;
    bp.count = 1;
    TRM_PROF(kgr, 2 * m2N, 2 * es * nm,
             gram<T>(N_, m_, Yc, bp, Bm_, part_, part_cap_, s_, &sc_->status,
                     bm32));                                     // C^T (S) P
    Blocks<T> b3;
    b3.p[0] = SPt;
    b3.p[1] = HP;
    b3.p[2] = G;
    b3.cols = m_;
    b3.count = 3;
    TRM_PROF(kgr, 6 * m2N, 4 * es * nm,
             gram<T>(N_, m_, P, b3, PG_, part_, part_cap_, s_, &sc_->status,
                     pg32));                                          // P^T[P HP G]
  }
  const double m3 = md * md * md;
  prof.begin(KC_SMALL, s_);
  if constexpr (sizeof(T) == 4 && sizeof(Tm) == 4)
    line_factor32(m_, Hp32_, HD_, Bm32_, PG32_, hpd, m_ + 1, trp, ntrp,
                  PG32_ + woff, nullptr, R_, sc_, mmw_, T1_,
                  s_);  // alpha, Fig. ONFIG
  else
    line_factor<Tm>(m_, Hp_, HD_, Bm_, PG_, hpd, m_ + 1, trp, ntrp,
                    PG_ + woff, nullptr, R_, sc_, mmw_, T1_,
                    sizeof(Tm) == 4, s_);
  prof.end(KC_SMALL, 4 * m3 + 2 * m3 / 3, 0.0, s_);
  TRM_PROF(krt, m2N, 3 * es * nm,
           (rotate<T, T>(N_, m_, C, P, R_, Cn, sc_, s_, &tw_)));  // (C+aP)L^-T
  if (gen) {  // S (C + aP) L^-T = (Y + a S P) L^-T
    if constexpr (sizeof(T) == 8) {
      TRM_PROF(krt, m2N, 3 * es * nm,
               (rotate<double, double>(N_, m_, Y64_, SP64_, R_, Y64n_, sc_,
                                       s_, &tw_)));
      std::swap(Y64_, Y64n_);
    } else {
      TRM_PROF(krt, m2N, 3 * es * nm,
               (rotate<float, float>(N_, m_, Y32_, SP32_, R_, Y32n_, sc_, s_,
                                     &tw_)));
      std::swap(Y32_, Y32n_);
    }
  }
  std::swap(C, Cn);
  std::swap(G, Gp);
}

// ---------------------------------------------------------------------------
// MP2 (Sec. 2.2): steps (1), (2), (3), (5) and E at FP64-class accuracy, in
// double-float (C and X = HC held as FP32 pairs, ~48 bits: GB300's FP64
// pipe is 1/64 of its FP32 rate); H' and G from FP32 products (diag(H') =
// 0) with C32 = the hi half of C; G, P, HP stored FP32; m x m work in FP32
// deviation form; the rotation split as C L_D (double-float) + C L' (FP32,
// tensor cores).
// ---------------------------------------------------------------------------
void Solver::iter_mp2() {
  float* G = static_cast<float*>(Gb_[0]);
  float* Gp = static_cast<float*>(Gb_[1]);
  float* P = static_cast<float*>(Pb_);
  float* HP = static_cast<float*>(HPb_);
  const float* minv = opt_.precond ? minv32_ : nullptr;
  const size_t mm = (size_t)m_ * m_;
  const size_t nm = (size_t)N_ * m_;
  const double Nd = (double)N_, md = m_;
  const double dnm = Nd * md, m2N = dnm * md, m3 = md * md * md;
  float* Ch = Cdf_;
  float* Cl = Cdf_ + nm;
  float* Xh = Xdf_;
  float* Xl = Xdf_ + nm;
  double f64, b64, f32, b32;
  spmm_cost(op_, m_, 8, &f64, &b64);
  spmm_cost(op_, m_, 4, &f32, &b32);
  // (1) with the column dots of (2) fused in where the stencil kernel allows
  int chunks = 0;
  TRM_PROF(KC_SPMMDF, f64, b64,
           chunks = apply_h_df_dots(op_, Ch, Cl, Xh, Xl, m_, part_, s_));
  if (chunks) {
    TRM_PROF(KC_ROWOPS, 2.0 * m_ * chunks, 8.0 * m_ * chunks,
             energy_from_dots(part_, chunks, m_, HD_, sc_, s_));  // (2), (3)
  } else {
    TRM_PROF(KC_SPMMDF, f64, b64, apply_h_df(op_, Ch, Cl, Xh, Xl, m_, s_));
    TRM_PROF(KC_ROWOPS, 2 * dnm, 16 * dnm,
             energy_diag_df(N_, m_, Ch, Cl, Xh, Xl, HD_, sc_, part_, s_));
  }
  TRM_PROF(KC_ROWOPS, 2 * dnm, 20 * dnm,
           xprime_df(N_, m_, Ch, Cl, Xh, Xl, HD_, X32_, s_));  // (5) FP32 X'
  Blocks<float> bx;
  bx.p[0] = X32_;
  bx.cols = m_;
  bx.count = 1;
  TRM_PROF(KC_GRAM32, 2 * m2N, 8 * dnm,
           gram<float>(N_, m_, Ch, bx, Hp_, part_, part_cap_, s_, &sc_->status,
                       Hp32_));                                       // (6)
  zero_diag(m_, Hp_, s_, Hp32_);
  TRM_PROF(KC_GRAD32, 2 * m2N, 20 * dnm,
           gradient<float>(N_, m_, Ch, X32_, Hp_, G, Gp, P, minv, sc_,
                           part_, part_cap_, s_, &tw_));      // (7)
  TRM_PROF(KC_ROWOPS, 2 * dnm, 12 * dnm,
           update_p<float>(N_, m_, G, P, minv, sc_, s_));
  const bool fused = line_grams_fusable<float>(Ch, P, G);
  const double* hpd = nullptr;
  const double* trp = nullptr;
  int ntrp = 0;
  size_t woff = mm;
  if (fused) {  // tr(P^T H P) as the stencil's column dots, no H P written
    int chunks = 0;
    TRM_PROF(KC_SPMM32, f32, b32 - 4 * dnm,
             chunks = apply_h_dots(op_, P, nullptr, m_, hpdots_, s_));
    trp = hpdots_;
    ntrp = chunks * m_;
    line_grams_fused<float>(Ch, P, G);
  } else {
    TRM_PROF(KC_SPMM32, f32, b32, apply_h(op_, P, HP, m_, s_));
    hpd = PG_ + mm;  // the diagonal of P^T H P, stride m + 1
    woff = 2 * mm;
    Blocks<float> bp;
    bp.p[0] = P;
    bp.cols = m_;
    bp.count = 1;
    TRM_PROF(KC_GRAM32, 2 * m2N, 8 * dnm,
             gram<float>(N_, m_, Ch, bp, Bm_, part_, part_cap_, s_,
                         &sc_->status, Bm32_));
    Blocks<float> b3;
    b3.p[0] = P;
    b3.p[1] = HP;
    b3.p[2] = G;
    b3.cols = m_;
    b3.count = 3;
    TRM_PROF(KC_GRAM32, 6 * m2N, 16 * dnm,
             gram<float>(N_, m_, P, b3, PG_, part_, part_cap_, s_,
                         &sc_->status, PG32_));
  }
  prof.begin(KC_SMALL, s_);
  line_factor32(m_, Hp32_, HD_, Bm32_, PG32_, hpd, m_ + 1, trp, ntrp,
                PG32_ + woff, nullptr, R_, sc_, mmw_, T1_, s_);
  prof.end(KC_SMALL, 4 * m3 + 2 * m3 / 3, 0.0, s_);
  TRM_PROF(KC_ROTDF, m2N, 24 * dnm,
           rotate_split_df(N_, m_, Ch, Cl, P, R_, Cdfn_, Cdfn_ + nm, sc_, s_,
                           &tw_));
  std::swap(Cdf_, Cdfn_);
  std::swap(Gb_[0], Gb_[1]);
}

// The MP2 blocks between FP64 and FP32 pairs (at re-orthonormalizations,
// Rayleigh-Ritz rotations and phase changes).
void Solver::c64_to_df() {
  const size_t nm = (size_t)N_ * m_;
  split_df(C64_, Cdf_, Cdf_ + nm, (int64_t)nm, s_);
}
void Solver::df_to_c64() {
  const size_t nm = (size_t)N_ * m_;
  join_df(Cdf_, Cdf_ + nm, C64_, (int64_t)nm, s_);
}

// The N-deep Grams of FP64 blocks: FP64 in the all-FP64 mode, double-float
// (FP64-class, on the FP32 pipe) in the mixed ladder.
void Solver::gram64(const double* A, const Blocks<double>& b, double* out) {
  if (opt_.precision == TRM_FP64)
    gram<double>(N_, m_, A, b, out, part_, part_cap_, s_, &sc_->status);
  else
    gram_df(N_, m_, A, b, out, part_, part_cap_, s_);
}

// N x m times m x m products of FP64 blocks, FP64 or double-float as gram64.
void Solver::mult64(const double* A, const double* M, double* Y) {
  if (opt_.precision == TRM_FP64)
    mult(N_, m_, m_, A, M, Y, s_);
  else
    mult_df(N_, m_, m_, A, M, Y, false, s_);
}

// Fig. ONFIG in FP64: S = C^T C, S = L L^T, C <- C L^{-T} (generalized
// problem: S = C^T Y with Y = S C recomputed, and Y <- Y L^{-T} too).
void Solver::orth_fp64(double*& C, double*& Cn) {
  Blocks<double> b;
  b.p[0] = C;
  b.cols = m_;
  b.count = 1;
  const double nm = (double)N_ * m_, m2N = nm * m_;
  if (has_S_) {
    double ffl, fby;
    spmm_cost(sop_, m_, 8, &ffl, &fby);
    TRM_PROF(KC_SPMM64, ffl, fby, apply_h(sop_, C, Y64_, m_, s_));
    b.p[0] = Y64_;
  }
  TRM_PROF(KC_GRAM64, 2 * m2N, 16 * nm, gram64(C, b, S_));
  TRM_PROF(KC_SMALL, 2.0 * m_ * m_ * m_ / 3, 0.0,
           chol_inv<double>(m_, S_, Linv_, R_, sc_, mmw_, s_));
  if (opt_.precision == TRM_FP64)
    TRM_PROF(KC_ROT64, m2N, 16 * nm,
             (rotate<double, double>(N_, m_, C, nullptr, R_, Cn, nullptr, s_)));
  else  // C L^{-T} in double-float
    TRM_PROF(KC_ROT64, m2N, 16 * nm, mult_df(N_, m_, m_, C, R_, Cn, true, s_));
  if (has_S_) {
    TRM_PROF(KC_ROT64, m2N, 16 * nm,
             (rotate<double, double>(N_, m_, Y64_, nullptr, R_, Y64n_, nullptr,
                                     s_)));
    std::swap(Y64_, Y64n_);
  }
  std::swap(C, Cn);
}

template <typename T>
void Solver::orth_uniform(T*& C, T*& Cn) {
  Blocks<T> b;
  b.p[0] = C;
  b.cols = m_;
  b.count = 1;
  bool gen = false;  // FP32 generalized: S = C^T Y with Y = S C recomputed
  if constexpr (sizeof(T) == 4) {
    if (has_S_) {
      apply_h(sop_, C, Y32_, m_, s_);
      b.p[0] = Y32_;
      gen = true;
    }
  }
  gram<T>(N_, m_, C, b, S_, part_, part_cap_, s_, &sc_->status);
  chol_inv<T>(m_, S_, Linv_, R_, sc_, mmw_, s_);
  rotate<T, T>(N_, m_, C, static_cast<const T*>(nullptr), R_, Cn, nullptr,
               s_, &tw_);
  if constexpr (sizeof(T) == 4) {
    if (gen) {  // Y follows C
      rotate<float, float>(N_, m_, Y32_, static_cast<const float*>(nullptr),
                           R_, Y32n_, nullptr, s_, &tw_);
      std::swap(Y32_, Y32n_);
    }
  }
  std::swap(C, Cn);
}

// Subspace rotation diagonalising C^T H C (Sec. 3, the MP2 accuracy remedy).
void Solver::rr_rotate_fp64() {
  apply_h(op_, C64_, X64_, m_, s_);
  Blocks<double> b;
  b.p[0] = X64_;
  b.cols = m_;
  b.count = 1;
  gram64(C64_, b, Hp_);
  make_A0(m_, Hp_, nullptr, A0_, s_);
  TRM_PROF(KC_EIG, 0.0, 0.0, sym_eig(m_, A0_, eigw_, Z_, eigws_, info_, s_));
  const double nm = (double)N_ * m_;
  TRM_PROF(KC_ROT64, 2 * nm * m_, 16 * nm, mult64(C64_, Z_, C64n_));
  std::swap(C64_, C64n_);
  if (has_S_) {  // Y = S C follows the rotation
    TRM_PROF(KC_ROT64, 2 * nm * m_, 16 * nm, mult64(Y64_, Z_, Y64n_));
    std::swap(Y64_, Y64n_);
  }
}

// Rayleigh-Ritz on span(C) (Sec. 2.1) in FP64, as the generalised problem
// (C^T H C) y = theta (C^T C) y: L = chol(C^T C), A~ = L^{-1} (C^T H C) L^{-T},
// A~ = Z diag(theta) Z^T, Y = L^{-T} Z, C Y and H C Y, column residuals
// (generalized problem: C^T S C in place of C^T C, residuals H c - theta S c).
void Solver::final_rr(double* C, double* Cfin, double* Xfin) {
  apply_h(op_, C, X64_, m_, s_);
  Blocks<double> bx;
  bx.p[0] = X64_;
  bx.cols = m_;
  bx.count = 1;
  gram64(C, bx, Hp_);
  Blocks<double> bc;
  bc.p[0] = C;
  bc.cols = m_;
  bc.count = 1;
  if (has_S_) {
    apply_h(sop_, C, Y64_, m_, s_);
    bc.p[0] = Y64_;
  }
  // the overlap in FP64 in every mode: the returned block is orthonormalized
  // by its factor (the double-float Gram's sum over N rows is good to about
  // sqrt(N) 2^-48, which left C^T C - I near 1e-12 at N ~ 1e6)
  gram<double>(N_, m_, C, bc, S_, part_, part_cap_, s_);
  chol_inv<double>(m_, S_, Linv_, R_, sc_, mmw_, s_);
  mm_gemm(m_, Linv_, false, Hp_, false, T1_, 1.0, 0.0, s_);
  mm_gemm(m_, T1_, false, Linv_, true, T2_, 1.0, 0.0, s_);
  make_A0(m_, T2_, nullptr, A0_, s_);
  sym_eig(m_, A0_, lam_, Z_, eigws_, info_, s_);
  mm_gemm(m_, R_, false, Z_, false, T1_, 1.0, 0.0, s_);
  // the returned block in FP64 in every mode; H C Y, used only for the
  // residual norms, keeps the FP64-class product
  mult(N_, m_, m_, C, T1_, Cfin, s_);
  mult64(X64_, T1_, Xfin);
  if (has_S_) {  // ||H c_j - theta_j S c_j|| (sign independent)
    mult64(Y64_, T1_, SP64_);
    column_residuals(N_, m_, Xfin, SP64_, lam_, res_, part_, s_);
    fix_signs(N_, m_, Cfin, Xfin, part_, s_);
    return;
  }
  fix_signs(N_, m_, Cfin, Xfin, part_, s_);
  column_residuals(N_, m_, Xfin, Cfin, lam_, res_, part_, s_);
}

// ---------------------------------------------------------------------------
// Iteration graphs
// ---------------------------------------------------------------------------
void Solver::iter_state(void** st) const {
  st[0] = C32_;
  st[1] = C32n_;
  st[2] = C64_;
  st[3] = C64n_;
  st[4] = Cdf_;
  st[5] = Cdfn_;
  st[6] = Gb_[0];
  st[7] = Gb_[1];
}

void Solver::set_iter_state(void* const* st) {
  C32_ = static_cast<float*>(st[0]);
  C32n_ = static_cast<float*>(st[1]);
  C64_ = static_cast<double*>(st[2]);
  C64n_ = static_cast<double*>(st[3]);
  Cdf_ = static_cast<float*>(st[4]);
  Cdfn_ = static_cast<float*>(st[5]);
  Gb_[0] = st[6];
  Gb_[1] = st[7];
}

template <typename F>
void Solver::run_iteration(int phase, F&& body) {
  void* pre[kStatePtrs];
  iter_state(pre);
  int k = -1;
  for (size_t i = 0; i < graphs_.size(); ++i)
    if (graphs_[i].phase == phase &&
        std::equal(pre, pre + kStatePtrs, graphs_[i].pre))
      k = (int)i;
  if (k < 0) {  // first run of this key: plain launches
    IterGraph g{};
    g.phase = phase;
    std::copy(pre, pre + kStatePtrs, g.pre);
    body();
    iter_state(g.post);
    graphs_.push_back(g);
    return;
  }
  IterGraph& g = graphs_[k];
  if (!g.exec) {  // second run: capture
    long long nk = 0;
    cudaGraph_t graph = nullptr;
    TRM_CUDA(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal));
    capture_launches(&nk);
    try {
      body();
    } catch (...) {
      capture_launches(nullptr);
      cudaStreamEndCapture(s_, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    capture_launches(nullptr);
    TRM_CUDA(cudaStreamEndCapture(s_, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    TRM_CUDA(e);
    g.kernels = nk;
    iter_state(g.post);
  } else {
    set_iter_state(g.post);
  }
  TRM_CUDA(cudaGraphLaunch(g.exec, s_));
  count_launches(g.kernels);
}

// ---------------------------------------------------------------------------
// Fig. TMFIG with the precision ladder.
// ---------------------------------------------------------------------------
int Solver::solve(double* lambda, double* E_G, double* C_out, int C_on_device,
                  const double* C0_host, trm_stats* stats) {
  const auto t_start = std::chrono::steady_clock::now();
  const long long launches0 = thread_launch_count();
  const size_t nm = (size_t)N_ * m_;
  history_.clear();
  if (C0_host)
    TRM_CUDA(cudaMemcpyAsync(C64_, C0_host, nm * 8, cudaMemcpyHostToDevice,
                             s_));
  else
    random_block(N_, m_, opt_.seed, C64_, s_);
  for (void* p : {Gb_[0], Gb_[1], Pb_})
    TRM_CUDA(cudaMemsetAsync(p, 0, nm * 8, s_));

  enum { PH_SP = 0, PH_MP2 = 1, PH_FP64 = 2 };
  const int prec = opt_.precision;
  int phase = prec == TRM_FP64 ? PH_FP64
              : prec == TRM_MP2 ? PH_MP2
                                : PH_SP;
  if (phase == PH_SP) {
    to_f32(C64_, C32_, (int64_t)nm, s_);
    orth_uniform<float>(C32_, C32n_);
  } else {
    orth_fp64(C64_, C64n_);
    if (phase == PH_MP2) c64_to_df();
  }
  set_restart();

  const int lag = std::max(1, std::min(opt_.lag, kRing / 2));
  int enq = 0, read = 0;
  int n_phase[3] = {0, 0, 0};
  int n_reorth = 0;
  bool converged = false;
  int status = TRM_OK;
  double r0 = -1.0, best = INFINITY;
  int best_at = 0;
  // Full SP has reached its floor when the energy (summed in FP64 from FP32
  // products, resolution ~1e-7 |E|) stops making new minima.
  double E_min = INFINITY;
  int E_min_at = 0;
  const int sp_floor_window = 30;
  int since_orth = 0, since_rr = 0, rescues = 0;
  // MP2 keeps C orthonormal between exact FP64 re-orthonormalizations only
  // to the FP32 accuracy of its overlap update, an error proportional to the
  // step alpha ||P|| and hence to the residual at the time. Re-orthonormalize
  // whenever the residual has dropped 100-fold since the last time (or after
  // reorth_every iterations), and rotate to the Ritz basis whenever it has
  // dropped 1000-fold (or after rr_every iterations), as Sec. 3 suggests.
  double r_orth = INFINITY, r_rr = INFINITY;
  // Full SP re-orthonormalizes (FP32) every sp_reorth iterations: its overlap
  // update drifts by about one FP32 rounding per step, and without the reset
  // that drift, times |lambda|, becomes the floor of the SP residual.
  const int sp_reorth = 20;
  int since_sp = 0;
  double E_last = NAN;
  // A phase has stalled when its best residual has not dropped by 30 % for
  // this many iterations (slow but steady CG on a small gap still passes).
  const int stall_window = 250;
  const bool trace = std::getenv("TRM_TRACE") != nullptr;

  // (the generalized problem swaps Y = S C too and runs without graphs)
  const bool graphs = opt_.graphs && s_ != nullptr && !prof.on && !has_S_;
  auto enqueue_one = [&]() {
    auto body = [&]() {
      if (phase == PH_SP) {
        float* G = static_cast<float*>(Gb_[0]);
        float* Gp = static_cast<float*>(Gb_[1]);
        iter_uniform<float, float>(C32_, C32n_, X32_, G, Gp,
                                   static_cast<float*>(Pb_),
                                   static_cast<float*>(HPb_));
        Gb_[0] = G;
        Gb_[1] = Gp;
      } else if (phase == PH_FP64) {
        double* G = static_cast<double*>(Gb_[0]);
        double* Gp = static_cast<double*>(Gb_[1]);
        iter_uniform<double, double>(C64_, C64n_, X64_, G, Gp,
                                     static_cast<double*>(Pb_),
                                     static_cast<double*>(HPb_));
        Gb_[0] = G;
        Gb_[1] = Gp;
      } else {
        iter_mp2();
      }
    };
    if (graphs)
      run_iteration(phase, body);
    else
      body();
    n_phase[phase == PH_SP ? 0 : 1]++;
    TRM_CUDA(cudaMemcpyAsync(&ring_[enq % kRing], sc_, sizeof(IterScalars),
                             cudaMemcpyDeviceToHost, s_));
    ring_phase_[enq % kRing] = phase;
    TRM_CUDA(cudaEventRecord(ev_[enq % kRing], s_));
    prof.cut();
    ++enq;
  };
  auto record = [&](int i) {
    history_.push_back({ring_[i % kRing], ring_phase_[i % kRing]});
  };
  auto drain = [&]() {  // wait for everything enqueued (and record it)
    TRM_CUDA(cudaStreamSynchronize(s_));
    for (int j = read; j < enq; ++j) record(j);
    read = enq;
  };

  while (true) {
    if (enq >= opt_.max_iter) {
      status = TRM_ENOCONV;
      break;
    }
    enqueue_one();
    if (enq - read <= lag) continue;
    const int i = read++;
    TRM_CUDA(cudaEventSynchronize(ev_[i % kRing]));
    if (prof.on) prof.resolve();
    const IterScalars v = ring_[i % kRing];
    record(i);
    E_last = v.E;
    if (trace)
      std::fprintf(stderr,
                   "trm it %5d ph %d E %.15e r %.3e alpha %.3e gamma %.3e "
                   "c2 %.3e dE %.3e st %d\n",
                   i, phase, v.E, v.rms, v.alpha, v.gamma, v.c2, v.dE,
                   v.status);
    if (!std::isfinite(v.E) || !std::isfinite(v.rms)) {
      status = TRM_ENOCONV;
      last_error = "non-finite energy or residual at iteration " +
                   std::to_string(i);
      break;
    }
    if (v.status & 2) {  // a bounded device wait gave up
      status = TRM_ETIMEOUT;
      last_error = "a tensor-core pipeline wait timed out";
      break;
    }
    if (v.status & 1) {  // overlap not positive definite: re-orthonormalise
      drain();
      if (++rescues > 5) {
        status = TRM_ENOTPD;
        last_error = "overlap matrix not positive definite";
        break;
      }
      if (phase == PH_SP) {
        orth_uniform<float>(C32_, C32n_);
      } else if (phase == PH_MP2) {
        df_to_c64();
        orth_fp64(C64_, C64n_);
        c64_to_df();
      } else {
        orth_fp64(C64_, C64n_);
      }
      set_restart();
      continue;
    }
    if (r0 < 0.0) r0 = v.rms;
    if (v.rms < 0.7 * best) {
      best = v.rms;
      best_at = i;
    }
    if (phase != PH_SP || prec == TRM_FULL_SP) {
      if (v.rms <= tol_) {
        converged = true;
        break;
      }
    }
    if (v.E < E_min - 1e-7 * std::fabs(v.E)) {
      E_min = v.E;
      E_min_at = i;
    }
    if (phase == PH_SP) {
      if (++since_sp >= sp_reorth) {
        orth_uniform<float>(C32_, C32n_);
        since_sp = 0;
      }
      const bool small = v.rms <= opt_.switch_tol[0] * r0;
      const bool stalled = i - best_at > stall_window ||
                           (prec != TRM_FULL_SP && i - E_min_at > sp_floor_window);
      if (prec == TRM_FULL_SP) {
        if (stalled) {
          status = TRM_ENOCONV;
          last_error = "full SP stagnated above the tolerance";
          break;
        }
      } else if (small || stalled) {
        drain();
        to_f64(C32_, C64_, (int64_t)nm, s_);
        orth_fp64(C64_, C64n_);  // (recomputes Y = S C in FP64)
        rr_rotate_fp64();
        // the generalized problem goes on in FP64 (its double-float MP2
        // would need Y and S C as FP32 pairs)
        if (!has_S_) c64_to_df();
        set_restart();
        phase = has_S_ ? PH_FP64 : PH_MP2;
        best = INFINITY;
        best_at = enq;
        since_orth = since_rr = 0;
        r_orth = r_rr = v.rms;
        continue;
      }
    } else {
      if (i - best_at > stall_window) {
        // stagnation: rotate to the Ritz basis and restart CG
        drain();
        if (++rescues > 5) {
          status = TRM_ENOCONV;
          last_error = "stagnated above the tolerance";
          break;
        }
        if (phase == PH_MP2) df_to_c64();
        orth_fp64(C64_, C64n_);
        rr_rotate_fp64();
        if (phase == PH_MP2) c64_to_df();
        set_restart();
        best = INFINITY;
        best_at = enq;
        continue;
      }
      if (phase == PH_MP2) {
        ++since_orth;
        ++since_rr;
        if (!std::isfinite(r_orth)) r_orth = r_rr = v.rms;
        const bool rr = v.rms < 1e-3 * r_rr ||
                        (opt_.rr_every > 0 && since_rr >= opt_.rr_every);
        const bool ro = v.rms < 1e-2 * r_orth ||
                        (opt_.reorth_every > 0 && since_orth >= opt_.reorth_every);
        if (rr || ro) {
          df_to_c64();
          orth_fp64(C64_, C64n_);
          ++n_reorth;
          since_orth = 0;
          r_orth = v.rms;
          if (rr) {
            rr_rotate_fp64();
            set_restart();
            since_rr = 0;
            r_rr = v.rms;
          }
          c64_to_df();
        }
      }
    }
  }
  drain();
  if (prof.on) prof.resolve();
  if (phase == PH_SP) to_f64(C32_, C64_, (int64_t)nm, s_);
  if (phase == PH_MP2) df_to_c64();
  double* Cfin = C64n_;
  double* Xfin = static_cast<double*>(Gb_[0]);
  final_rr(C64_, Cfin, Xfin);
  std::vector<double> lam(m_), res(m_);
  TRM_CUDA(cudaMemcpyAsync(lam.data(), lam_, m_ * 8, cudaMemcpyDeviceToHost,
                           s_));
  TRM_CUDA(cudaMemcpyAsync(res.data(), res_, m_ * 8, cudaMemcpyDeviceToHost,
                           s_));
  if (C_out)
    TRM_CUDA(cudaMemcpyAsync(C_out, Cfin, nm * 8,
                             C_on_device ? cudaMemcpyDeviceToDevice
                                         : cudaMemcpyDeviceToHost,
                             s_));
  TRM_CUDA(cudaStreamSynchronize(s_));
  if (lambda) std::memcpy(lambda, lam.data(), m_ * 8);
  if (E_G) *E_G = neumaier_sum(lam.data(), m_);
  if (stats) {
    double ss = 0.0, mx = 0.0;
    for (double r : res) {
      ss += r * r;
      mx = std::max(mx, r);
    }
    stats->iterations = enq;
    stats->iterations_phase[0] = n_phase[0];
    stats->iterations_phase[1] = n_phase[1];
    stats->iterations_phase[2] = n_reorth;
    stats->converged = converged ? 1 : 0;
    stats->rms_residual = std::sqrt(ss / m_);
    stats->max_residual = mx;
    stats->E_last = E_last;
    stats->launches = thread_launch_count() - launches0;
    stats->seconds = std::chrono::duration<double>(
                         std::chrono::steady_clock::now() - t_start)
                         .count();
  }
  if (status == TRM_OK && !converged) status = TRM_ENOCONV;
  return status;
}

// ---------------------------------------------------------------------------
// Step operations
// ---------------------------------------------------------------------------
void Solver::apply(int din, const void* in, int dout, void* out, int ncols) {
  if (din == TRM_F32 && dout == TRM_F32)
    apply_h(op_, static_cast<const float*>(in), static_cast<float*>(out),
            ncols, s_);
  else if (din == TRM_F64 && dout == TRM_F64)
    apply_h(op_, static_cast<const double*>(in), static_cast<double*>(out),
            ncols, s_);
  else
    throw Error(-1, "apply: unsupported dtype combination");
  TRM_CUDA(cudaStreamSynchronize(s_));
}

void Solver::energy_gradient(const double* C, double* E, double* HD,
                             double* Hprime, void* G, int G_dtype,
                             int zdiag) {
  apply_h(op_, C, X64_, m_, s_);
  energy_diag<double>(N_, m_, C, X64_, HD_, sc_, part_, s_);
  set_restart();
  if (G_dtype == TRM_F64) {
    xprime<double>(N_, m_, C, X64_, HD_, nullptr, nullptr, s_);
    Blocks<double> b;
    b.p[0] = X64_;
    b.cols = m_;
    b.count = 1;
    gram<double>(N_, m_, C, b, Hp_, part_, part_cap_, s_, &sc_->status);
    if (zdiag) zero_diag(m_, Hp_, s_);
    gradient<double>(N_, m_, C, X64_, Hp_, static_cast<double*>(G), nullptr,
                     nullptr, nullptr, sc_, part_, part_cap_, s_);
  } else if (G_dtype == TRM_F32) {
    xprime<double>(N_, m_, C, X64_, HD_, C32_, X32_, s_, false);
    Blocks<float> b;
    b.p[0] = X32_;
    b.cols = m_;
    b.count = 1;
    gram<float>(N_, m_, C32_, b, Hp_, part_, part_cap_, s_, &sc_->status);
    if (zdiag) zero_diag(m_, Hp_, s_);
    gradient<float>(N_, m_, C32_, X32_, Hp_, static_cast<float*>(G), nullptr,
                    nullptr, nullptr, sc_, part_, part_cap_, s_, &tw_);
  } else {
    throw Error(-1, "energy_gradient: G_dtype must be TRM_F32 or TRM_F64");
  }
  if (HD)
    TRM_CUDA(cudaMemcpyAsync(HD, HD_, m_ * 8, cudaMemcpyDeviceToDevice, s_));
  if (Hprime)
    TRM_CUDA(cudaMemcpyAsync(Hprime, Hp_, (size_t)m_ * m_ * 8,
                             cudaMemcpyDeviceToDevice, s_));
  IterScalars v;
  read_scalars(&v);
  if (v.status & 2) throw Error(-6, "a bounded device wait gave up");
  if (E) *E = v.E;
}

void Solver::set_block(const double* C_dev) {
  TRM_CUDA(cudaMemcpyAsync(C64_, C_dev, (size_t)N_ * m_ * 8,
                           cudaMemcpyDeviceToDevice, s_));
  for (void* p : {Gb_[0], Gb_[1], Pb_})
    TRM_CUDA(cudaMemsetAsync(p, 0, (size_t)N_ * m_ * 8, s_));
  set_restart();
  TRM_CUDA(cudaStreamSynchronize(s_));
}

void Solver::get_block(double* C_dev) {
  TRM_CUDA(cudaMemcpyAsync(C_dev, C64_, (size_t)N_ * m_ * 8,
                           cudaMemcpyDeviceToDevice, s_));
  TRM_CUDA(cudaStreamSynchronize(s_));
}

void Solver::iterate(int mode, int restart, double* E, double* rms,
                     double* alpha) {
  const size_t nm = (size_t)N_ * m_;
  if (restart) {
    for (void* p : {Gb_[0], Gb_[1], Pb_})
      TRM_CUDA(cudaMemsetAsync(p, 0, nm * 8, s_));
    set_restart();
  }
  if (mode == TRM_FP64) {
    double* G = static_cast<double*>(Gb_[0]);
    double* Gp = static_cast<double*>(Gb_[1]);
    iter_uniform<double, double>(C64_, C64n_, X64_, G, Gp,
                                 static_cast<double*>(Pb_),
                                 static_cast<double*>(HPb_));
    Gb_[0] = G;
    Gb_[1] = Gp;
  } else if (mode == TRM_FULL_SP) {
    to_f32(C64_, C32_, (int64_t)nm, s_);
    float* G = static_cast<float*>(Gb_[0]);
    float* Gp = static_cast<float*>(Gb_[1]);
    iter_uniform<float, float>(C32_, C32n_, X32_, G, Gp,
                               static_cast<float*>(Pb_),
                               static_cast<float*>(HPb_));
    Gb_[0] = G;
    Gb_[1] = Gp;
    to_f64(C32_, C64_, (int64_t)nm, s_);
  } else if (mode == TRM_MP2) {
    c64_to_df();
    iter_mp2();
    df_to_c64();
  } else {
    throw Error(-1, "iterate: mode must be TRM_FP64, TRM_FULL_SP or TRM_MP2");
  }
  IterScalars v;
  read_scalars(&v);
  if (E) *E = v.E;
  if (rms) *rms = v.rms;
  if (alpha) *alpha = v.alpha;
  if (v.status & 2) throw Error(-6, "a bounded device wait gave up");
  if (v.status & 1) throw Error(-3, "overlap matrix not positive definite");
}

void Solver::rayleigh_ritz(double* C_dev, double* lambda_host,
                           double* res_host) {
  double* Xfin = static_cast<double*>(Gb_[0]);
  final_rr(C_dev, C64n_, Xfin);
  TRM_CUDA(cudaMemcpyAsync(C_dev, C64n_, (size_t)N_ * m_ * 8,
                           cudaMemcpyDeviceToDevice, s_));
  if (lambda_host)
    TRM_CUDA(cudaMemcpyAsync(lambda_host, lam_, m_ * 8, cudaMemcpyDeviceToHost,
                             s_));
  if (res_host)
    TRM_CUDA(cudaMemcpyAsync(res_host, res_, m_ * 8, cudaMemcpyDeviceToHost,
                             s_));
  TRM_CUDA(cudaStreamSynchronize(s_));
  for (void* p : {Gb_[0], Gb_[1], Pb_})
    TRM_CUDA(cudaMemsetAsync(p, 0, (size_t)N_ * m_ * 8, s_));
  set_restart();
}

template void Solver::orth_uniform<float>(float*&, float*&);
template void Solver::orth_uniform<double>(double*&, double*&);

}  // namespace trm
