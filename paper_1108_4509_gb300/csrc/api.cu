// C ABI of the library (include/trm.h): argument checks, status codes and
// error messages around the solver. Nothing is thrown across this boundary.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>

#include "solver.cuh"

struct trm_ctx {
  std::unique_ptr<trm::Solver> solver;
  std::string err;
};

namespace {

thread_local std::string g_err;

int fail(trm_ctx* h, int status, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return status;
}

template <class F>
trm_status guarded(trm_ctx* h, F&& f) {
  // An exception that leaves library code may have skipped the end of a
  // launch-counting scope (an autotuner's timing launches): no scope
  // outlives a call, so the thread's count sink is cleared here.
  try {
    return static_cast<trm_status>(f());
  } catch (const trm::Error& e) {
    trm::capture_launches(nullptr);
    return static_cast<trm_status>(fail(h, e.status, e.what()));
  } catch (const std::bad_alloc&) {
    trm::capture_launches(nullptr);
    return static_cast<trm_status>(fail(h, TRM_ENOMEM, "host allocation failed"));
  } catch (const std::exception& e) {
    trm::capture_launches(nullptr);
    return static_cast<trm_status>(fail(h, TRM_ECUDA, e.what()));
  } catch (...) {
    trm::capture_launches(nullptr);
    return static_cast<trm_status>(fail(h, TRM_ECUDA, "unknown error"));
  }
}

bool valid_options(const trm_options& o, std::string* why) {
  if (o.precision < TRM_FP64 || o.precision > TRM_MIXED) {
    *why = "precision must be one of TRM_FP64..TRM_MIXED";
    return false;
  }
  if (o.precision == TRM_MP1) {
    *why = "TRM_MP1 is not available in this build";
    return false;
  }
  if (o.precond != 0 && o.precond != 1) {
    *why = "precond must be 0 or 1";
    return false;
  }
  if (o.max_iter < 1) {
    *why = "max_iter must be >= 1";
    return false;
  }
  if (!(o.switch_tol[0] >= 0.0)) {
    *why = "switch_tol[0] must be >= 0";
    return false;
  }
  return true;
}

trm_options resolve(const trm_options* opt) {
  trm_options o;
  trm_default_options(&o);
  if (opt) o = *opt;
  if (o.lag < 1) o.lag = 1;
  return o;
}

}  // namespace

namespace trm {
void set_global_error(const std::string& msg) { g_err = msg; }
}  // namespace trm

extern "C" {

trm_status trm_default_options(trm_options* opt) {
  if (!opt) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "opt is NULL"));
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = TRM_MIXED;
  opt->precond = 0;
  opt->max_iter = 20000;
  opt->seed = 0;
  opt->switch_tol[0] = 1e-5;
  opt->switch_tol[1] = 0.0;
  opt->reorth_every = 400;
  opt->rr_every = 0;
  opt->lag = 2;
  opt->graphs = 1;
  opt->stream = nullptr;
  return TRM_OK;
}

trm_status trm_create_stencil(trm_handle* out, int nx, int ny, int nz,
                              int order, double h, const double* V, int m,
                              double tol, const trm_options* opt) {
  if (!out) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "out is NULL"));
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "grid dimensions must be >= 1"));
  if (order != 2 && order != 4)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "order must be 2 or 4"));
  if (!(h > 0.0) || !std::isfinite(h))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "h must be positive"));
  const int64_t N = (int64_t)nx * ny * nz;
  if (m < 1 || m >= N || m > 1024)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "need 1 <= m < N and m <= 1024"));
  if (!(tol >= 0.0))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "tol must be >= 0"));
  trm_options o = resolve(opt);
  std::string why;
  if (!valid_options(o, &why)) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, why));
  auto ctx = std::make_unique<trm_ctx>();
  trm_status st = guarded(nullptr, [&]() {
    ctx->solver = std::make_unique<trm::Solver>(N, m, tol, o);
    ctx->solver->init_stencil(nx, ny, nz, order, h, V);
    return TRM_OK;
  });
  if (st != TRM_OK) return st;
  *out = ctx.release();
  return TRM_OK;
}

trm_status trm_create_csr(trm_handle* out, int64_t N, const int32_t* rowptr,
                          const int32_t* cols, const void* vals,
                          int vals_dtype, int m, double tol,
                          const trm_options* opt) {
  if (!out) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "out is NULL"));
  *out = nullptr;
  if (N < 2 || N >= ((int64_t)1 << 31))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "need 2 <= N < 2^31"));
  if (!rowptr || !cols || !vals)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "CSR arrays must be non-NULL"));
  if (vals_dtype != TRM_F32 && vals_dtype != TRM_F64)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "vals_dtype must be TRM_F32 or TRM_F64"));
  if (m < 1 || m >= N || m > 1024)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "need 1 <= m < N and m <= 1024"));
  if (!(tol >= 0.0))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "tol must be >= 0"));
  if (rowptr[0] != 0)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "rowptr[0] must be 0"));
  for (int64_t r = 0; r < N; ++r) {
    if (rowptr[r + 1] < rowptr[r])
      return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "rowptr must be non-decreasing"));
  }
  const int64_t nnz = rowptr[N];
  for (int64_t k = 0; k < nnz; ++k) {
    if (cols[k] < 0 || cols[k] >= N)
      return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "column index out of range"));
  }
  trm_options o = resolve(opt);
  std::string why;
  if (!valid_options(o, &why)) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, why));
  auto ctx = std::make_unique<trm_ctx>();
  trm_status st = guarded(nullptr, [&]() {
    ctx->solver = std::make_unique<trm::Solver>(N, m, tol, o);
    ctx->solver->init_csr(rowptr, cols, vals, vals_dtype == TRM_F64);
    return TRM_OK;
  });
  if (st != TRM_OK) return st;
  *out = ctx.release();
  return TRM_OK;
}

trm_status trm_set_overlap_csr(trm_handle h, const int32_t* rowptr,
                               const int32_t* cols, const double* vals) {
  if (!h) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "handle is NULL"));
  if (!rowptr || !cols || !vals)
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "CSR arrays must be non-NULL"));
  if (h->solver->precision() == TRM_MP2)
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "the generalized problem runs in the TRM_FP64, TRM_MIXED and TRM_FULL_SP modes (MP2's double-float blocks do not carry S C)"));
  const int64_t N = h->solver->N();
  if (rowptr[0] != 0)
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "rowptr[0] must be 0"));
  for (int64_t r = 0; r < N; ++r) {
    if (rowptr[r + 1] < rowptr[r])
      return static_cast<trm_status>(fail(h, TRM_EINVAL, "rowptr must be non-decreasing"));
  }
  for (int64_t r = 0; r < N; ++r) {
    double d = 0.0;
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      if (cols[k] < 0 || cols[k] >= N)
        return static_cast<trm_status>(fail(h, TRM_EINVAL, "column index out of range"));
      if (cols[k] == r) d += vals[k];
    }
    if (!(d > 0.0))
      return static_cast<trm_status>(fail(h, TRM_EINVAL, "S must have a positive diagonal"));
  }
  return guarded(h, [&]() {
    h->solver->init_overlap(rowptr, cols, vals);
    return TRM_OK;
  });
}

trm_status trm_solve(trm_handle h, double* lambda, double* E_G, double* C,
                     int C_on_device, const double* C0, trm_stats* stats) {
  if (!h) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "handle is NULL"));
  return guarded(h, [&]() {
    h->solver->last_error.clear();
    int st = h->solver->solve(lambda, E_G, C, C_on_device, C0, stats);
    if (st != TRM_OK)
      fail(h, st, h->solver->last_error.empty() ? "did not converge"
                                                : h->solver->last_error);
    return st;
  });
}

int trm_history(trm_handle h, trm_iter_record* out, int cap) {
  if (!h || cap < 0 || (cap > 0 && !out))
    return fail(h, TRM_EINVAL, "invalid arguments to trm_history");
  const auto& hist = h->solver->history();
  const int n = (int)hist.size();
  for (int i = 0; i < n && i < cap; ++i) {
    const auto& r = hist[i];
    out[i].E = r.v.E;
    out[i].rms = r.v.rms;
    out[i].alpha = r.v.alpha;
    out[i].gamma = r.v.gamma;
    out[i].phase = r.phase;
    out[i].restart = r.v.restart;
  }
  return n;
}

trm_status trm_destroy(trm_handle h) {
  if (!h) return TRM_OK;
  return guarded(nullptr, [&]() {
    delete h;
    return TRM_OK;
  });
}

const char* trm_strerror(trm_status s) {
  switch (s) {
    case TRM_OK: return "success";
    case TRM_EINVAL: return "invalid argument";
    case TRM_ENOMEM: return "out of device memory";
    case TRM_ENOTPD: return "overlap matrix not positive definite";
    case TRM_ENOCONV: return "no convergence within max_iter";
    case TRM_ECUDA: return "CUDA error";
    case TRM_ETIMEOUT: return "device wait timed out";
    case TRM_EGAP: return "spectral gap test failed";
  }
  return "unknown status";
}

const char* trm_last_error(trm_handle h) {
  return h ? h->err.c_str() : g_err.c_str();
}

const char* trm_last_global_error(void) { return g_err.c_str(); }

int64_t trm_dim(trm_handle h) { return h ? h->solver->N() : -1; }

trm_status trm_apply_h(trm_handle h, int dtype_in, const void* C,
                       int dtype_out, void* X, int ncols) {
  if (!h || !C || !X || ncols < 0)
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "invalid arguments to trm_apply_h"));
  return guarded(h, [&]() {
    h->solver->apply(dtype_in, C, dtype_out, X, ncols);
    return TRM_OK;
  });
}

trm_status trm_energy_gradient(trm_handle h, const double* C, double* E,
                               double* HD, double* Hprime, void* G,
                               int G_dtype, int zero_diag) {
  if (!h || !C || !G)
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "invalid arguments to trm_energy_gradient"));
  if (h && h->solver->generalized())
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "the step operations cover the standard problem; a handle with an overlap S solves with trm_solve"));
  return guarded(h, [&]() {
    h->solver->energy_gradient(C, E, HD, Hprime, G, G_dtype, zero_diag);
    return TRM_OK;
  });
}

trm_status trm_gram(int64_t N, int m, int n, int dtype, const void* A,
                    const void* B, double* out, void* stream) {
  if (N < 1 || m < 1 || n < 1 || !A || !B || !out ||
      (dtype != TRM_F32 && dtype != TRM_F64))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "invalid arguments to trm_gram"));
  return guarded(nullptr, [&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t cap = trm::gram_partials_doubles(N, m, n);
    double* part = nullptr;
    TRM_CUDA(cudaMallocAsync(&part, (cap + 1) * sizeof(double), s));
    int* err = reinterpret_cast<int*>(part + cap);
    int herr = 0;
    try {
      TRM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      if (dtype == TRM_F32) {
        trm::Blocks<float> b;
        b.p[0] = static_cast<const float*>(B);
        b.cols = n;
        b.count = 1;
        trm::gram<float>(N, m, static_cast<const float*>(A), b, out, part, cap,
                         s, err);
      } else {
        trm::Blocks<double> b;
        b.p[0] = static_cast<const double*>(B);
        b.cols = n;
        b.count = 1;
        trm::gram<double>(N, m, static_cast<const double*>(A), b, out, part,
                          cap, s, err);
      }
      TRM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost,
                               s));
    } catch (...) {
      cudaFreeAsync(part, s);
      throw;
    }
    TRM_CUDA(cudaFreeAsync(part, s));
    TRM_CUDA(cudaStreamSynchronize(s));
    if (herr & 2)
      return fail(nullptr, TRM_ETIMEOUT, "trm_gram: a device wait timed out");
    return (int)TRM_OK;
  });
}

trm_status trm_orthonormalize(int64_t N, int m, double* C, void* stream) {
  if (N < 1 || m < 1 || m > 1024 || m > N || !C)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "invalid arguments to trm_orthonormalize"));
  return guarded(nullptr, [&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t mm = (size_t)m * m;
    const size_t cap = trm::gram_partials_doubles(N, m, m);
    const size_t cw = trm::chol_work_elems(m);
    const size_t bytes = (cap + 3 * mm + cw + (size_t)N * m) * sizeof(double) +
                         sizeof(trm::IterScalars);
    char* w = nullptr;
    TRM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&w), bytes, s));
    double* part = reinterpret_cast<double*>(w);
    double* S = part + cap;
    double* Linv = S + mm;
    double* R = Linv + mm;
    double* gw = R + mm;        // padded factorisation workspace
    double* Cn = gw + cw;
    auto* sc = reinterpret_cast<trm::IterScalars*>(Cn + (size_t)N * m);
    int status = 0;
    try {
      TRM_CUDA(cudaMemsetAsync(sc, 0, sizeof(trm::IterScalars), s));
      trm::Blocks<double> b;
      b.p[0] = C;
      b.cols = m;
      b.count = 1;
      trm::gram<double>(N, m, C, b, S, part, cap, s);
      trm::chol_inv<double>(m, S, Linv, R, sc, gw, s);
      trm::rotate<double, double>(N, m, C, nullptr, R, Cn, nullptr, s);
      TRM_CUDA(cudaMemcpyAsync(C, Cn, (size_t)N * m * 8,
                               cudaMemcpyDeviceToDevice, s));
      TRM_CUDA(cudaMemcpyAsync(&status, &sc->status, sizeof(int),
                               cudaMemcpyDeviceToHost, s));
      TRM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      cudaFreeAsync(w, s);
      throw;
    }
    TRM_CUDA(cudaFreeAsync(w, s));
    TRM_CUDA(cudaStreamSynchronize(s));
    if (status & 1)
      return fail(nullptr, TRM_ENOTPD, "C^T C is not positive definite");
    return (int)TRM_OK;
  });
}

trm_status trm_extrapolate(int64_t N, int m, const double* C_prev,
                           const double* C_cur, double alpha, double* C_next,
                           void* stream) {
  if (N < 1 || m < 1 || m > 1024 || m > N || !C_prev || !C_cur || !C_next ||
      C_next == C_prev || C_next == C_cur || !(alpha == alpha))
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "invalid arguments to trm_extrapolate"));
  return guarded(nullptr, [&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t mm = (size_t)m * m;
    const size_t Nm = (size_t)N * m;
    const size_t cap = trm::gram_partials_doubles(N, m, m);
    const size_t pw = trm::polar_work_doubles(m);
    const size_t cw = trm::chol_work_elems(m);
    const size_t bytes = (cap + 5 * mm + pw + cw + Nm) * sizeof(double) +
                         sizeof(trm::IterScalars) + 2 * sizeof(int);
    char* w = nullptr;
    TRM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&w), bytes, s));
    double* part = reinterpret_cast<double*>(w);
    double* M = part + cap;
    double* U = M + mm;
    double* S = U + mm;
    double* Linv = S + mm;
    double* R = Linv + mm;
    double* pwork = R + mm;
    double* gw = pwork + pw;
    double* Y = gw + cw;
    auto* sc = reinterpret_cast<trm::IterScalars*>(Y + Nm);
    int* info = reinterpret_cast<int*>(sc + 1);  // [eig sweeps, polar status]
    int flags[2] = {0, 0};
    int status = 0;
    try {
      TRM_CUDA(cudaMemsetAsync(sc, 0, sizeof(trm::IterScalars) + 2 * sizeof(int), s));
      // align C_prev to C_cur: U = polar(C_prev^T C_cur)
      trm::Blocks<double> b;
      b.p[0] = C_cur;
      b.cols = m;
      b.count = 1;
      trm::gram<double>(N, m, C_prev, b, M, part, cap, s);
      trm::polar_factor(m, M, U, pwork, info + 1, info, s);
      TRM_CUDA(cudaMemcpyAsync(flags, info, 2 * sizeof(int),
                               cudaMemcpyDeviceToHost, s));
      TRM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      cudaFreeAsync(w, s);
      throw;
    }
    if (flags[1] & 1) {
      TRM_CUDA(cudaFreeAsync(w, s));
      TRM_CUDA(cudaStreamSynchronize(s));
      return fail(nullptr, TRM_ENOTPD,
                  "C_prev^T C_cur is singular: the subspaces are too far "
                  "apart to align");
    }
    try {
      trm::Blocks<double> b;
      b.cols = m;
      b.count = 1;
      // C_next = (1 + alpha) C_cur - alpha C_prev U
      trm::mult(N, m, m, C_prev, U, Y, s);
      trm::lin_comb((int64_t)Nm, 1.0 + alpha, C_cur, -alpha, Y, C_next, s);
      // Fig. ONFIG: C_next <- C_next L^{-T}
      b.p[0] = C_next;
      trm::gram<double>(N, m, C_next, b, S, part, cap, s);
      trm::chol_inv<double>(m, S, Linv, R, sc, gw, s);
      trm::rotate<double, double>(N, m, C_next, nullptr, R, Y, nullptr, s);
      TRM_CUDA(cudaMemcpyAsync(C_next, Y, Nm * 8, cudaMemcpyDeviceToDevice, s));
      TRM_CUDA(cudaMemcpyAsync(&status, &sc->status, sizeof(int),
                               cudaMemcpyDeviceToHost, s));
      TRM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      cudaFreeAsync(w, s);
      throw;
    }
    TRM_CUDA(cudaFreeAsync(w, s));
    TRM_CUDA(cudaStreamSynchronize(s));
    if (status & 1)
      return fail(nullptr, TRM_ENOTPD, "C_next^T C_next is not positive definite");
    return (int)TRM_OK;
  });
}

trm_status trm_set_block(trm_handle h, const double* C_device) {
  if (!h || !C_device) return static_cast<trm_status>(fail(h, TRM_EINVAL, "invalid arguments"));
  if (h && h->solver->generalized())
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "the step operations cover the standard problem; a handle with an overlap S solves with trm_solve"));
  return guarded(h, [&]() {
    h->solver->set_block(C_device);
    return TRM_OK;
  });
}

trm_status trm_get_block(trm_handle h, double* C_device) {
  if (!h || !C_device) return static_cast<trm_status>(fail(h, TRM_EINVAL, "invalid arguments"));
  return guarded(h, [&]() {
    h->solver->get_block(C_device);
    return TRM_OK;
  });
}

trm_status trm_iterate(trm_handle h, int mode, int restart, double* E_out,
                       double* rms_out, double* alpha_out) {
  if (!h) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "handle is NULL"));
  if (h && h->solver->generalized())
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "the step operations cover the standard problem; a handle with an overlap S solves with trm_solve"));
  return guarded(h, [&]() {
    h->solver->iterate(mode, restart, E_out, rms_out, alpha_out);
    return TRM_OK;
  });
}

trm_status trm_rayleigh_ritz(trm_handle h, double* C, double* lambda,
                             double* residuals) {
  if (!h || !C) return static_cast<trm_status>(fail(h, TRM_EINVAL, "invalid arguments"));
  if (h && h->solver->generalized())
    return static_cast<trm_status>(fail(h, TRM_EINVAL, "the step operations cover the standard problem; a handle with an overlap S solves with trm_solve"));
  return guarded(h, [&]() {
    h->solver->rayleigh_ritz(C, lambda, residuals);
    return TRM_OK;
  });
}

trm_status trm_profile(trm_handle h, int enable) {
  if (!h) return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "handle is NULL"));
  return guarded(h, [&]() {
    h->solver->prof.reset();
    h->solver->prof.on = enable != 0;
    return TRM_OK;
  });
}

int trm_profile_read(trm_handle h, trm_kernel_stats* out, int max) {
  if (!h) return fail(nullptr, TRM_EINVAL, "handle is NULL");
  if (out && max > 0) {
    const trm::Profiler& p = h->solver->prof;
    for (int k = 0; k < trm::KC_COUNT && k < max; ++k) {
      std::memset(out[k].name, 0, sizeof(out[k].name));
      std::strncpy(out[k].name, trm::kClassNames[k], sizeof(out[k].name) - 1);
      out[k].ms = p.ms[k];
      out[k].launches = p.launches[k];
      out[k].flops = p.flops[k];
      out[k].bytes = p.bytes[k];
    }
  }
  return trm::KC_COUNT;
}

long long trm_launch_count(void) { return trm::launch_count(); }

trm_status trm_random_block(int64_t N, int m, uint64_t seed, double* C,
                            void* stream) {
  if (N < 1 || m < 1 || !C)
    return static_cast<trm_status>(fail(nullptr, TRM_EINVAL, "invalid arguments to trm_random_block"));
  return guarded(nullptr, [&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    trm::random_block(N, m, seed, C, s);
    TRM_CUDA(cudaStreamSynchronize(s));
    return TRM_OK;
  });
}

}  // extern "C"
