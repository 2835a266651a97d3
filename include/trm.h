/*
 * trm.h - C ABI of the GB300 (sm_103a) trace-minimization eigensolver.
 *
 * Computes the m lowest eigenvalues lambda_1..lambda_m of a large sparse
 * symmetric matrix H, their sum E_G and an orthonormal basis C of the
 * corresponding invariant subspace, by minimising E(C) = trace(C^T H C)
 * subject to C^T C = I_m with nonlinear conjugate gradients (Tsuchida and Choe,
 * "Iterative diagonalization of symmetric matrices in mixed precision",
 * Sec. 2.1, Eqs. TRHEQ/CIJEQ, Fig. TMFIG), in full FP64 or in the mixed
 * precision of Sec. 2.2 (MP2, full SP, and a ladder full SP -> MP2 ->
 * FP64 Rayleigh-Ritz; MP1 is not offered).
 *
 * Conventions used by every entry point:
 *  - N x m blocks are column-major with leading dimension N (column j of C is
 *    the contiguous range C[j*N .. j*N + N-1]); m x m matrices are
 *    column-major with leading dimension m.
 *  - "device" pointers are CUDA global-memory addresses of the current
 *    device; "host" pointers are ordinary CPU memory (pageable or pinned).
 *  - Inputs are owned by the caller and are copied (create) or only read
 *    (step operations); the library never frees a caller pointer.
 *  - No entry point throws, exits or traps: every failure is returned as a
 *    negative trm_status, with a message from trm_last_error() where a
 *    handle exists, or trm_last_global_error() otherwise.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef TRM_H
#define TRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trm_ctx* trm_handle;

typedef enum {
  TRM_OK = 0,
  TRM_EINVAL = -1,   /* invalid argument (sizes, pointers, options) */
  TRM_ENOMEM = -2,   /* device memory for the solve could not be allocated */
  TRM_ENOTPD = -3,   /* an overlap matrix C^T C was not positive definite */
  TRM_ENOCONV = -4,  /* max_iter reached; outputs hold the best iterate */
  TRM_ECUDA = -5,    /* a CUDA runtime call failed */
  TRM_ETIMEOUT = -6, /* a bounded device wait gave up */
  TRM_EGAP = -7      /* reserved: gap test failed */
} trm_status;

/* Precision modes (Sec. 2.2). */
typedef enum {
  TRM_FP64 = 0,    /* "full DP": every operation in FP64 */
  TRM_MP1 = 1,     /* reserved: Sec. 2.2's MP1 (G, P stored FP32, split
                      rotation) is not offered -- its O(m^2 N) Grams stay
                      FP64, the slowest part on this GPU; create returns
                      TRM_EINVAL */
  TRM_MP2 = 2,     /* MP2: G, P stored FP32, split rotation C L_D + C L',
                      and the two O(m^2 N) gradient GEMMs in FP32 */
  TRM_FULL_SP = 3, /* "full SP": all block work in FP32 */
  TRM_MIXED = 4    /* full SP until stagnation, then MP2, then FP64 Rayleigh-Ritz */
} trm_precision;

/* Element types of caller buffers in the step operations. */
typedef enum { TRM_F32 = 0, TRM_F64 = 1 } trm_dtype;

typedef struct {
  int precision;        /* trm_precision; default TRM_MIXED */
  int precond;          /* 0: M = I; 1: diagonal M = diag(1/(H_jj - sigma)),
                           sigma = min_k H_kk - 1 (Eq. PCEQ). Default 0 */
  int max_iter;         /* iteration cap over all phases; default 20000 */
  uint64_t seed;        /* random C0 = splitmix64 block of this seed */
  double switch_tol[2]; /* [0]: leave full SP when the RMS residual stops
                           improving or falls below switch_tol[0]*r_0;
                           [1]: reserved. Defaults 1e-5, 0 */
  int reorth_every;     /* MP2 phase: exact FP64 re-orthonormalization at
                           least every this many iterations, and whenever
                           the residual has dropped 100-fold since the
                           last one; default 400; 0: residual rule only */
  int rr_every;         /* MP2 phase: subspace rotation diagonalising
                           C^T H C (Sec. 3) at least every this many
                           iterations, and whenever the residual has
                           dropped 1000-fold; default 0: residual rule */
  int lag;              /* iterations the host may run ahead of the
                           convergence flags it has read; default 2 */
  void* stream;         /* cudaStream_t for all work; NULL = default stream */
  int graphs;           /* 1 (default): after its first run, each kind of
                           block iteration is captured once as a CUDA graph
                           and replayed (fewer launch gaps; same kernels,
                           same results); needs a non-NULL stream and is
                           off while trm_profile is on. 0: plain launches */
} trm_options;

typedef struct {
  int iterations;           /* total iterations */
  int iterations_phase[3];  /* full SP, MP2 or FP64, reorth count */
  int converged;            /* 1 if the residual test passed */
  double rms_residual;      /* final FP64 ||H C - C Lambda||_F / sqrt(m) */
  double max_residual;      /* final FP64 max_j ||H c_j - lambda_j c_j|| */
  double E_last;            /* energy of the last iterate (FP64 trace) */
  double seconds;           /* host wall time of trm_solve */
  long long launches;       /* library kernel launches this solve issued */
} trm_stats;

/* Per-class kernel timing of one handle (see trm_profile). */
typedef struct {
  char name[16];       /* kernel class, e.g. "gram_f32", "spmm_f64" */
  double ms;           /* summed CUDA-event time of its launches */
  long long launches;  /* launcher calls timed (a call may be 2 kernels) */
  double flops;        /* summed algorithmic flops of those calls */
  double bytes;        /* summed algorithmic bytes moved by those calls */
} trm_kernel_stats;

/* Fill *opt with the defaults listed above. */
trm_status trm_default_options(trm_options* opt);

/*
 * Create a solver for H = -1/2 nabla^2_h + diag(V) on an nx x ny x nz grid with
 * zero Dirichlet boundaries (grid point idx = x + nx*(y + ny*z)); an axis of
 * length 1 is absent, so nz = 1 is a 2-D problem. order = 2 uses the 3-point
 * rule per axis (7-point stencil in 3-D), order = 4 the 5-point 4th-order
 * rule (13-point). V: host, N = nx*ny*nz doubles, copied; NULL means V = 0.
 * tol: the solve stops when the RMS column residual
 * ||H C - C (C^T H C)||_F / sqrt(m) <= tol (the paper's "||G|| sufficiently
 * small", Sec. 2.1). 1 <= m < N. opt may be NULL for defaults.
 */
trm_status trm_create_stencil(trm_handle* out, int nx, int ny, int nz,
                              int order, double h, const double* V, int m,
                              double tol, const trm_options* opt);

/*
 * Create a solver for an explicit symmetric CSR matrix (N rows, int32 row
 * pointers and column indices, ascending columns per row, values FP32
 * (vals_dtype = TRM_F32) or FP64 (TRM_F64)). All arrays are host memory and
 * are copied. Symmetry is the caller's responsibility (Eq. BASICEQ).
 */
trm_status trm_create_csr(trm_handle* out, int64_t N, const int32_t* rowptr,
                          const int32_t* cols, const void* vals,
                          int vals_dtype, int m, double tol,
                          const trm_options* opt);

/*
 * Generalized problem H e = lambda S e with S symmetric positive definite
 * (Sec. 2.1: trace minimization extends to it directly, which admits
 * non-orthogonal basis functions). Attaches S to a handle made by
 * trm_create_stencil or trm_create_csr with precision TRM_FP64, TRM_MIXED
 * or TRM_FULL_SP; trm_solve then minimises tr(C^T H C) under C^T S C = I
 * (TRM_MIXED: full SP with S applied in FP32 -- its values rounded -- and
 * Y = S C carried in FP32, then FP64 iterations in place of MP2, then the
 * FP64 Rayleigh-Ritz step; TRM_FULL_SP: full SP, then that step): the orthonormalization
 * factors C^T S C, the gradient is G = -2 (H C - S C H_C), the line search
 * uses the overlap (C + aP)^T S (C + aP), the diagonal preconditioner
 * becomes 1 / (H_ii - sigma S_ii) with sigma = min_k H_kk / S_kk - 1, and
 * the closing Rayleigh-Ritz step solves (C^T H C) y = theta (C^T S C) y.
 * The returned C is S-orthonormal and the residuals are ||H c - theta S c||.
 * rowptr: host, N + 1 int32 (rowptr[0] = 0, non-decreasing); cols: host,
 * rowptr[N] int32 in [0, N); vals: host, rowptr[N] FP64 (duplicates add).
 * The arrays are copied before the call returns. S's symmetry and
 * definiteness are not checked (an indefinite S shows as TRM_ENOTPD from
 * trm_solve); every diagonal entry must be positive. TRM_EINVAL for
 * TRM_MP2 or invalid arrays. The step operations (trm_energy_gradient,
 * trm_set_block, trm_iterate, trm_rayleigh_ritz) cover the standard problem
 * only and return TRM_EINVAL on a handle with an overlap.
 */
trm_status trm_set_overlap_csr(trm_handle h, const int32_t* rowptr,
                               const int32_t* cols, const double* vals);

/*
 * Run Fig. TMFIG to convergence, then diagonalise C^T H C (Rayleigh-Ritz,
 * Sec. 2.1) in FP64. Outputs (any may be NULL):
 *   lambda - host, m doubles, ascending;
 *   E_G    - host, sum of lambda (Eq. EGEQ);
 *   C      - N x m FP64 column-major Ritz vectors, on the device if
 *            C_on_device != 0, else in host memory;
 *   stats  - host.
 * C0: optional N x m FP64 starting block (host memory, need not be
 * orthonormal); NULL draws it from opt.seed. Returns TRM_ENOCONV (with the
 * best result written) when max_iter is reached.
 */
trm_status trm_solve(trm_handle h, double* lambda, double* E_G, double* C,
                     int C_on_device, const double* C0, trm_stats* stats);

trm_status trm_destroy(trm_handle h);

/* One iteration of the last trm_solve, as the host read it (Fig. TMFIG;
 * the quantities behind the paper's convergence plots: with the returned
 * E_G, R_i = (E - E_G) / E_G). */
typedef struct {
  double E;      /* tr(C_i^T H C_i) (FP32 products summed in FP64 in full SP) */
  double rms;    /* RMS column residual ||G_i||_F / (2 sqrt(m)) */
  double alpha;  /* line step taken from C_i (0 on a restart without a step) */
  double gamma;  /* Polak-Ribiere coefficient of the direction P_i */
  int phase;     /* 0 full SP, 1 MP2, 2 FP64 */
  int restart;   /* 1 when P_i was not a descent direction, so P_{i+1}
                    restarts CG (gamma = 0) */
} trm_iter_record;

/* Per-iteration history of the last trm_solve on h: writes the first
 * min(count, cap) records to out (host; may be NULL when cap = 0) and
 * returns count, one record per iteration run (stats.iterations). The
 * convergence test passes on record count - 1 - lag (lag =
 * trm_options.lag): the host reads the scalars that many iterations late,
 * and the iterations already enqueued then still run. Negative trm_status
 * for a NULL handle or cap < 0. */
int trm_history(trm_handle h, trm_iter_record* out, int cap);
const char* trm_strerror(trm_status s);
const char* trm_last_error(trm_handle h);
const char* trm_last_global_error(void);

/* ------------------------------------------------------------------------
 * Step operations: one row of the per-iteration block step each, on caller
 * device buffers and the stream in the handle's options. They synchronise
 * that stream before returning. Used to check each step in isolation.
 * ---------------------------------------------------------------------- */

/* N of the handle's operator. */
int64_t trm_dim(trm_handle h);

/*
 * X = H C for ncols columns (Fig. EGFIG step (1)). C, X: device, N x ncols,
 * dtype_in / dtype_out in {TRM_F32, TRM_F64}; the sum is formed in the output
 * precision. Stencil operators support (F32,F32) and (F64,F64); CSR
 * operators the same two.
 */
trm_status trm_apply_h(trm_handle h, int dtype_in, const void* C,
                       int dtype_out, void* X, int ncols);

/*
 * Fig. EGFIG Algorithm-2, steps (1)-(7), for an orthonormal C (device, N x m
 * FP64). Writes E (host double), H_D (device, m doubles), H' (device, m x m
 * FP64, diag set to 0 when zero_diag != 0, Sec. 2.2) and
 * G = -2 (X' - C H') (device, N x m in G_dtype). With G_dtype = TRM_F32 the
 * products of steps (6) and (7) run in FP32 as in MP2; steps (1), (2), (3),
 * (5) stay FP64.
 */
trm_status trm_energy_gradient(trm_handle h, const double* C, double* E,
                               double* HD, double* Hprime, void* G,
                               int G_dtype, int zero_diag);

/*
 * out = A^T B (m x n, device FP64, column-major ld = m) for A: N x m and
 * B: N x n (device, leading dimensions N, element type dtype). FP32 inputs
 * are multiplied and summed in FP32 within a tile of rows and the tiles are
 * summed in FP64 in a fixed order. Covers the Gram products C^T X' of
 * Fig. EGFIG step (6), C^T C of Fig. ONFIG step (1) and the line-search
 * projections C^T P, P^T P, P^T H P.
 */
trm_status trm_gram(int64_t N, int m, int n, int dtype, const void* A,
                    const void* B, double* out, void* stream);

/*
 * Fig. ONFIG in FP64 on the device: S = C^T C, S = L L^T, C <- C L^{-T}.
 * C: device, N x m FP64, overwritten. Returns TRM_ENOTPD if S is not
 * positive definite.
 */
trm_status trm_orthonormalize(int64_t N, int m, double* C, void* stream);

/*
 * Initial-guess extrapolation for a chain of related problems (Secs. 3 and
 * 4 cite it as the way to start close to the solution): from
 * the converged blocks of the two previous problems, a block for the next.
 * C_cur's columns are any basis of its subspace, so C_prev is first aligned
 * to it by the orthogonal U that minimises ||C_prev U - C_cur||_F (the polar
 * factor of M = C_prev^T C_cur, formed on the device as
 * M (M^T M)^{-1/2} from the eigendecomposition of M^T M); then
 *   C_next = C_cur + alpha (C_cur - C_prev U),
 * orthonormalized as trm_orthonormalize does (C_next^T C_next = I, Cholesky
 * factor, so the result is unique). alpha = 1 is linear extrapolation in
 * equal steps; alpha = dt_next / dt_prev for unequal ones.
 * C_prev, C_cur: device, N x m column-major FP64, orthonormal, read only.
 * C_next: device, N x m, written (may not alias the inputs).
 * Returns TRM_ENOTPD if M^T M has an eigenvalue below 1e-12 of its largest
 * (the two subspaces are too far apart to align) or if C_next^T C_next is
 * not positive definite; C_next then holds no result.
 */
trm_status trm_extrapolate(int64_t N, int m, const double* C_prev,
                           const double* C_cur, double alpha, double* C_next,
                           void* stream);

/*
 * One iteration of Fig. TMFIG from the handle's current state in the given
 * precision mode (TRM_FP64 or TRM_FULL_SP or TRM_MP2), starting a new CG
 * sequence when restart != 0. The state is set by trm_set_block and read by
 * trm_get_block. E_out (host) receives E_i and rms_out (host) the RMS
 * residual of G_i, both before the update; alpha_out the step taken.
 */
trm_status trm_set_block(trm_handle h, const double* C_device);
trm_status trm_get_block(trm_handle h, double* C_device);
trm_status trm_iterate(trm_handle h, int mode, int restart, double* E_out,
                       double* rms_out, double* alpha_out);

/*
 * Rayleigh-Ritz on span(C) in FP64 (Sec. 2.1): solves (C^T H C) y = theta
 * (C^T C) y, overwrites C (device, N x m FP64) with C Y (unit columns, each
 * column's largest-magnitude entry positive), and writes lambda (host, m,
 * ascending) and the residual norms ||H c_j - lambda_j c_j|| (host, m).
 */
trm_status trm_rayleigh_ritz(trm_handle h, double* C, double* lambda,
                             double* residuals);

/*
 * Timing of the library's kernels by class, with a pair of CUDA events on the
 * handle's stream around each launcher call of a solve (no paper
 * counterpart: measurement support). Classes, one kernel family each:
 * spmm_f32, spmm_f64, spmm_df (MP2's double-float H C), gram_f32, gram_f64,
 * grad_f32, grad_f64, rotate_f32, rotate_f64, rotate_df (MP2's split
 * rotation), rowops, small_mm, eig. enable != 0 zeroes the counters and
 * starts timing; 0 stops it. trm_profile_read copies up to max classes into
 * out (host) and returns how many exist, or a negative status.
 */
trm_status trm_profile(trm_handle h, int enable);
int trm_profile_read(trm_handle h, trm_kernel_stats* out, int max);

/* Kernel launches issued by the library in this process (all handles). */
long long trm_launch_count(void);

/*
 * trm_gram_noalloc: out = A^T B as trm_gram computes it, for callers that
 * must not allocate device memory (no counterpart in the paper). Some callers
 * cannot call cudaMalloc: they have given the device's memory to their own
 * allocator (a framework's caching pool or an arena sized at start-up), or
 * they run under a budget that must not grow, or cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree inside a timed loop.
 * This variant keeps its split partial sums in a fixed 24 MiB array
 * (3 * 2^20 doubles) compiled into the library, which every GPU that loads
 * the library holds until the process exits; it calls no allocation routine.
 * Limit: m * n <= 2^20 (up to 1024 x 1024); larger sizes return TRM_EINVAL
 * with a message in trm_last_global_error().
 * Kernels: FP32 operands that trm_gram sends to the tensor cores (N % 4 == 0,
 * m >= 32, A and B 16-byte aligned) run that same kernel (error below
 * 1.4e-5 sum_k |a_ki||b_kj|), with the same row slices and sum order, so the
 * same bytes as trm_gram's, whenever m * n * slices <= 3 * 2^20 - 1 (else
 * with fewer, longer slices); other FP32 operands and all FP64 operands run
 * trm_gram's SIMT kernel (products summed in the operands' precision within
 * a slice of rows, the slices in FP64), with fewer, longer row slices when
 * its partials would not fit, which changes only the summation order.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture. All calls share the one array and each overwrites every
 * partial it reads, so nothing needs clearing, but calls that overlap on the
 * GPU (different streams or host threads at once) race on it. Like trm_gram,
 * the call synchronizes the stream before it returns. A, B, out: device;
 * stream as in trm_gram.
 */
trm_status trm_gram_noalloc(int64_t N, int m, int n, int dtype, const void* A,
                            const void* B, double* out, void* stream);

/* Fill an N x m FP64 device block with the splitmix64 random guess of the
 * given seed: entry (i, j) = u(seed, i + N j) - 0.5 (Sec. 3: random C0). */
trm_status trm_random_block(int64_t N, int m, uint64_t seed, double* C,
                            void* stream);

/* ------------------------------------------------------------------------
 * Slab partition for several GPUs (host logic; no paper counterpart beyond
 * Sec. 2.1's observation that every block step is a loop over grid points).
 * Rank r of `ranks` owns the z-planes [z0, z1) of an nx x ny x nz stencil
 * grid (planes split as evenly as possible, the first nz % ranks ranks one
 * more), i.e. the rows [row0, row0 + rows) of every N x m block. Applying H
 * to its rows needs `radius` planes on either side (1 for order 2, 2 for
 * order 4) from the neighbouring ranks: halo_lo planes below z0 and halo_hi
 * above z1 (0 at the grid's walls, where the Dirichlet boundary applies).
 * The rank's extended grid is nx x ny x ext_nz planes starting at ext_z0
 * (ext_rows rows): a stencil handle on that grid, with the halo planes
 * filled from the neighbours, gives H C exactly on the owned rows. The
 * N-deep sums (Grams, energies) are the sums over ranks of the partials
 * over owned rows. TRM_EINVAL if a slab would be thinner than the stencil's
 * reach (ranks > 1 and nz / ranks < radius) or for invalid arguments.
 * ------------------------------------------------------------------------ */
typedef struct {
  int z0, z1;           /* owned planes [z0, z1) */
  int halo_lo, halo_hi; /* planes received from rank - 1 and rank + 1 */
  int64_t row0, rows;   /* owned rows [row0, row0 + rows) of every block */
  int ext_z0, ext_nz;   /* extended grid: planes [ext_z0, ext_z0 + ext_nz) */
  int64_t ext_rows;     /* nx * ny * ext_nz */
} trm_slab;

trm_status trm_slab_plan(int nx, int ny, int nz, int order, int ranks,
                         int rank, trm_slab* out);

/* ------------------------------------------------------------------------
 * Serving: a request server that solves eigenproblems of different sizes as
 * they arrive (no counterpart in the paper; it serves many independent
 * trace minimizations on one GPU). A request is admitted in arrival order
 * while the device footprints of the live solves fit device_bytes and fewer
 * than max_live solves run; every live solve has its own CUDA stream and host
 * thread, so solves overlap on the device. Each result is the one trm_solve
 * returns for the same problem and options on its own handle: the same
 * bytes alone and in the mix.
 * ------------------------------------------------------------------------ */
typedef struct trm_server_ctx* trm_server;

/* A stencil problem (as trm_create_stencil): V is a host array of
 * nx*ny*nz FP64 values (or NULL), copied at submission; opt.stream is
 * ignored (the server owns the streams); opt may be all defaults
 * (trm_default_options). Warm start across related requests (e.g. the same
 * grid with a perturbed potential): C0 (host, N x m column-major FP64, or
 * NULL for the seeded random block) is copied at submission and starts the
 * iteration, as trm_solve's C0; C_out (host, N x m, or NULL) receives the
 * converged block when the solve ends, so the caller keeps it alive until
 * trm_server_wait for this ticket returns. */
typedef struct {
  int nx, ny, nz, order;
  double h;
  const double* V;
  int m;
  double tol;
  trm_options opt;
  const double* C0;
  double* C_out;
} trm_problem;

/* Device bytes a solve of an N x m problem allocates (the admission
 * estimate); 0 for invalid sizes. */
size_t trm_footprint_bytes(int64_t N, int m);

/* Start a server on the current device. device_bytes: admission budget;
 * max_live: most concurrent solves. TRM_EINVAL if either is 0. */
trm_status trm_server_create(trm_server* out, size_t device_bytes,
                             int max_live);

/* The scheduler alone: a server whose admitted requests call fn on their
 * host thread instead of solving on the GPU (admission order, budget,
 * max_live, waits and latencies are those of trm_server_create). fn gets
 * the problem as submitted (V and C0 NULL: the copies stay with the
 * server), writes lambda[m] (zeroed before the call), *E_G and *stats, and
 * returns a trm_status, which trm_server_wait returns. For testing the
 * scheduler without a GPU and for callers that run their own solver. No
 * CUDA call is made. TRM_EINVAL if fn is NULL or a size is 0. */
typedef int (*trm_server_fn)(const trm_problem* p, double* lambda,
                             double* E_G, trm_stats* stats, void* ctx);
trm_status trm_server_create_fn(trm_server* out, size_t device_bytes,
                                int max_live, trm_server_fn fn, void* ctx);

/* Queue a problem; never blocks. *ticket identifies it for trm_server_wait.
 * TRM_EINVAL for invalid sizes, TRM_ENOMEM when its footprint alone exceeds
 * the budget. */
trm_status trm_server_submit(trm_server s, const trm_problem* p,
                             int64_t* ticket);

/* Block until the ticket's solve is done; writes lambda[m] (host), *E_G,
 * *stats and *latency (seconds from submission to completion; any output
 * may be NULL) and releases the ticket. One caller waits per ticket: a
 * second wait on a ticket that another thread is waiting on, or on one
 * already released, returns TRM_EINVAL. Returns the solve's status (as
 * trm_solve); details in trm_last_global_error(). */
trm_status trm_server_wait(trm_server s, int64_t ticket, double* lambda,
                           double* E_G, trm_stats* stats, double* latency);

/* Finish every queued and live solve, then free the server. */
trm_status trm_server_destroy(trm_server s);

#ifdef __cplusplus
}
#endif

#endif /* TRM_H */
