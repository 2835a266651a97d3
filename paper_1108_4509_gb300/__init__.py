"""Python binding of libtrm, the sm_103a trace-minimization eigensolver.

Argument marshalling only: every step of the solver runs in the CUDA library
behind the C ABI of include/trm.h, and the functions here carry the same names
as the C entry points. Host arrays are numpy arrays; device arrays are passed
as integer addresses (for example ``tensor.data_ptr()`` of a CUDA tensor) and
streams as ``torch.cuda.current_stream().cuda_stream``.

Importing this module loads the compiled library and raises ``ImportError``
when it is missing: there is no CPU fallback. Build it with
``paper_1108_4509_gb300._build.build()`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

__all__ = [
    "TRM_FP64", "TRM_MP1", "TRM_MP2", "TRM_FULL_SP", "TRM_MIXED", "TRM_F32",
    "TRM_F64", "TrmError", "trm_options", "trm_stats", "lib", "LIB_PATH",
    "trm_default_options", "trm_create_stencil", "trm_create_csr",
    "trm_set_overlap_csr", "trm_solve", "trm_history",
    "trm_destroy", "trm_strerror", "trm_last_error", "trm_dim", "trm_apply_h",
    "trm_energy_gradient", "trm_gram", "trm_gram_noalloc",
    "trm_orthonormalize", "trm_extrapolate", "trm_set_block",
    "trm_get_block", "trm_iterate", "trm_rayleigh_ritz", "trm_random_block",
    "trm_profile", "trm_profile_read", "trm_launch_count", "trm_kernel_stats",
    "trm_slab", "trm_slab_plan", "Solver",
]

TRM_FP64, TRM_MP1, TRM_MP2, TRM_FULL_SP, TRM_MIXED = 0, 1, 2, 3, 4
TRM_F32, TRM_F64 = 0, 1

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtrm.so")


class trm_options(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("precond", ct.c_int),
                ("max_iter", ct.c_int), ("seed", ct.c_uint64),
                ("switch_tol", ct.c_double * 2), ("reorth_every", ct.c_int),
                ("rr_every", ct.c_int), ("lag", ct.c_int),
                ("stream", ct.c_void_p), ("graphs", ct.c_int)]


class trm_stats(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("iterations_phase", ct.c_int * 3),
                ("converged", ct.c_int), ("rms_residual", ct.c_double),
                ("max_residual", ct.c_double), ("E_last", ct.c_double),
                ("seconds", ct.c_double), ("launches", ct.c_longlong)]

    def as_dict(self):
        return {"iterations": self.iterations,
                "iterations_phase": list(self.iterations_phase),
                "converged": bool(self.converged),
                "rms_residual": self.rms_residual,
                "max_residual": self.max_residual, "E_last": self.E_last,
                "seconds": self.seconds, "launches": self.launches}


class trm_iter_record(ct.Structure):
    _fields_ = [("E", ct.c_double), ("rms", ct.c_double),
                ("alpha", ct.c_double), ("gamma", ct.c_double),
                ("phase", ct.c_int), ("restart", ct.c_int)]


class trm_kernel_stats(ct.Structure):
    _fields_ = [("name", ct.c_char * 16), ("ms", ct.c_double),
                ("launches", ct.c_longlong), ("flops", ct.c_double),
                ("bytes", ct.c_double)]


class trm_slab(ct.Structure):
    _fields_ = [("z0", ct.c_int), ("z1", ct.c_int), ("halo_lo", ct.c_int),
                ("halo_hi", ct.c_int), ("row0", ct.c_int64),
                ("rows", ct.c_int64), ("ext_z0", ct.c_int),
                ("ext_nz", ct.c_int), ("ext_rows", ct.c_int64)]


class trm_problem(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("order", ct.c_int), ("h", ct.c_double), ("V", ct.c_void_p),
                ("m", ct.c_int), ("tol", ct.c_double), ("opt", trm_options),
                ("C0", ct.c_void_p), ("C_out", ct.c_void_p)]


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(paper_1108_4509_gb300._build.build())")
lib = ct.CDLL(LIB_PATH)

_h = ct.c_void_p
_p = ct.c_void_p
_i = ct.c_int
_i64 = ct.c_int64
_d = ct.c_double
_dp = ct.POINTER(ct.c_double)

_SIGS = {
    "trm_default_options": (_i, [ct.POINTER(trm_options)]),
    "trm_create_stencil": (_i, [ct.POINTER(_h), _i, _i, _i, _i, _d, _p, _i, _d,
                                ct.POINTER(trm_options)]),
    "trm_create_csr": (_i, [ct.POINTER(_h), _i64, _p, _p, _p, _i, _i, _d,
                            ct.POINTER(trm_options)]),
    "trm_set_overlap_csr": (_i, [_h, _p, _p, _p]),
    "trm_history": (_i, [_h, ct.POINTER(trm_iter_record), _i]),
    "trm_solve": (_i, [_h, _p, _p, _p, _i, _p, ct.POINTER(trm_stats)]),
    "trm_destroy": (_i, [_h]),
    "trm_strerror": (ct.c_char_p, [_i]),
    "trm_last_error": (ct.c_char_p, [_h]),
    "trm_last_global_error": (ct.c_char_p, []),
    "trm_dim": (_i64, [_h]),
    "trm_apply_h": (_i, [_h, _i, _p, _i, _p, _i]),
    "trm_energy_gradient": (_i, [_h, _p, _p, _p, _p, _p, _i, _i]),
    "trm_gram": (_i, [_i64, _i, _i, _i, _p, _p, _p, _p]),
    "trm_gram_noalloc": (_i, [_i64, _i, _i, _i, _p, _p, _p, _p]),
    "trm_orthonormalize": (_i, [_i64, _i, _p, _p]),
    "trm_extrapolate": (_i, [_i64, _i, _p, _p, _d, _p, _p]),
    "trm_set_block": (_i, [_h, _p]),
    "trm_get_block": (_i, [_h, _p]),
    "trm_iterate": (_i, [_h, _i, _i, _p, _p, _p]),
    "trm_rayleigh_ritz": (_i, [_h, _p, _p, _p]),
    "trm_random_block": (_i, [_i64, _i, ct.c_uint64, _p, _p]),
    "trm_profile": (_i, [_h, _i]),
    "trm_profile_read": (_i, [_h, ct.POINTER(trm_kernel_stats), _i]),
    "trm_launch_count": (ct.c_longlong, []),
    "trm_footprint_bytes": (ct.c_size_t, [_i64, _i]),
    "trm_slab_plan": (_i, [_i, _i, _i, _i, _i, _i, ct.POINTER(trm_slab)]),
    "trm_server_create": (_i, [ct.POINTER(_h), ct.c_size_t, _i]),
    "trm_server_submit": (_i, [_h, ct.POINTER(trm_problem),
                               ct.POINTER(ct.c_int64)]),
    "trm_server_wait": (_i, [_h, ct.c_int64, _p, _p, ct.POINTER(trm_stats),
                             _p]),
    "trm_server_destroy": (_i, [_h]),
    "trm_server_create_fn": (_i, [ct.POINTER(_h), ct.c_size_t, _i, _p, _p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class TrmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib.trm_strerror(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status, handle=None):
    if status != 0:
        msg = (lib.trm_last_error(handle) if handle else
               lib.trm_last_global_error())
        raise TrmError(status, (msg or b"").decode())
    return status


def _host(a, dtype):
    """Pointer to a contiguous host numpy array of the given dtype (or None)."""
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype) if not (
        isinstance(a, np.ndarray) and a.dtype == dtype
        and (a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"])) else a
    return arr, arr.ctypes.data_as(ct.c_void_p)


def _colmajor(a, dtype):
    """Host N x m block as column-major (Fortran) memory."""
    arr = np.asfortranarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ct.c_void_p)


# --------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------
def trm_default_options(**overrides) -> trm_options:
    o = trm_options()
    _check(lib.trm_default_options(ct.byref(o)))
    for k, v in overrides.items():
        if k == "switch_tol":
            for i, x in enumerate(v):
                o.switch_tol[i] = x
        elif k == "stream":
            o.stream = ct.c_void_p(int(v) if v else 0)
        else:
            setattr(o, k, v)
    return o


def trm_create_stencil(nx, ny, nz, order, h, V, m, tol, opt=None):
    handle = _h()
    Varr, Vp = _host(V, np.float64)
    if Varr is not None and Varr.size != nx * ny * nz:
        raise ValueError("V must have nx*ny*nz entries")
    _check(lib.trm_create_stencil(ct.byref(handle), nx, ny, nz, order, h, Vp,
                                  m, tol, ct.byref(opt) if opt else None))
    return handle


def trm_create_csr(N, rowptr, cols, vals, m, tol, opt=None):
    handle = _h()
    rp, rpp = _host(rowptr, np.int32)
    ci, cip = _host(cols, np.int32)
    vals = np.asarray(vals)
    dt = TRM_F64 if vals.dtype == np.float64 else TRM_F32
    va, vap = _host(vals, np.float64 if dt == TRM_F64 else np.float32)
    _check(lib.trm_create_csr(ct.byref(handle), N, rpp, cip, vap, dt, m, tol,
                              ct.byref(opt) if opt else None))
    return handle


def trm_set_overlap_csr(handle, rowptr, cols, vals):
    """The SPD overlap S of the generalized problem H e = lambda S e (host
    CSR arrays, copied); the handle must use precision TRM_FP64."""
    N = trm_dim(handle)
    rp, rpp = _host(rowptr, np.int32)
    if rp.shape != (N + 1,):
        raise ValueError("rowptr must have N + 1 entries")
    nnz = int(rp[-1])
    ci, cip = _host(cols, np.int32)
    va, vap = _host(vals, np.float64)
    if ci.shape != (nnz,) or va.shape != (nnz,):
        raise ValueError("cols and vals must have rowptr[N] entries")
    _check(lib.trm_set_overlap_csr(handle, rpp, cip, vap), handle)


def trm_solve(handle, N, m, C_out=None, C_on_device=False, C0=None):
    """Returns (lambda, E_G, stats, status). C_out: device address (int) when
    C_on_device, else a host float64 array of shape (N, m) in Fortran order
    that receives C, or None."""
    lam = np.zeros(m)
    eg = ct.c_double(0.0)
    st = trm_stats()
    c0arr, c0p = _colmajor(C0, np.float64) if C0 is not None else (None, None)
    if C_out is None:
        cp = None
    elif C_on_device:
        cp = ct.c_void_p(int(C_out))
    else:
        if not (isinstance(C_out, np.ndarray) and C_out.flags["F_CONTIGUOUS"]
                and C_out.dtype == np.float64 and C_out.shape == (N, m)):
            raise ValueError("host C_out must be a Fortran-ordered float64 (N, m) array")
        cp = C_out.ctypes.data_as(ct.c_void_p)
    status = lib.trm_solve(handle, lam.ctypes.data_as(ct.c_void_p),
                           ct.cast(ct.byref(eg), ct.c_void_p), cp,
                           1 if C_on_device else 0, c0p, ct.byref(st))
    if status not in (0, -4):
        _check(status, handle)
    return lam, eg.value, st, status


def trm_history(handle):
    """Per-iteration records of the last solve on the handle, as arrays:
    {"E", "rms", "alpha", "gamma", "phase", "restart"}."""
    n = lib.trm_history(handle, None, 0)
    if n < 0:
        _check(n, handle)
    buf = (trm_iter_record * max(n, 1))()
    lib.trm_history(handle, buf, n)
    return {k: np.array([getattr(buf[i], k) for i in range(n)])
            for k in ("E", "rms", "alpha", "gamma", "phase", "restart")}


def trm_destroy(handle):
    if handle:
        _check(lib.trm_destroy(handle))


def trm_strerror(status):
    return lib.trm_strerror(status).decode()


def trm_last_error(handle=None):
    r = lib.trm_last_error(handle) if handle else lib.trm_last_global_error()
    return (r or b"").decode()


def trm_dim(handle):
    return int(lib.trm_dim(handle))


def trm_apply_h(handle, dtype_in, C_ptr, dtype_out, X_ptr, ncols):
    return _check(lib.trm_apply_h(handle, dtype_in, ct.c_void_p(C_ptr),
                                  dtype_out, ct.c_void_p(X_ptr), ncols), handle)


def trm_energy_gradient(handle, C_ptr, HD_ptr, Hprime_ptr, G_ptr, G_dtype,
                        zero_diag):
    E = ct.c_double(0.0)
    _check(lib.trm_energy_gradient(handle, ct.c_void_p(C_ptr),
                                   ct.cast(ct.byref(E), ct.c_void_p),
                                   ct.c_void_p(HD_ptr) if HD_ptr else None,
                                   ct.c_void_p(Hprime_ptr) if Hprime_ptr else None,
                                   ct.c_void_p(G_ptr), G_dtype,
                                   1 if zero_diag else 0), handle)
    return E.value


def trm_gram(N, m, n, dtype, A_ptr, B_ptr, out_ptr, stream=0):
    return _check(lib.trm_gram(N, m, n, dtype, ct.c_void_p(A_ptr),
                               ct.c_void_p(B_ptr), ct.c_void_p(out_ptr),
                               ct.c_void_p(stream or 0)))


def trm_gram_noalloc(N, m, n, dtype, A_ptr, B_ptr, out_ptr, stream=0):
    """trm_gram without any device allocation (fixed in-library scratch)."""
    return _check(lib.trm_gram_noalloc(N, m, n, dtype, ct.c_void_p(A_ptr),
                                       ct.c_void_p(B_ptr),
                                       ct.c_void_p(out_ptr),
                                       ct.c_void_p(stream or 0)))


def trm_orthonormalize(N, m, C_ptr, stream=0):
    return _check(lib.trm_orthonormalize(N, m, ct.c_void_p(C_ptr),
                                         ct.c_void_p(stream or 0)))


def trm_extrapolate(N, m, C_prev_ptr, C_cur_ptr, alpha, C_next_ptr, stream=0):
    """Device pointers (N x m column-major FP64): C_next = orth(C_cur +
    alpha (C_cur - C_prev U)), U the orthogonal alignment of C_prev to
    C_cur."""
    return _check(lib.trm_extrapolate(N, m, ct.c_void_p(C_prev_ptr),
                                      ct.c_void_p(C_cur_ptr), float(alpha),
                                      ct.c_void_p(C_next_ptr),
                                      ct.c_void_p(stream or 0)))


def trm_set_block(handle, C_ptr):
    return _check(lib.trm_set_block(handle, ct.c_void_p(C_ptr)), handle)


def trm_get_block(handle, C_ptr):
    return _check(lib.trm_get_block(handle, ct.c_void_p(C_ptr)), handle)


def trm_iterate(handle, mode, restart=False):
    E, r, a = ct.c_double(), ct.c_double(), ct.c_double()
    _check(lib.trm_iterate(handle, mode, 1 if restart else 0,
                           ct.cast(ct.byref(E), ct.c_void_p),
                           ct.cast(ct.byref(r), ct.c_void_p),
                           ct.cast(ct.byref(a), ct.c_void_p)), handle)
    return E.value, r.value, a.value


def trm_rayleigh_ritz(handle, C_ptr, m):
    lam = np.zeros(m)
    res = np.zeros(m)
    _check(lib.trm_rayleigh_ritz(handle, ct.c_void_p(C_ptr),
                                 lam.ctypes.data_as(ct.c_void_p),
                                 res.ctypes.data_as(ct.c_void_p)), handle)
    return lam, res


def trm_random_block(N, m, seed, C_ptr, stream=0):
    return _check(lib.trm_random_block(N, m, ct.c_uint64(seed),
                                       ct.c_void_p(C_ptr),
                                       ct.c_void_p(stream or 0)))


def trm_profile(handle, enable):
    return _check(lib.trm_profile(handle, 1 if enable else 0), handle)


def trm_profile_read(handle):
    """{class name: {ms, launches, flops, bytes}} of the handle's timed calls."""
    buf = (trm_kernel_stats * 32)()
    n = lib.trm_profile_read(handle, buf, 32)
    if n < 0:
        _check(n, handle)
    return {buf[k].name.decode(): {"ms": buf[k].ms, "launches": buf[k].launches,
                                   "flops": buf[k].flops, "bytes": buf[k].bytes}
            for k in range(min(n, 32))}


def trm_launch_count():
    return int(lib.trm_launch_count())


class Solver:
    """Owns one handle. ``Solver.stencil(...)`` / ``Solver.csr(...)`` create
    it; ``solve()`` runs it; ``close()`` (or the context manager) frees it."""

    def __init__(self, handle, N, m):
        self.handle, self.N, self.m = handle, N, m

    @classmethod
    def stencil(cls, shape, order, h, V, m, tol, **opts):
        nx, ny, nz = (tuple(shape) + (1, 1))[:3]
        opt = trm_default_options(**opts)
        return cls(trm_create_stencil(nx, ny, nz, order, h, V, m, tol, opt),
                   nx * ny * nz, m)

    @classmethod
    def csr(cls, N, rowptr, cols, vals, m, tol, **opts):
        opt = trm_default_options(**opts)
        return cls(trm_create_csr(N, rowptr, cols, vals, m, tol, opt), N, m)

    def set_overlap(self, rowptr, cols, vals):
        """Make it the generalized problem H e = lambda S e (S SPD, CSR; the
        handle must use precision TRM_FP64)."""
        trm_set_overlap_csr(self.handle, rowptr, cols, vals)
        return self

    def solve(self, C0=None, want_C=True):
        C = np.zeros((self.N, self.m), order="F") if want_C else None
        lam, eg, st, status = trm_solve(self.handle, self.N, self.m, C_out=C,
                                        C0=C0)
        return lam, eg, C, st.as_dict(), status

    def history(self):
        """Per-iteration records of the last solve (see trm_history)."""
        return trm_history(self.handle)

    def close(self):
        if self.handle:
            trm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Serving: concurrent solves of problems submitted as they arrive
# ---------------------------------------------------------------------------
def trm_slab_plan(nx, ny, nz, order, ranks, rank):
    """The z-slab of `rank` among `ranks` (see trm_slab in trm.h)."""
    out = trm_slab()
    _check(lib.trm_slab_plan(nx, ny, nz, order, ranks, rank, ct.byref(out)))
    return out


def trm_footprint_bytes(N, m):
    return int(lib.trm_footprint_bytes(N, m))


def trm_server_create(device_bytes, max_live):
    h = _h()
    _check(lib.trm_server_create(ct.byref(h), device_bytes, max_live))
    return h


# int fn(const trm_problem*, double* lambda, double* E_G, trm_stats*, void*)
TRM_SERVER_FN = ct.CFUNCTYPE(ct.c_int, ct.c_void_p, ct.POINTER(ct.c_double),
                             ct.POINTER(ct.c_double), ct.c_void_p, ct.c_void_p)


def trm_server_create_fn(device_bytes, max_live, fn, ctx=None):
    """A server whose admitted requests call fn (a TRM_SERVER_FN; the caller
    keeps it alive until trm_server_destroy returns) instead of solving."""
    h = _h()
    _check(lib.trm_server_create_fn(ct.byref(h), device_bytes, max_live,
                                    ct.cast(fn, ct.c_void_p),
                                    ct.c_void_p(ctx) if ctx else None))
    return h


def trm_server_submit(server, shape, order, h, V, m, tol, opt=None, C0=None,
                      C_out=None):
    """Queue a stencil problem; returns its ticket. V (host, nx*ny*nz FP64
    or None) and the warm start C0 (host (N, m) or None) are copied before
    this returns; C_out (a Fortran-ordered float64 (N, m) array or None)
    receives the converged block, so keep it alive until the wait returns."""
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    N = nx * ny * nz
    Varr, Vp = _host(V, np.float64)
    if Varr is not None and Varr.size != N:
        raise ValueError("V must have nx*ny*nz entries")
    c0arr, c0p = _colmajor(C0, np.float64) if C0 is not None else (None, None)
    if c0arr is not None and c0arr.shape != (N, m):
        raise ValueError("C0 must be an (N, m) block")
    cop = None
    if C_out is not None:
        if not (isinstance(C_out, np.ndarray) and C_out.flags["F_CONTIGUOUS"]
                and C_out.dtype == np.float64 and C_out.shape == (N, m)):
            raise ValueError("C_out must be a Fortran-ordered float64 (N, m) array")
        cop = C_out.ctypes.data_as(ct.c_void_p)
    p = trm_problem(nx=nx, ny=ny, nz=nz, order=order, h=h, V=Vp, m=m,
                    tol=tol, opt=opt if opt is not None else trm_default_options(),
                    C0=c0p, C_out=cop)
    t = ct.c_int64()
    _check(lib.trm_server_submit(server, ct.byref(p), ct.byref(t)))
    return t.value


def trm_server_wait(server, ticket, m):
    """Block until the ticket's solve is done: (lambda, E_G, stats, status,
    latency_seconds); the status is trm_solve's (not raised)."""
    lam = np.zeros(m)
    eg = ct.c_double()
    st = trm_stats()
    lat = ct.c_double()
    status = lib.trm_server_wait(server, ticket,
                                 lam.ctypes.data_as(ct.c_void_p),
                                 ct.cast(ct.byref(eg), ct.c_void_p),
                                 ct.byref(st), ct.cast(ct.byref(lat), ct.c_void_p))
    return lam, eg.value, st.as_dict(), status, lat.value


def trm_server_destroy(server):
    return _check(lib.trm_server_destroy(server))
