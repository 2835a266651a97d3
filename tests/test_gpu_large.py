"""Parity at the full sizes of the larger configurations: the 96^3 grid with
m = 512, and the 100^3 grid with m = 1024 as a stencil and as an explicit CSR
with FP32 values and int32 columns. Checked on outputs the oracle computes
one at a time (sampled entries of H C, sampled H_D = c_j^T H c_j), on
properties of one solver step that hold at any size (orthonormality of
sampled columns, the energy decrease), and by whole mixed-precision solves
checked a posteriori: the oracle recomputes in FP64 on the host, from the
GPU's C, C^T C, C^T (H C), its eigenvalues and every column residual, and
compares the eigenvalues and E_G with the reference the oracle's own
filtered subspace iteration stored (tests/golden/workloads.json, written by
make_workloads.py from oracle/ only), with the Kato-Temple and Davis-Kahan
bounds that the residuals and the reference gaps give.

Tolerances: H C entries are sums of at most 13 products, so the FP64 path is
held to 32 u64 sum|H_ik||c_k| and the FP32 path to 32 u32 sum|H_ik||c_k|
(inputs and coefficients rounded to FP32 included). H_D is an FP64 sum of N
products: gamma_N(u64) sum_i |c_i||(H c)_i|. The tensor-core Gram splits each
FP32 value into two TF32 terms (hi the value truncated to TF32, lo rounded:
the dropped lo.lo and the roundings stay below 2^-19 of |a b|) and
accumulates chunks of 8 stages (96 MMA steps, each dropping up to 2^-23 of
the running sum) before folding them into a double-float sum: |error| <=
(96 * 2^-23 + 2^-19) sum|a_i||b_i| < 1.4e-5 sum|a_i||b_i|; a wrong tile,
index or operand is off by O(1) of that sum.
"""
import numpy as np
import pytest

import trm_inputs as ti
from oracle import operator as op

from . import gpu_util as gu

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53
SEED = 11

CASES = {
    "grid96_m512": ("grid96_o4_w512_m512", False),
    "grid100_m1024": ("grid100_o4_w1000_m1024", False),
    "grid100_m1024_csr": ("grid100_o4_w1000_m1024", True),
}


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


class Case:
    def __init__(self, trm, key):
        name, csr = CASES[key]
        self.w = w = ti.workload(name, seed=0)
        self.N, self.m = w.N, w.m
        V = w.potential()
        opt = trm.trm_default_options(stream=gu.stream(), precond=1)
        if csr:
            rp, ci, va = ti.grid_csr(w.shape, w.order, w.h, V, np.float32)
            self.h = trm.trm_create_csr(w.N, rp, ci, va, w.m, 1e-8, opt)
            # the matrix the GPU holds: FP32 values, exact in FP64
            import scipy.sparse as sp
            self.H = sp.csr_matrix((va.astype(np.float64), ci, rp),
                                   shape=(w.N, w.N))
        else:
            nx, ny, nz = w.shape
            self.h = trm.trm_create_stencil(nx, ny, nz, w.order, w.h, V, w.m,
                                            1e-8, opt)
            self.H = op.grid_hamiltonian(w.shape, w.order, w.h, V)
        self.cols = {}

    def col(self, j):
        if j not in self.cols:
            self.cols[j] = ti.random_block_column(self.N, j, SEED)
        return self.cols[j]


@pytest.fixture(scope="module", params=list(CASES))
def case(request, trm):
    c = Case(trm, request.param)
    yield c
    trm.trm_destroy(c.h)


def _device_block(trm, N, m):
    torch = gu.torch_mod()
    C = torch.empty(N * m, dtype=torch.float64, device="cuda")
    trm.trm_random_block(N, m, SEED, C.data_ptr(), gu.stream())
    return C


def _samples(N, m, k, seed):
    """k (row, column) pairs over 12 distinct columns (each column is
    regenerated on the host) including the first and the last."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, N, k)
    rows[:4] = [0, 1, N - 2, N - 1]  # grid boundaries
    pool = np.concatenate([[0, m - 1], rng.integers(1, m - 1, 10)])
    return rows, rng.choice(pool, k)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_apply_h_sampled(trm, case, dtype):
    torch = gu.torch_mod()
    N, m = case.N, case.m
    C = _device_block(trm, N, m)
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    Cin = C if dtype == "f64" else C.to(torch.float32)
    del C
    X = torch.empty(N * m, dtype=tdt, device="cuda")
    code = {"f64": trm.TRM_F64, "f32": trm.TRM_F32}[dtype]
    trm.trm_apply_h(case.h, code, Cin.data_ptr(), code, X.data_ptr(), m)
    rows, cols = _samples(N, m, 160, 3)
    got = X.view(m, N)[torch.as_tensor(cols, device="cuda"),
                       torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
    del X, Cin
    u = U64 if dtype == "f64" else U32
    H = case.H
    for r, c, g in zip(rows, cols, got):
        x = case.col(int(c))
        if dtype == "f32":
            x = x.astype(np.float32).astype(np.float64)
        lo, hi = H.indptr[r], H.indptr[r + 1]
        vals, idx = H.data[lo:hi], H.indices[lo:hi]
        ref = float(np.dot(vals, x[idx]))
        scale = float(np.dot(np.abs(vals), np.abs(x[idx])))
        assert abs(g - ref) <= 32 * u * scale, (r, c, g, ref)


def test_energy_terms_sampled(trm, case):
    """H_D[j] = c_j^T H c_j from the FP64 energy step, sampled columns."""
    torch = gu.torch_mod()
    N, m = case.N, case.m
    C = _device_block(trm, N, m)
    hd = torch.zeros(m, dtype=torch.float64, device="cuda")
    G = torch.empty(N * m, dtype=torch.float32, device="cuda")
    trm.trm_energy_gradient(case.h, C.data_ptr(), hd.data_ptr(), 0,
                            G.data_ptr(), trm.TRM_F32, 1)
    hd = hd.cpu().numpy()
    del C, G
    for j in (0, 1, m // 2, m - 1):
        c = case.col(j)
        Hc = case.H @ c
        ref = float(np.dot(c, Hc))
        scale = float(np.dot(np.abs(c), np.abs(Hc)))
        gam = N * U64 / (1 - N * U64)
        assert abs(hd[j] - ref) <= gam * scale + 1e-300, (j, hd[j], ref)


def test_gram_sampled(trm, case):
    """C^T C of the FP32 block on the tensor cores, sampled entries."""
    torch = gu.torch_mod()
    N, m = case.N, case.m
    C = _device_block(trm, N, m).to(torch.float32)
    out = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    trm.trm_gram(N, m, m, trm.TRM_F32, C.data_ptr(), C.data_ptr(),
                 out.data_ptr(), gu.stream())
    torch.cuda.synchronize()
    out = out.view(m, m).cpu().numpy()  # out[j, i] = (C^T C)(i, j)
    del C
    rng = np.random.default_rng(5)
    pairs = [(0, 0), (0, m - 1), (m - 1, m - 1)] + [
        tuple(rng.integers(0, m, 2)) for _ in range(12)]
    for i, j in pairs:
        a = case.col(int(i)).astype(np.float32).astype(np.float64)
        b = case.col(int(j)).astype(np.float32).astype(np.float64)
        ref = float(np.dot(a, b))
        scale = float(np.dot(np.abs(a), np.abs(b)))
        assert abs(out[j, i] - ref) <= 1.4e-5 * scale, (i, j, out[j, i], ref)


@pytest.mark.parametrize("mode", ["sp", "mp2"])
def test_iterate_step_properties(trm, case, mode):
    """One step from an orthonormal block: the energy drops and sampled
    columns of the new block stay orthonormal (to the phase's accuracy)."""
    torch = gu.torch_mod()
    N, m = case.N, case.m
    C = _device_block(trm, N, m)
    trm.trm_orthonormalize(N, m, C.data_ptr(), gu.stream())
    md = {"sp": trm.TRM_FULL_SP, "mp2": trm.TRM_MP2}[mode]
    trm.trm_set_block(case.h, C.data_ptr())
    E0, r0, a0 = trm.trm_iterate(case.h, md, restart=True)
    E1, r1, a1 = trm.trm_iterate(case.h, md, restart=False)
    assert np.isfinite([E0, E1, r0, r1]).all()
    assert a0 > 0 and E1 < E0
    out = torch.empty_like(C)
    trm.trm_get_block(case.h, out.data_ptr())
    idx = torch.as_tensor([0, 1, m // 2, m - 1], device="cuda")
    S = out.view(m, N)[idx].cpu().numpy()
    del out, C
    # MP2 factors S(a) = I + a (B + B^T) + a^2 Q in FP32 deviation form: the
    # columns stay orthonormal to a few FP32 roundings of S(a) - I (of order
    # one in the first steps from a random block) summed over m terms,
    # ~ 4 sqrt(m) 2^-24; full SP also rounds the block itself to FP32
    tol = {"sp": 1e-4, "mp2": 4 * np.sqrt(m) * 2.0 ** -24}[mode]
    assert np.max(np.abs(S @ S.T - np.eye(4))) < tol


# ---------------------------------------------------------------------------
# Whole solves, checked a posteriori by the oracle
# ---------------------------------------------------------------------------
LAM_TOL, EG_RTOL = 1e-9, 1e-10
SOLVE_TOL = 1e-10  # the solves' stopping tolerance (RMS column residual)
# The largest principal angle the Davis-Kahan bound may show: an FP32-class
# subspace sits near 2^-24 ||H|| / gap ~ 1e-3 at these gaps (||H|| ~ 10,
# gap >= 2e-4); the stopping rule gives ||R||_2 <= sqrt(m) 1e-10, i.e. at
# most 1.5e-5 at m = 1024 with the 100^3 workload's gap of 2.2e-4.
ANGLE_TOL = 2e-5


def _reference(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "workloads.json")
    return json.load(open(path))[name]


def _columns_product(H, C, threads=16):
    """X = H C for a Fortran-ordered host block, by column blocks in threads
    (each column is the plain sparse product)."""
    import concurrent.futures as cf
    N, m = C.shape
    X = np.empty((N, m), order="F")
    cuts = np.linspace(0, m, min(m, 4 * threads) + 1).astype(int)

    def one(i):
        lo, hi = cuts[i], cuts[i + 1]
        X[:, lo:hi] = H @ C[:, lo:hi]
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, range(len(cuts) - 1)))
    return X


_SOLVED = {}  # stencil solutions kept for the warm-started CSR solve


def _a_posteriori(H, lam, eg, C, g, m, exact_reference):
    """The oracle's FP64 checks of a returned (lambda, E_G, C) on the host."""
    ref = np.array(g["lambdas"] + g["lambdas_guard"])
    S = C.T @ C
    assert np.max(np.abs(S - np.eye(m))) <= 1e-12
    X = _columns_product(H, C)
    A = C.T @ X
    theta = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert np.max(np.abs(theta - lam)) <= LAM_TOL, np.max(np.abs(theta - lam))
    assert abs(eg - np.sum(theta)) <= EG_RTOL * abs(eg)
    # the Rayleigh quotients of the returned columns, in FP64 on the host,
    # their residuals, and the rounding of N-term dots (statistical,
    # 10 sqrt(N) 2^-53 sum |c| |H c|), once for these quotients and once for
    # the reference's own Rayleigh-Ritz values
    rq = np.diag(A) / np.diag(S)
    dot_slack = 20 * np.sqrt(C.shape[0]) * 2.0 ** -53 * np.einsum(
        "ij,ij->j", np.abs(C), np.abs(X))
    X -= C * rq[None, :]                      # H c_j - rq_j c_j
    r = np.linalg.norm(X, axis=0)
    X -= C * (lam - rq)[None, :]              # R = H C - C diag(lambda)
    RtR = X.T @ X
    r2 = float(np.sqrt(max(np.linalg.eigvalsh(0.5 * (RtR + RtR.T))[-1], 0.0)))
    del X
    if not exact_reference:
        # FP32 CSR values: its eigenvalues differ from the FP64 stencil's by
        # at most ||dH||_2 <= max row sum |dH| <= 2^-24 * 10 (rows of |H|
        # sum to at most 3.75 + 4.25 + |V| <= 10)
        assert np.max(np.abs(lam - ref[:m])) <= 2 * 10 * 2.0 ** -24
        return
    assert np.max(np.abs(lam - ref[:m])) <= LAM_TOL, np.max(np.abs(lam - ref[:m]))
    assert abs(eg - g["E_G"]) <= EG_RTOL * abs(g["E_G"]), (eg, g["E_G"])
    checked = 0
    for j in range(m):
        d_lo = rq[j] - ref[j - 1] if j > 0 else np.inf
        d_hi = ref[j + 1] - rq[j]
        if min(d_lo, d_hi) <= 10 * r[j]:
            continue
        assert rq[j] - r[j] ** 2 / d_hi - dot_slack[j] <= ref[j] <= \
            rq[j] + r[j] ** 2 / d_lo + dot_slack[j], (j, rq[j], ref[j], r[j])
        checked += 1
    assert checked >= m // 2
    # the stopping rule, recomputed in FP64 on the host: ||R||_2 <= ||R||_F
    # = sqrt(m) RMS (twice, for the solver's own residual rounding)
    assert r2 <= 2 * np.sqrt(m) * SOLVE_TOL, r2
    gap = ref[m] - lam[m - 1]
    assert r2 / gap <= ANGLE_TOL, (r2, gap)


def _solve_large(trm, name, csr, C0=None):
    torch = gu.torch_mod()
    g = _reference(name)
    w = ti.workload(name, seed=g["seed"])
    V = w.potential()
    side = torch.cuda.Stream()
    opts = dict(precision=trm.TRM_MIXED, precond=1, seed=w.seed + 100,
                stream=side.cuda_stream)
    with torch.cuda.stream(side):
        if csr:
            rp, ci, va = ti.grid_csr(w.shape, w.order, w.h, V, np.float32)
            import scipy.sparse as sp
            H = sp.csr_matrix((va.astype(np.float64), ci, rp), shape=(w.N, w.N))
            s = trm.Solver.csr(w.N, rp, ci, va, w.m, SOLVE_TOL, **opts)
        else:
            H = op.grid_hamiltonian(w.shape, w.order, w.h, V)
            s = trm.Solver.stencil(w.shape, w.order, w.h, V, w.m, SOLVE_TOL,
                                  **opts)
        with s:
            lam, eg, C, st, status = s.solve(C0=C0)
    side.synchronize()
    assert status == 0, st
    return g, w, H, lam, eg, C, st


@pytest.mark.parametrize("key", ["grid96_m512", "grid100_m1024"])
def test_whole_solve_a_posteriori(trm, key):
    """A cold mixed-precision solve to an RMS residual of 1e-10 (as bench.py
    launches it: diagonal preconditioner, iteration graphs on a side stream).
    The oracle, in FP64 from the GPU's C: C^T C = I to 1e-12; the Ritz values
    theta of C^T (H C) equal the returned lambda to 1e-9 and their sum E_G to
    1e-10; against the stored reference (lambda_1..lambda_{m+4}): every
    lambda_j to 1e-9 and E_G to 1e-10; Kato-Temple: with q_j the Rayleigh
    quotient of the returned column c_j and r_j = ||H c_j - q_j c_j||, where
    the reference neighbours lie further than 10 r_j away, lambda_ref_j is
    in [q_j - r_j^2 / d_hi, q_j + r_j^2 / d_lo] (widened by the rounding of
    the host's N-term dots); ||R||_2 = ||H C - C diag(lambda)||_2 within
    twice the sqrt(m) 1e-10 the stopping rule allows; Davis-Kahan: the
    largest principal angle to the exact invariant subspace is at most
    ||R||_2 / (lambda_ref_{m+1} - theta_m) <= 2e-5 (FP32-class subspaces sit
    near 1e-3)."""
    name, _ = CASES[key]
    g, w, H, lam, eg, C, st = _solve_large(trm, name, False)
    _a_posteriori(H, lam, eg, C, g, w.m, True)
    _SOLVED[name] = C


def test_whole_solve_csr_warm_start_a_posteriori(trm):
    """The 100^3, m = 1024 operator as an explicit CSR matrix (FP32 values,
    int32 columns), solved from the stencil solve's converged block (the
    warm start of related requests; a cold solve at this size takes about
    six minutes): the same a-posteriori checks against the matrix the GPU
    holds, and its eigenvalues within the FP32 rounding of the entries of
    the reference's."""
    name = "grid100_o4_w1000_m1024"
    C0 = _SOLVED.get(name)
    if C0 is None:
        C0 = _solve_large(trm, name, False)[5]
    g, w, H, lam, eg, C, st = _solve_large(trm, name, True, C0=C0)
    _a_posteriori(H, lam, eg, C, g, w.m, False)
