"""Generalized problem H e = lambda S e through the C ABI (S the overlap of
trilinear hat functions, trm_set_overlap_csr): the eigenvalues equal the
closed form of the V = 0 pencil and the oracle's generalized
eigensolutions, the returned C is S-orthonormal with small residuals
||H c - lambda S c||, stencil and CSR forms of H agree, in the FP64 mode,
the mixed ladder (full SP with S in FP32, then FP64) and full SP, and the
handle refuses what the generalized path does not cover."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import trm_inputs as ti
from oracle import operator as op

from . import gpu_util as gu
from .test_oracle import _hat_closed_form

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


def _overlap(shape):
    rp, ci, v = ti.hat_overlap_csr(shape)
    N = int(np.prod(shape))
    return (rp, ci, v), sp.csr_matrix((v, ci, rp), shape=(N, N))


def _solve(trm, shape, order, V, m, S_arrays, precond, csr=False,
           tol=1e-10, precision=None):
    N = int(np.prod(shape))
    if precision is None:
        precision = trm.TRM_FP64
    opt = trm.trm_default_options(precision=precision, precond=precond,
                                  seed=5)
    opt.stream = gu.stream()
    if csr:
        rp, ci, v = ti.grid_csr(shape, order, 1.0, V)
        h = trm.trm_create_csr(N, rp, ci, v, m, tol, opt)
    else:
        h = trm.trm_create_stencil(*shape, order, 1.0, V, m, tol, opt)
    try:
        trm.trm_set_overlap_csr(h, *S_arrays)
        C = np.zeros((N, m), order="F")
        lam, _, st, status = trm.trm_solve(h, N, m, C_out=C)
    finally:
        trm.trm_destroy(h)
    assert status == 0
    return lam, C, st


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", [0, 1])
def test_closed_form_pencil(trm, precond, mode):
    shape, m = (10, 11, 12), 8
    S_arrays, S = _overlap(shape)
    prec = trm.TRM_FP64 if mode == "fp64" else trm.TRM_MIXED
    lam, C, st = _solve(trm, shape, 2, np.zeros(int(np.prod(shape))), m,
                        S_arrays, precond, precision=prec)
    if mode == "mixed":
        assert st.iterations_phase[0] > 0  # a full-SP phase ran first
    want = _hat_closed_form(shape, 1.0)[:m]
    assert np.max(np.abs(lam - want)) < 1e-10 * np.abs(want).max()
    assert np.max(np.abs(C.T @ (S @ C) - np.eye(m))) < 1e-10
    assert st.max_residual < 1e-8


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("csr", [False, True])
def test_wells_against_dense_generalized_eigh(trm, csr, mode):
    shape, order, m = (12, 12, 12), 4, 10
    V = ti.gaussian_wells(shape, 6, seed=2)
    S_arrays, S = _overlap(shape)
    prec = trm.TRM_FP64 if mode == "fp64" else trm.TRM_MIXED
    lam, C, st = _solve(trm, shape, order, V, m, S_arrays, 1, csr=csr,
                        precision=prec)
    H = op.grid_hamiltonian(shape, order, 1.0, V)
    want = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True,
                    subset_by_index=[0, m - 1])
    assert np.max(np.abs(lam - want)) < 1e-9
    assert np.max(np.abs(C.T @ (S @ C) - np.eye(m))) < 1e-10
    R = H @ C - (S @ C) * lam[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) < 1e-7


def test_full_sp_pencil(trm):
    """Full SP with S: the FP32 iteration stops at its floor (tolerance
    1e-4 on the RMS residual) and the closing FP64 Rayleigh-Ritz step on
    its span gives eigenvalues within r^2 / gap of the dense ones and an
    S-orthonormal block."""
    shape, order, m = (12, 12, 12), 4, 10
    V = ti.gaussian_wells(shape, 6, seed=2)
    S_arrays, S = _overlap(shape)
    lam, C, st = _solve(trm, shape, order, V, m, S_arrays, 1, tol=1e-4,
                        precision=trm.TRM_FULL_SP)
    H = op.grid_hamiltonian(shape, order, 1.0, V)
    want = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True,
                    subset_by_index=[0, m - 1])
    assert np.max(np.abs(lam - want)) < 1e-5
    assert np.max(np.abs(C.T @ (S @ C) - np.eye(m))) < 1e-10


def test_ragged_grid_against_shift_invert_lanczos(trm):
    shape, m = (20, 18, 23), 24
    N = int(np.prod(shape))
    V = ti.gaussian_wells(shape, 10, seed=3)
    S_arrays, S = _overlap(shape)
    lam, C, _ = _solve(trm, shape, 2, V, m, S_arrays, 1)
    H = op.grid_hamiltonian(shape, 2, 1.0, V)
    w = spla.eigsh(H.tocsc(), k=m + 1, M=S.tocsc(), sigma=-3.0, which="LM",
                   tol=0)[0]
    want = np.sort(w)[:m]
    assert np.max(np.abs(lam - want)) < 1e-9
    assert np.max(np.abs(C.T @ (S @ C) - np.eye(m))) < 1e-10
    assert N == 8280


def test_refusals(trm):
    shape, m = (6, 6, 6), 4
    N = int(np.prod(shape))
    S_arrays, _ = _overlap(shape)
    opt = trm.trm_default_options(precision=trm.TRM_MP2)
    opt.stream = gu.stream()
    h = trm.trm_create_stencil(*shape, 2, 1.0, None, m, 1e-8, opt)
    try:
        with pytest.raises(trm.TrmError) as e:
            trm.trm_set_overlap_csr(h, *S_arrays)
        assert e.value.status == -1
    finally:
        trm.trm_destroy(h)
    opt = trm.trm_default_options(precision=trm.TRM_FP64)
    opt.stream = gu.stream()
    h = trm.trm_create_stencil(*shape, 2, 1.0, None, m, 1e-8, opt)
    try:
        rp, ci, v = S_arrays
        bad = v.copy()
        bad[rp[3]:rp[4]] = 0.0                     # row 3 loses its diagonal
        with pytest.raises(trm.TrmError) as e:
            trm.trm_set_overlap_csr(h, rp, ci, bad)
        assert e.value.status == -1
        trm.trm_set_overlap_csr(h, *S_arrays)
        with pytest.raises(trm.TrmError) as e:
            trm.trm_iterate(h, trm.TRM_FP64)
        assert e.value.status == -1
    finally:
        trm.trm_destroy(h)
