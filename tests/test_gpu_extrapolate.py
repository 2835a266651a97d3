"""Initial-guess extrapolation through the C ABI (trm_extrapolate): the
device result equals the oracle's element by element, a singular alignment
is reported, and in a chain of related solves the extrapolated block starts
closer to the next solution than the previous block does."""
import numpy as np
import pytest

import trm_inputs as ti
from oracle import operator as op
from oracle import trm as otrm

from . import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


def _related(N, m, seed, eps):
    """An orthonormal C_prev and C_cur = orth(C_prev Q + a perturbation of
    column norm about eps), Q a random rotation."""
    rng = np.random.default_rng(seed)
    C0 = otrm.orthonormalize(rng.standard_normal((N, m)))
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    B = rng.standard_normal((N, m)) * (eps / np.sqrt(N))
    return C0, otrm.orthonormalize(C0 @ Q + B)


# several 128-row tiles with a ragged tail, tiny N, m above a warp, m = 128
@pytest.mark.parametrize("N,m,alpha", [(4099, 37, 1.0), (1000, 8, 0.5),
                                       (20011, 64, 1.0), (300, 128, 2.0)])
def test_extrapolate_matches_oracle(trm, N, m, alpha):
    C0, C1 = _related(N, m, N + m, 0.1)
    want = otrm.extrapolate(C0, C1, alpha)
    d0, d1 = gu.to_dev(C0), gu.to_dev(C1)
    dn = gu.empty(N, m, np.float64)
    trm.trm_extrapolate(N, m, d0.data_ptr(), d1.data_ptr(), alpha,
                        dn.data_ptr(), gu.stream())
    got = gu.from_dev(dn)
    assert np.max(np.abs(got - want)) < 1e-11
    assert np.max(np.abs(got.T @ got - np.eye(m))) < 1e-12


def test_extrapolate_reports_a_singular_alignment(trm):
    """span(C_cur) holds a direction orthogonal to span(C_prev): C_prev^T
    C_cur has a zero singular value and no unique alignment exists."""
    N, m = 64, 4
    eye = np.eye(N)
    C0 = eye[:, :m]
    C1 = np.concatenate([eye[:, :m - 1], eye[:, m:m + 1]], axis=1)
    d0, d1 = gu.to_dev(C0), gu.to_dev(C1)
    dn = gu.empty(N, m, np.float64)
    with pytest.raises(trm.TrmError) as e:
        trm.trm_extrapolate(N, m, d0.data_ptr(), d1.data_ptr(), 1.0,
                            dn.data_ptr(), gu.stream())
    assert e.value.status == -3


def test_chain_of_related_solves(trm):
    """V(t) = V0 + t V1 at t = 0, dt, 2 dt (16^3, 7-point, m = 12): the
    block extrapolated from the first two solutions is closer to the third
    than the second solution is, and every start reaches the oracle's
    eigenvalues."""
    n, order, m, dt = 16, 2, 12, 0.02
    shape, N = (n, n, n), n ** 3
    V0 = ti.gaussian_wells(shape, 8, seed=31)
    V1 = ti.gaussian_wells(shape, 8, seed=32)

    def solve(t, C0=None):
        opt = trm.trm_default_options(precision=trm.TRM_MIXED, precond=1,
                                      seed=3)
        opt.stream = gu.stream()
        h = trm.trm_create_stencil(n, n, n, order, 1.0, V0 + t * V1, m, 1e-9,
                                   opt)
        C = np.zeros((N, m), order="F")
        try:
            lam, _, st, status = trm.trm_solve(h, N, m, C_out=C, C0=C0)
        finally:
            trm.trm_destroy(h)
        assert status == 0
        return lam, C, st.iterations

    _, Ca, _ = solve(0.0)
    _, Cb, _ = solve(dt)
    dA, dB = gu.to_dev(Ca), gu.to_dev(Cb)
    dX = gu.empty(N, m, np.float64)
    trm.trm_extrapolate(N, m, dA.data_ptr(), dB.data_ptr(), 1.0,
                        dX.data_ptr(), gu.stream())
    Cx = gu.from_dev(dX)
    assert np.max(np.abs(Cx - otrm.extrapolate(Ca, Cb))) < 1e-11
    lam_c, Cc, it_c = solve(2 * dt)
    lam_p, _, it_p = solve(2 * dt, Cb)
    lam_x, _, it_x = solve(2 * dt, Cx)
    ref = op.lowest_eigenvalues(
        op.grid_hamiltonian(shape, order, 1.0, V0 + 2 * dt * V1), m)
    for lam in (lam_c, lam_p, lam_x):
        assert np.max(np.abs(lam - ref)) < 1e-9
    e_prev = otrm.sin_max_angle(Cb, Cc)
    e_extr = otrm.sin_max_angle(Cx, Cc)
    assert e_extr < 0.5 * e_prev, (e_extr, e_prev)
    assert it_x < it_c and it_p < it_c, (it_c, it_p, it_x)
