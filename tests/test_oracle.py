"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties a piece of the oracle to a closed form, a value printed in the
paper, brute-force dense diagonalisation, a finite difference or an invariant,
chosen so that a dropped term, a wrong sign or index or a transposed operand in
the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import trm_inputs as ti
from oracle import filtered
from oracle import operator as op
from oracle import trm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _edge_m(lam, lo, hi, min_gap=1e-3):
    """Smallest m in [lo, hi] with lambda_{m+1} - lambda_m >= min_gap."""
    for m in range(lo, hi + 1):
        if lam[m] - lam[m - 1] >= min_gap:
            return m
    raise AssertionError("no gapped m in range")


# ---------------------------------------------------------------------------
# Operator and closed forms (Sec. 3, Eq. LAPLACE and the eigenvalue formula)
# ---------------------------------------------------------------------------
def test_laplace_block_form_equals_kronecker_form():
    n = 9
    A = op.laplace2d(n).toarray()
    B = op.grid_hamiltonian((n, n, 1), 2, math.sqrt(0.5)).toarray()
    assert np.allclose(A, B, rtol=0, atol=1e-15)
    assert np.allclose(np.diag(A), 4.0)
    assert A[0, 1] == -1.0 and A[0, n] == -1.0 and A[n - 1, n] == 0.0


def test_laplace_closed_form_vs_dense():
    for n in (5, 12):
        dense = op.dense_spectrum(op.laplace2d(n))
        assert np.allclose(op.laplace2d_spectrum(n), dense, atol=1e-12)


def test_order2_closed_form_vs_dense():
    shape = (7, 6, 5)
    dense = op.dense_spectrum(op.grid_hamiltonian(shape, 2, 1.3))
    assert np.allclose(op.order2_spectrum(shape, 1.3), dense, atol=1e-12)


def test_order4_kronecker_spectrum_vs_dense():
    shape = (7, 6, 5)
    dense = op.dense_spectrum(op.grid_hamiltonian(shape, 4, 0.9))
    assert np.allclose(op.kron_sum_spectrum(shape, 4, 0.9), dense, atol=1e-12)


def test_table_restbl_E_G_and_gap_from_closed_form():
    """E_G = sum of the m lowest lambda_{p,q} and eps_gap = lambda_{m+1} - lambda_m
    reproduce the printed columns of Table RESTBL to the printed figures."""
    tab = json.load(open(os.path.join(GOLDEN, "table_restbl.json")))
    for row in tab["rows"]:
        lam = op.laplace2d_spectrum(row["n"])
        m = row["m"]
        E = float(np.sum(lam[:m]))
        gap = lam[m] - lam[m - 1]
        assert float(f"{E:.{row['E_G_sig']}g}") == pytest.approx(row["E_G"], rel=1e-12)
        assert float(f"{gap:.{row['gap_sig']}g}") == pytest.approx(row["gap"], rel=1e-12)


def test_table_restbl_reference_file_matches_the_closed_form():
    """tests/golden/table_restbl_reference.json (the E_G references bench.py
    --table compares against) holds the closed form's values for every row
    of the printed table, and they round to the printed E_G."""
    ref = json.load(open(os.path.join(GOLDEN, "table_restbl_reference.json")))
    tab = json.load(open(os.path.join(GOLDEN, "table_restbl.json")))
    assert [(r["n"], r["m"]) for r in ref["rows"]] == \
        [(r["n"], r["m"]) for r in tab["rows"]]
    for r, t in zip(ref["rows"], tab["rows"]):
        lam = op.laplace2d_spectrum(r["n"])
        m = r["m"]
        assert r["E_G"] == float(np.sum(lam[:m]))
        assert r["lambda_m"] == float(lam[m - 1])
        assert r["gap"] == float(lam[m] - lam[m - 1])
        assert float(f"{r['E_G']:.{t['E_G_sig']}g}") == pytest.approx(t["E_G"], rel=1e-12)


# ---------------------------------------------------------------------------
# Fig. ONFIG
# ---------------------------------------------------------------------------
def test_orthonormalize_is_orthonormal_and_keeps_span():
    C = ti.random_block(400, 9, seed=5)
    Q = trm.orthonormalize(C)
    assert np.max(np.abs(Q.T @ Q - np.eye(9))) < 1e-13
    assert trm.sin_max_angle(C, Q) < 1e-12
    # Q = C U^{-1} with U upper triangular: Q^T C is upper triangular
    R = Q.T @ C
    assert np.max(np.abs(np.tril(R, -1))) < 1e-12


def test_printed_onfig_product_is_not_orthonormal():
    """The literal C_in L^{-1} of Fig. ONFIG step (4) fails C^T C = I for a
    generic C; the transposed product (the reading used) passes."""
    C = ti.random_block(50, 4, seed=9)
    L = np.linalg.cholesky(C.T @ C)
    Li = np.linalg.inv(L)
    assert np.max(np.abs((C @ Li).T @ (C @ Li) - np.eye(4))) > 1e-3
    assert np.max(np.abs((C @ Li.T).T @ (C @ Li.T) - np.eye(4))) < 1e-13


# ---------------------------------------------------------------------------
# Fig. EGFIG
# ---------------------------------------------------------------------------
def _small_problem(seed=1, shape=(6, 5, 4), order=4, m=5):
    V = ti.gaussian_wells(shape, 3, seed=seed)
    H = op.grid_hamiltonian(shape, order, 1.0, V)
    C = trm.orthonormalize(ti.random_block(H.shape[0], m, seed=seed + 100))
    return H, C


def test_energy_is_sum_of_rayleigh_terms():
    H, C = _small_problem()
    Hd = H.toarray()
    E, G, X, Hc = trm.energy_gradient_alg1(H, C)
    E_direct = sum(float(C[:, j] @ Hd @ C[:, j]) for j in range(C.shape[1]))
    assert E == pytest.approx(E_direct, rel=1e-13)


def test_algorithm1_equals_algorithm2():
    H, C = _small_problem()
    E1, G1, _, _ = trm.energy_gradient_alg1(H, C)
    E2, G2, _, HD, Xp, Hp = trm.energy_gradient_alg2(H, C)
    assert E1 == pytest.approx(E2, rel=1e-14)
    assert np.max(np.abs(G1 - G2)) < 1e-12
    # with C^T C = I, H' has (numerically) zero diagonal, so zeroing it is harmless
    assert np.max(np.abs(np.diag(Hp))) < 1e-13
    _, G3, _, _, _, _ = trm.energy_gradient_alg2(H, C, zero_diag=True)
    assert np.max(np.abs(G3 - G1)) < 1e-12


def test_gradient_is_minus_directional_derivative():
    """d/de E(orthonormalize(C + e D)) at e = 0 equals -tr(D^T G)."""
    H, C = _small_problem()
    E, G, _, _ = trm.energy_gradient_alg1(H, C)
    D = ti.random_block(C.shape[0], C.shape[1], seed=77)
    eps = 1e-5
    Ep = trm.energy_gradient_alg1(H, trm.orthonormalize(C + eps * D))[0]
    Em = trm.energy_gradient_alg1(H, trm.orthonormalize(C - eps * D))[0]
    fd = (Ep - Em) / (2 * eps)
    assert fd == pytest.approx(-float(np.sum(D * G)), rel=1e-7)


def test_gradient_orthogonal_to_C_and_trace_invariance():
    H, C = _small_problem()
    E, G, _, _ = trm.energy_gradient_alg1(H, C)
    assert np.max(np.abs(C.T @ G)) < 1e-12
    Q, _ = np.linalg.qr(ti.random_block(C.shape[1], C.shape[1], seed=3))
    E_rot, G_rot, _, _ = trm.energy_gradient_alg1(H, C @ Q)
    assert E_rot == pytest.approx(E, rel=1e-13)
    assert np.max(np.abs(G_rot - G @ Q)) < 1e-12


# ---------------------------------------------------------------------------
# Line minimization
# ---------------------------------------------------------------------------
def _line_setup():
    H, C = _small_problem(m=4)
    E, G, X, _ = trm.energy_gradient_alg1(H, C)
    P = G
    HP = op.apply_h(H, P)
    return H, C, P, G, trm.line_matrices(C, P, X, HP)


def test_line_energy_equals_explicit_orthonormalize_and_evaluate():
    H, C, P, G, M = _line_setup()
    for a in (0.0, 0.05, 0.3, 1.2):
        explicit = trm.energy_gradient_alg1(H, trm.orthonormalize(C + a * P))[0]
        assert trm.line_energy(a, M) == pytest.approx(explicit, rel=1e-12)


def test_line_slope_matches_finite_difference_and_gradient():
    H, C, P, G, M = _line_setup()
    assert trm.line_slope(0.0, M) == pytest.approx(-float(np.sum(G * P)), rel=1e-10)
    for a in (0.02, 0.2, 0.7):
        h = 1e-5 * max(a, 1e-3)
        fd = (trm.line_energy(a + h, M) - trm.line_energy(a - h, M)) / (2 * h)
        assert trm.line_slope(a, M) == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_line_minimize_finds_minimum():
    H, C, P, G, M = _line_setup()
    a, g0 = trm.line_minimize(M, 1e-3)
    assert g0 < 0 and a > 0
    assert abs(trm.line_slope(a, M)) <= 1e-8 * abs(g0)
    Ea = trm.line_energy(a, M)
    for b in np.linspace(0.0, 3 * a, 31):
        assert Ea <= trm.line_energy(b, M) + 1e-13


# ---------------------------------------------------------------------------
# Rayleigh-Ritz and the full loop (Fig. TMFIG)
# ---------------------------------------------------------------------------
def test_rayleigh_ritz_on_exact_eigenvectors():
    H, _ = _small_problem()
    w, Z = sla.eigh(H.toarray())
    m = 5
    Q, _ = np.linalg.qr(ti.random_block(m, m, seed=8))
    lam, Cr, res = trm.rayleigh_ritz(H, Z[:, :m] @ Q * 3.0)
    assert np.allclose(lam, w[:m], atol=1e-12)
    assert np.max(res) < 1e-12
    assert np.max(np.abs(Cr.T @ Cr - np.eye(m))) < 1e-12


def test_solve_laplace2d_vs_closed_form():
    n = 20
    lam_ex = op.laplace2d_spectrum(n)
    m = _edge_m(lam_ex, 12, 40, min_gap=2e-2)
    H = op.laplace2d(n)
    res = trm.solve(H, ti.random_block(n * n, m, seed=2), tol=1e-10)
    assert res.converged
    assert res.E_G == pytest.approx(float(np.sum(lam_ex[:m])), rel=1e-12)
    assert np.max(np.abs(res.lam - lam_ex[:m])) < 1e-10
    # energies decrease monotonically with an exact line search in FP64
    e = np.array(res.energies)
    assert np.all(np.diff(e) <= 1e-12 * np.abs(e[1:]))


def test_solve_order2_3d_vs_closed_form():
    shape = (8, 7, 6)
    lam_ex = op.order2_spectrum(shape, 1.0)
    m = _edge_m(lam_ex, 8, 30, min_gap=1e-2)
    H = op.grid_hamiltonian(shape, 2, 1.0)
    res = trm.solve(H, ti.random_block(H.shape[0], m, seed=4), tol=1e-10)
    assert res.converged
    assert res.E_G == pytest.approx(float(np.sum(lam_ex[:m])), rel=1e-12)
    assert np.max(np.abs(res.lam - lam_ex[:m])) < 1e-10


def test_solve_order4_wells_vs_dense_and_preconditioned():
    shape = (8, 8, 8)
    V = ti.gaussian_wells(shape, 6, seed=3)
    H = op.grid_hamiltonian(shape, 4, 1.0, V)
    dense = op.dense_spectrum(H)
    m = _edge_m(dense, 10, 30, min_gap=1e-2)
    C0 = ti.random_block(512, m, seed=6)
    for pc in (False, True):
        res = trm.solve(H, C0, tol=1e-10, precond=pc)
        assert res.converged
        assert res.E_G == pytest.approx(float(np.sum(dense[:m])), rel=1e-12)
        assert np.max(np.abs(res.lam - dense[:m])) < 1e-10
        assert np.max(res.residuals) < 1e-8


def test_ritz_values_interlace_before_convergence():
    """Cauchy interlacing: on any m-dimensional subspace the Ritz values are
    bounded below by the exact lambda_j, and E_i >= E_G."""
    shape = (7, 7, 7)
    H = op.grid_hamiltonian(shape, 4, 1.0, ti.gaussian_wells(shape, 4, seed=2))
    dense = op.dense_spectrum(H)
    res = trm.solve(H, ti.random_block(343, 10, seed=1), tol=0.0, max_iter=8)
    assert not res.converged
    assert np.all(res.lam >= dense[:10] - 1e-12)
    assert min(res.energies) >= float(np.sum(dense[:10])) - 1e-12


def test_polak_ribiere_beats_steepest_descent():
    """With the Polak-Ribiere term the loop converges far faster than with
    gamma = 0; a sign or index slip in gamma would not."""
    n = 16
    lam_ex = op.laplace2d_spectrum(n)
    m = _edge_m(lam_ex, 10, 30, min_gap=2e-2)
    H = op.laplace2d(n)
    C0 = ti.random_block(n * n, m, seed=7)
    cg = trm.solve(H, C0, tol=1e-8)
    sd = trm.solve(H, C0, tol=1e-8, cg=False, max_iter=3 * cg.iterations)
    assert cg.converged
    assert (not sd.converged) or sd.iterations > 2 * cg.iterations



def test_polak_ribiere_restarts_itself_when_the_gradient_repeats():
    """Polak-Ribiere's known property (as against Fletcher-Reeves, which
    gives 1): a gradient that repeats the previous one gives gamma = 0, and
    gamma is unchanged when both gradients are scaled by the same factor and
    is linear in the new gradient's change; with M-orthogonal gradients it
    reduces to the Fletcher-Reeves ratio."""
    rng = np.random.default_rng(4)
    G = rng.standard_normal((50, 3))
    Gp = rng.standard_normal((50, 3))
    Md = 0.5 + rng.random(50)
    M = lambda X: X * Md[:, None]                       # noqa: E731
    assert trm.polak_ribiere(G, G, M(G), M(G)) == 0.0
    g = trm.polak_ribiere(G, Gp, M(G), M(Gp))
    assert trm.polak_ribiere(3 * G, 3 * Gp, M(3 * G), M(3 * Gp)) == \
        pytest.approx(g, rel=1e-13)
    # make G M-orthogonal to Gp: then gamma = tr(G^T M G) / tr(Gp^T M Gp)
    Go = G - Gp * (np.sum(Gp * M(G)) / np.sum(Gp * M(Gp)))
    fr = np.sum(Go * M(Go)) / np.sum(Gp * M(Gp))
    assert trm.polak_ribiere(Go, Gp, M(Go), M(Gp)) == pytest.approx(fr,
                                                                    rel=1e-12)

# ----------------------------------------------------------------------------
# Initial-guess extrapolation for a chain of related problems
# ----------------------------------------------------------------------------
def _rotation(m, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))
    return q * np.sign(np.diag(r))


def _subspace_path(N, m, seed):
    """A smooth family of m-dimensional subspaces with a closed form:
    C(t) = exp(t K) E_m (K skew, E_m the first m unit vectors)."""
    K = np.random.default_rng(seed).standard_normal((N, N))
    K = (K - K.T) / (2.0 * math.sqrt(N))
    E = np.eye(N)[:, :m]
    return lambda t: sla.expm(t * K) @ E


def test_procrustes_recovers_a_rotation_and_minimises():
    N, m = 80, 6
    C = trm.orthonormalize(np.random.default_rng(3).standard_normal((N, m)))
    Q = _rotation(m, 4)
    U = trm.procrustes(C, C @ Q)
    assert np.max(np.abs(U - Q)) < 1e-13          # U^T would fail here
    B = trm.orthonormalize(C + 0.3 * np.random.default_rng(5).standard_normal((N, m)))
    U = trm.procrustes(C, B)
    assert np.max(np.abs(U.T @ U - np.eye(m))) < 1e-13
    best = np.linalg.norm(C @ U - B)
    rng = np.random.default_rng(6)
    for _ in range(30):
        S = rng.standard_normal((m, m)) * 0.05
        W = sla.expm(S - S.T)
        assert np.linalg.norm(C @ U @ W - B) >= best - 1e-12


def test_extrapolate_keeps_a_stationary_subspace():
    N, m = 70, 5
    C = trm.orthonormalize(np.random.default_rng(7).standard_normal((N, m)))
    assert np.max(np.abs(trm.extrapolate(C @ _rotation(m, 8), C) - C)) < 1e-13
    assert np.max(np.abs(trm.extrapolate(
        trm.orthonormalize(C + 0.1), C, alpha=0.0) - C)) < 1e-13


def test_extrapolate_is_second_order_along_a_smooth_path():
    """The previous block is off the next subspace by O(dt), the extrapolated
    one by O(dt^2): halving dt halves the first error and quarters the
    second, whatever basis each block is given in."""
    N, m = 60, 5
    C = _subspace_path(N, m, 9)
    e_prev, e_extr = [], []
    for k, dt in enumerate((0.04, 0.02, 0.01)):
        C0 = C(0.0) @ _rotation(m, 10 + k)
        C1 = C(dt) @ _rotation(m, 20 + k)
        e_prev.append(trm.sin_max_angle(C1, C(2 * dt)))
        e_extr.append(trm.sin_max_angle(trm.extrapolate(C0, C1), C(2 * dt)))
    for a, b in zip(e_prev, e_prev[1:]):
        assert 1.8 < a / b < 2.2
    for a, b in zip(e_extr, e_extr[1:]):
        assert 3.5 < a / b < 4.5
    assert e_extr[-1] < 0.05 * e_prev[-1]


def test_extrapolate_is_equivariant_under_basis_changes():
    N, m = 50, 4
    C = _subspace_path(N, m, 11)
    C0, C1 = C(0.0), C(0.1)
    Q0, Q1 = _rotation(m, 12), _rotation(m, 13)
    a = trm.extrapolate(C0, C1, alpha=0.7)
    b = trm.extrapolate(C0 @ Q0, C1 @ Q1, alpha=0.7)
    assert trm.sin_max_angle(a, b) < 1e-13


# ----------------------------------------------------------------------------
# Generalized problem H e = lambda S e (S SPD: hat-function overlap)
# ----------------------------------------------------------------------------
def _overlap(shape):
    import scipy.sparse as sp
    rp, ci, v = ti.hat_overlap_csr(shape)
    N = int(np.prod(shape))
    return sp.csr_matrix((v, ci, rp), shape=(N, N))


def _hat_closed_form(shape, h):
    """V = 0, order 2: H and S are tensor products of tridiagonal Toeplitz
    matrices with the common eigenvectors sin(j k pi / (n + 1)), so
    lambda = sum_a t (2 - 2 cos th_a) / prod_a (4 + 2 cos th_a) / 6."""
    t = 0.5 / (h * h)
    ths = [np.pi * np.arange(1, n + 1) / (n + 1) for n in shape]
    num = sum(np.meshgrid(*[t * (2 - 2 * np.cos(th)) for th in ths],
                          indexing="ij"))
    den = np.prod(np.meshgrid(*[(4 + 2 * np.cos(th)) / 6 for th in ths],
                              indexing="ij"), axis=0)
    return np.sort((num / den).ravel())


def test_hat_overlap_is_the_tensor_product_and_spd():
    shape = (5, 4, 6)
    S = _overlap(shape).toarray()
    T = [np.diag(np.full(n, 4 / 6)) + np.diag(np.full(n - 1, 1 / 6), 1)
         + np.diag(np.full(n - 1, 1 / 6), -1) for n in shape]
    K = np.kron(T[2], np.kron(T[1], T[0]))       # x fastest
    assert np.max(np.abs(S - K)) == 0.0
    w = np.linalg.eigvalsh(S)
    assert w.min() > 0.0 and np.allclose(S, S.T)


def test_generalized_dense_spectrum_equals_closed_form():
    shape, h = (5, 4, 6), 1.0
    H = op.grid_hamiltonian(shape, 2, h).toarray()
    S = _overlap(shape).toarray()
    lam = sla.eigh(H, S, eigvals_only=True)
    assert np.max(np.abs(lam - _hat_closed_form(shape, h))) < 1e-12


def test_generalized_gradient_is_minus_constrained_derivative():
    """C^T S C = I: d/de E(orthonormalize_S(C + e D)) at e = 0 is
    -tr(D^T G) with G = -2 (H C - S C H_C); C^T G = 0 still holds."""
    shape = (6, 5, 4)
    N, m = int(np.prod(shape)), 4
    H = op.grid_hamiltonian(shape, 2, 1.0, ti.gaussian_wells(shape, 3, seed=5))
    S = _overlap(shape)
    C = trm.orthonormalize(ti.random_block(N, m, seed=6), S)
    assert np.max(np.abs(C.T @ (S @ C) - np.eye(m))) < 1e-13
    E, G, _, _ = trm.energy_gradient_alg1(H, C, S)
    E2, G2, _, _, _, _ = trm.energy_gradient_alg2(H, C, S=S)
    assert E2 == pytest.approx(E, rel=1e-13)
    assert np.max(np.abs(G2 - G)) < 1e-12
    assert np.max(np.abs(C.T @ G)) < 1e-12
    D = ti.random_block(N, m, seed=78)
    eps = 1e-5
    Ep = trm.energy_gradient_alg1(H, trm.orthonormalize(C + eps * D, S), S)[0]
    Em = trm.energy_gradient_alg1(H, trm.orthonormalize(C - eps * D, S), S)[0]
    assert (Ep - Em) / (2 * eps) == pytest.approx(-float(np.sum(D * G)),
                                                  rel=1e-7)
    # the line-search overlap is that of the S-orthonormalized pencil
    P = ti.random_block(N, m, seed=79)
    LM = trm.line_matrices(C, P, H @ C, H @ P, S)
    a = 0.3
    Y = C + a * P
    assert np.max(np.abs(LM.S0 + a * (LM.B + LM.B.T) + a * a * LM.Q
                         - Y.T @ (S @ Y))) < 1e-12


@pytest.mark.parametrize("precond", [False, True])
def test_generalized_solve_vs_dense_and_closed_form(precond):
    shape = (7, 6, 8)
    N, m = int(np.prod(shape)), 6
    S = _overlap(shape)
    H0 = op.grid_hamiltonian(shape, 2, 1.0)
    r = trm.solve(H0, ti.random_block(N, m, seed=1), tol=1e-11,
                  precond=precond, S=S)
    assert r.converged
    want = _hat_closed_form(shape, 1.0)[:m]
    assert np.max(np.abs(r.lam - want)) < 1e-10 * abs(want).max()
    H = op.grid_hamiltonian(shape, 4, 1.0, ti.gaussian_wells(shape, 6, seed=2))
    r = trm.solve(H, ti.random_block(N, m, seed=3), tol=1e-11,
                  precond=precond, S=S)
    assert r.converged
    lam = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True,
                   subset_by_index=[0, m - 1])
    assert np.max(np.abs(r.lam - lam)) < 1e-10
    assert np.max(np.abs(r.C.T @ (S @ r.C) - np.eye(m))) < 1e-12
    assert r.residuals.max() < 1e-9


def test_generalized_with_diagonal_S_is_the_scaled_standard_problem():
    """S = D diagonal: H e = lambda D e is D^{-1/2} H D^{-1/2} f = lambda f."""
    import scipy.sparse as sp
    shape = (6, 6, 6)
    N, m = int(np.prod(shape)), 5
    d = 0.5 + ti.uniform01(9, np.arange(N))
    H = op.grid_hamiltonian(shape, 2, 1.0, ti.gaussian_wells(shape, 4, seed=8))
    r = trm.solve(H, ti.random_block(N, m, seed=4), tol=1e-11, precond=True,
                  S=sp.diags(d).tocsr())
    Hs = H.toarray() / np.sqrt(d)[:, None] / np.sqrt(d)[None, :]
    assert np.max(np.abs(r.lam - np.linalg.eigvalsh(Hs)[:m])) < 1e-10


# ----------------------------------------------------------------------------
# Stencil consistency, independent of the weights' own spectra
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("order,rate", [(2, 4.0), (4, 16.0)])
def test_stencil_truncation_error_has_the_rule_order(order, rate):
    """H u for u = sin(pi x) sin(2 pi y) sin(3 pi z) sampled on the unit cube
    equals -1/2 lap u = pi^2 (1 + 4 + 9) / 2 u at interior points up to
    O(h^order): halving h divides the error by 4 (3-point rule) or 16
    (5-point rule). A wrong weight breaks the consistency altogether."""
    errs = []
    for n in (15, 31, 63):
        h = 1.0 / (n + 1)
        x = h * np.arange(1, n + 1)
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        u = (np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
             * np.sin(3 * np.pi * Z))
        uf = u.transpose(2, 1, 0).reshape(-1)       # x fastest
        Hu = (op.grid_hamiltonian((n, n, n), order, h) @ uf).reshape(n, n, n)
        Hu = Hu.transpose(2, 1, 0)
        want = 0.5 * np.pi ** 2 * 14.0 * u
        k = 2                                       # stay off the boundary
        errs.append(np.max(np.abs(Hu - want)[k:-k, k:-k, k:-k]))
    for a, b in zip(errs, errs[1:]):
        assert 0.85 * rate < a / b < 1.15 * rate


def test_dirichlet_eigenvalues_converge_to_the_continuum():
    """The lowest eigenvalues of -1/2 d^2/dx^2 on (0, 1) are (k pi)^2 / 2.
    The 3-point rule converges at second order; the 5-point rule, whose
    neighbours outside the grid are taken as zero (the Dirichlet wall),
    only at first order: that zero-ghost closure is first-order accurate at
    the wall."""
    exact = 0.5 * (np.pi * np.arange(1, 4)) ** 2
    for order, rate in ((2, 4.0), (4, 2.0)):
        errs = []
        for n in (31, 63, 127):
            h = 1.0 / (n + 1)
            T = op.axis_operator(n, order).toarray() * op.kinetic_scale(h)
            errs.append(np.abs(sla.eigvalsh(T)[:3] - exact))
        for a, b in zip(errs, errs[1:]):
            assert np.all((0.9 * rate < a / b) & (a / b < 1.1 * rate))


# ---------------------------------------------------------------------------
# Comparison helpers and the preconditioner, pinned to known values
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [1e-9, 1e-4, 0.3, 1.2])
def test_sin_max_angle_of_a_known_rotation(theta):
    """span{e1, e2} against span{e1, cos t e2 + sin t e3}: the principal
    angles are 0 and t, so the sine of the largest is sin t, for any basis of
    either span (here rotated and rescaled, not orthonormal)."""
    N = 40
    A = np.zeros((N, 2))
    A[0, 0] = A[1, 1] = 1.0
    B = np.zeros((N, 2))
    B[0, 0] = 1.0
    B[1, 1], B[2, 1] = math.cos(theta), math.sin(theta)
    rng = np.random.default_rng(1)
    Ma, Mb = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    for a, b in ((A, B), (A @ Ma, B @ Mb), (B @ Mb, A @ Ma)):
        assert abs(trm.sin_max_angle(a, b) - math.sin(theta)) <= 1e-15 + 1e-12 * theta


def test_sin_max_angle_two_angles_takes_the_largest():
    """Two rotated directions at angles 0.1 and 0.5: the 2-norm of the
    projection residual is sin 0.5 (a Frobenius norm would give
    sqrt(sin^2 0.1 + sin^2 0.5))."""
    N = 30
    A = np.zeros((N, 2))
    A[0, 0] = A[1, 1] = 1.0
    B = np.zeros((N, 2))
    B[0, 0], B[2, 0] = math.cos(0.1), math.sin(0.1)
    B[1, 1], B[3, 1] = math.cos(0.5), math.sin(0.5)
    assert abs(trm.sin_max_angle(A, B) - math.sin(0.5)) < 1e-15


def test_diagonal_preconditioner_inverts_a_diagonal_operator():
    """For a diagonal H (a potential with no kinetic coupling) the diagonal
    preconditioner is the exact inverse of H - sigma I with
    sigma = min_k H_kk - 1 (and of H - sigma S for a diagonal S, sigma =
    min_k H_kk / S_kk - 1): M (H - sigma S) y = y for every y, and M is SPD
    with entries at most 1."""
    rng = np.random.default_rng(4)
    d = rng.uniform(-3.0, 2.0, 50)
    H = sp.diags(d).tocsr()
    M = trm.diagonal_preconditioner(H)
    sigma = d.min() - 1.0
    y = rng.standard_normal(50)
    assert np.allclose(M * (spsolve_diag(H, sigma) @ y), y, rtol=1e-14, atol=0)
    assert np.all(M > 0) and np.max(M) <= 1.0 + 1e-15
    s = rng.uniform(0.5, 2.0, 50)
    S = sp.diags(s).tocsr()
    Ms = trm.diagonal_preconditioner(H, S)
    sig = np.min(d / s) - 1.0
    assert np.allclose(Ms * ((d - sig * s) * y), y, rtol=1e-14, atol=0)
    assert np.all(Ms > 0)


def spsolve_diag(H, sigma):
    """H - sigma I as a dense matrix (helper of the preconditioner pin)."""
    return H.toarray() - sigma * np.eye(H.shape[0])


# ---------------------------------------------------------------------------
# The large-workload reference eigensolver (oracle.filtered)
# ---------------------------------------------------------------------------
def test_filtered_eigenpairs_vs_dense_with_wells():
    """Brute force: the 20 lowest eigenvalues of an 8^3 13-point grid with
    wells equal dense diagonalisation; the residuals are what is returned."""
    shape = (8, 8, 8)
    H = op.grid_hamiltonian(shape, 4, 1.0, ti.gaussian_wells(shape, 6, seed=3))
    ref = op.dense_spectrum(H)[:20]
    r = filtered.lowest_eigenpairs(H, 20, tol=1e-11, want_vectors=True,
                                   max_iter=60)
    assert r.converged
    assert np.max(np.abs(r.lam - ref)) < 1e-12
    res = np.linalg.norm(H @ r.X - r.X * r.lam[None, :], axis=0)
    assert np.max(np.abs(res - r.residuals)) < 1e-12
    assert np.max(np.abs(r.X.T @ r.X - np.eye(20))) < 1e-12


def test_filtered_eigenpairs_vs_closed_forms():
    """V = 0: the 7-point 16^3 spectrum (cosine closed form, m = 17 at a
    cluster edge, E_G = 2.972191256741) and the 13-point 20^3 spectrum
    (Kronecker sum of the dense 1-D spectra), at the first 40 or so."""
    H = op.grid_hamiltonian((16, 16, 16), 2, 1.0, None)
    r = filtered.lowest_eigenpairs(H, 17, tol=1e-10)
    spec = op.order2_spectrum((16, 16, 16), 1.0)
    assert np.max(np.abs(r.lam - spec[:17])) < 1e-12
    assert abs(math.fsum(r.lam) - 2.972191256741) < 5e-12
    shape = (20, 20, 20)
    spec = op.kron_sum_spectrum(shape, 4, 1.0)
    edges = np.nonzero(np.diff(spec[:80]) > 1e-8)[0] + 1
    k = int(edges[edges <= 60][-1])
    r = filtered.lowest_eigenpairs(op.grid_hamiltonian(shape, 4, 1.0, None),
                                   k, tol=1e-10)
    assert k >= 30 and np.max(np.abs(r.lam - spec[:k])) < 1e-12


def test_gershgorin_upper_bounds_the_spectrum():
    shape = (6, 7, 5)
    H = op.grid_hamiltonian(shape, 4, 1.0, ti.gaussian_wells(shape, 4, seed=1))
    top = op.dense_spectrum(H)[-1]
    ub = filtered.gershgorin_upper(H)
    assert top <= ub
    # interior rows of the 13-point rule: 3.75 + 6 (2/3) + 6 (1/24) = 8 + V_i
    assert abs(ub - 8.0) < 1e-12 + np.max(np.abs(H.diagonal() - 3.75))
