"""The oracle's pins catch plausible mistakes: each case plants one error in
an oracle function (on the CPU, through monkeypatch) and checks that a pin
of tests/test_oracle.py then fails. A pin that kept passing would not be
pinning that part of the oracle."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import operator as op
from oracle import trm

from . import test_oracle as pins


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_printed_onfig_product_is_caught(monkeypatch):
    """C L^{-1} (the product as printed) instead of C L^{-T}."""
    def bad(C, S=None):
        Sc = C.T @ (C if S is None else S @ C)
        L = np.linalg.cholesky(Sc)
        return C @ sla.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    monkeypatch.setattr(trm, "orthonormalize", bad)
    _fails(pins.test_orthonormalize_is_orthonormal_and_keeps_span)


@pytest.mark.parametrize("mistake", ["factor", "sign"])
def test_gradient_mistakes_are_caught(monkeypatch, mistake):
    """G = -(X - C H_C) (a lost factor 2) or +2 (X - C H_C) (a sign)."""
    orig = trm.energy_gradient_alg1

    def bad(H, C, S=None):
        E, G, X, Hc = orig(H, C, S)
        return E, (0.5 * G if mistake == "factor" else -G), X, Hc
    monkeypatch.setattr(trm, "energy_gradient_alg1", bad)
    _fails(pins.test_gradient_is_minus_directional_derivative)


def test_generalized_gradient_without_S_is_caught(monkeypatch):
    """G = -2 (H C - C H_C) in the generalized problem (S dropped)."""
    orig = trm.energy_gradient_alg1

    def bad(H, C, S=None):
        return orig(H, C, None)
    monkeypatch.setattr(trm, "energy_gradient_alg1", bad)
    _fails(pins.test_generalized_gradient_is_minus_constrained_derivative)


def test_dropped_line_slope_term_is_caught(monkeypatch):
    """dE/dalpha without the S' S^{-1} A term."""
    def bad(alpha, M):
        S = M.S0 + alpha * (M.B + M.B.T) + alpha * alpha * M.Q
        A1 = (M.K + M.K.T) + 2.0 * alpha * M.Ap
        cf = sla.cho_factor(0.5 * (S + S.T), lower=True)
        return float(np.trace(sla.cho_solve(cf, A1)))
    monkeypatch.setattr(trm, "line_slope", bad)
    _fails(pins.test_line_slope_matches_finite_difference_and_gradient)


def test_transposed_procrustes_rotation_is_caught(monkeypatch):
    """U^T in place of U: the alignment rotates the wrong way."""
    orig = trm.procrustes
    monkeypatch.setattr(trm, "procrustes", lambda A, B: orig(A, B).T)
    _fails(pins.test_procrustes_recovers_a_rotation_and_minimises)
    _fails(pins.test_extrapolate_is_second_order_along_a_smooth_path)


def test_extrapolation_without_alignment_is_caught(monkeypatch):
    """C_cur + (C_cur - C_prev): raw blocks, no rotation onto C_cur."""
    monkeypatch.setattr(trm, "procrustes",
                        lambda A, B: np.eye(A.shape[1]))
    _fails(pins.test_extrapolate_is_second_order_along_a_smooth_path)


def test_kinetic_scale_mistake_is_caught(monkeypatch):
    """t = 1/h^2 instead of 1/(2 h^2) (the -1/2 of -1/2 nabla^2 lost)."""
    monkeypatch.setattr(op, "kinetic_scale", lambda h: 1.0 / (h * h))
    _fails(pins.test_laplace_block_form_equals_kronecker_form)


def test_generalized_rayleigh_ritz_without_S_is_caught(monkeypatch):
    """The closing Rayleigh-Ritz with C^T C in place of C^T S C."""
    orig = trm.rayleigh_ritz
    monkeypatch.setattr(trm, "rayleigh_ritz",
                        lambda H, C, S=None: orig(H, C, None))
    _fails(pins.test_generalized_solve_vs_dense_and_closed_form, False)


def test_wrong_fourth_order_weight_is_caught(monkeypatch):
    """The 5-point rule with 1/6 in place of 1/12 for the second neighbour."""
    w = dict(op._WEIGHTS)
    w[4] = (2.5, -4.0 / 3.0, 1.0 / 6.0)
    monkeypatch.setattr(op, "_WEIGHTS", w)
    _fails(pins.test_stencil_truncation_error_has_the_rule_order, 4, 16.0)


def test_fletcher_reeves_in_place_of_polak_ribiere_is_caught(monkeypatch):
    """gamma = tr(G^T M G) / tr(G_prev^T M G_prev) (no G_prev subtracted)."""
    monkeypatch.setattr(trm, "polak_ribiere",
                        lambda G, Gp, MG, MGp: float(np.sum(G * MG))
                        / float(np.sum(Gp * MGp)))
    _fails(pins.test_polak_ribiere_restarts_itself_when_the_gradient_repeats)



def test_frobenius_angle_is_caught(monkeypatch):
    """sin_max_angle with the Frobenius norm in place of the 2-norm."""
    def bad(A, B):
        Qa, _ = np.linalg.qr(A)
        Qb, _ = np.linalg.qr(B)
        return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb)))
    monkeypatch.setattr(trm, "sin_max_angle", bad)
    _fails(pins.test_sin_max_angle_two_angles_takes_the_largest)


def test_angle_without_orthonormalising_is_caught(monkeypatch):
    """sin_max_angle on the raw bases (no QR)."""
    monkeypatch.setattr(trm, "sin_max_angle", lambda A, B: float(
        np.linalg.norm(B - A @ (A.T @ B), 2)))
    _fails(pins.test_sin_max_angle_of_a_known_rotation, 0.3)


def test_preconditioner_shift_sign_is_caught(monkeypatch):
    """sigma = min_k H_kk + 1: H - sigma I is no longer positive definite."""
    def bad(H, S=None):
        d = H.diagonal()
        return 1.0 / (d - (d.min() + 1.0))
    monkeypatch.setattr(trm, "diagonal_preconditioner", bad)
    _fails(pins.test_diagonal_preconditioner_inverts_a_diagonal_operator)


def test_filtered_without_orthonormalization_is_caught(monkeypatch):
    """Rayleigh-Ritz on a basis that was never orthonormalized."""
    from oracle import filtered
    monkeypatch.setattr(filtered, "_orthonormalize_rows", lambda X, f: None)
    _fails(pins.test_filtered_eigenpairs_vs_dense_with_wells)


def test_filtered_damping_the_wanted_end_is_caught(monkeypatch):
    """The damped interval starting at the lowest Ritz value (theta[0] for
    theta[-1]): the wanted eigenvalues are no longer amplified."""
    from oracle import filtered
    monkeypatch.setattr(filtered, "filter_interval", lambda th, up: (
        0.5 * (th[0] + up), 0.5 * (up - th[0])))
    _fails(pins.test_filtered_eigenpairs_vs_dense_with_wells)
