"""Trace minimization by nonlinear conjugate gradients, plain FP64 numpy.

Follows Sec. 2.1 of Tsuchida and Choe step by step. Library primitives (matrix
products, a Cholesky factorisation, triangular solves, a symmetric-definite
eigensolver) serve as single steps; nothing is blocked, fused or reordered.

Notation as in the paper: H (N x N, sparse, symmetric), C, G, P (N x m),
E(C) = trace(C^T H C) with C^T C = I_m (Eqs. TRHEQ, CIJEQ).

Readings where the paper is silent or ambiguous (each also listed in the design
notes of the repository):

* Fig. ONFIG step (4) prints C_out = C_in L^{-1}; with L lower triangular only
  C_in L^{-T} is orthonormal, so that is what :func:`orthonormalize` computes.
* The line minimization along P_i (Sec. 2.1, refs. RCP and KV) is not
  specified. The energy after orthonormalization is exact from m x m data,
  E(alpha) = trace(S(alpha)^{-1} A(alpha)), S and A the projections of
  C + alpha P; :func:`line_minimize` finds the first root of dE/dalpha by a
  bracketed regula falsi. This only changes the path, never the converged
  result.
* Convergence ("||G|| sufficiently small"): stop when the RMS column residual
  r = ||G||_F / (2 sqrt(m)) = ||H C - C H_C||_F / sqrt(m) is <= tol.
* Diagonal preconditioner (Eq. PCEQ, Sec. 4): M = diag(1 / (H_jj - sigma)) with
  sigma = min_k H_kk - 1, so M is SPD. The Polak-Ribiere gamma generalises to
  trace((G_i - G_{i-1})^T M G_i) / trace(G_{i-1}^T M G_{i-1}) (exactly the
  printed formula when M = I). CG restarts (gamma = 0) when P_i is not a
  descent direction, trace(G_i^T P_i) <= 0.
* Initial-guess extrapolation (cited in Secs. 3 and 4, ref. APJ, not
  defined in the paper): :func:`extrapolate` aligns the previous block
  to the current one by the orthogonal Procrustes rotation (the blocks are
  only defined up to a rotation, Eq. TRHEQ's invariance), extrapolates
  linearly, and orthonormalizes by Fig. ONFIG.
* Generalized problem H e = lambda S e with S symmetric positive definite
  (Sec. 2.1 calls the extension straightforward and gives no formulas): the
  constraint becomes C^T S C = I, so the orthonormalization factors C^T S C,
  the gradient is G = -2 (H C - S C H_C), the line-search overlap is
  (C + aP)^T S (C + aP), the preconditioner is diag(1 / (H_jj - sigma S_jj))
  with sigma = min_k H_kk / S_kk - 1, and the Rayleigh-Ritz step solves
  (C^T H C) y = theta (C^T S C) y. Every function takes S = None (the
  identity) for the standard problem.
* The closing diagonalisation of H (Sec. 2.1, after "HC = CH") is a
  Rayleigh-Ritz step on span(C) solved as the generalised problem
  (C^T H C) y = theta (C^T C) y, so a residual loss of orthonormality in C
  cannot bias the eigenvalues.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .operator import apply_h



# ----------------------------------------------------------------------------
# Fig. ONFIG: orthonormalization by Cholesky factorisation
# ----------------------------------------------------------------------------
def _apply_s(S, C):
    """S C, or C when S is None (the standard problem)."""
    return C if S is None else apply_h(S, C)


def orthonormalize(C: np.ndarray, S=None) -> np.ndarray:
    """Fig. ONFIG. (1) S_C = C^T S C; (2) S_C = L L^T; (3) L^{-1};
    (4) C_out = C_in L^{-T} (S = None: C^T C)."""
    Sc = C.T @ _apply_s(S, C)                                # (1) DSYRK
    L = np.linalg.cholesky(Sc)                               # (2) DPOTRF
    Linv = sla.solve_triangular(L, np.eye(L.shape[0]), lower=True)  # (3) DTRTRI
    return C @ Linv.T                                        # (4) DTRMM


# ----------------------------------------------------------------------------
# Fig. EGFIG: energy and gradient
# ----------------------------------------------------------------------------
def energy_gradient_alg1(H, C, S=None):
    """Fig. EGFIG, Algorithm-1: X = HC; H = C^T X; E = tr H; G = -2 (X - C H)
    (generalized: G = -2 (X - S C H)).

    Returns (E, G, X, Hc)."""
    X = apply_h(H, C)                       # (1)
    Hc = C.T @ X                            # (2)
    E = float(np.trace(Hc))                 # (3)
    G = -2.0 * (X - _apply_s(S, C) @ Hc)    # (4)
    return E, G, X, Hc


def energy_gradient_alg2(H, C, zero_diag: bool = False, need_gradient=True,
                         S=None):
    """Fig. EGFIG, Algorithm-2, steps (1)-(7).

    (1) X = HC; (2) H_D = diag(C^T X); (3) E = tr H_D; (4) stop here if G is not
    needed; (5) X' = X - C H_D; (6) H' = C^T X'; (7) G = -2 (X' - C H').
    ``zero_diag`` sets diag(H') = 0 after step (6), as Sec. 2.2 advises for MP2.
    Returns (E, G, X, H_D, X', H'); G, X', H' are None when not needed."""
    X = apply_h(H, C)                                       # (1)
    HD = np.einsum("ij,ij->j", C, X)                        # (2)
    E = float(np.sum(HD))                                   # (3)
    if not need_gradient:                                   # (4)
        return E, None, X, HD, None, None
    SC = _apply_s(S, C)                     # generalized: S C for C below
    Xp = X - SC * HD[None, :]                               # (5)
    Hp = C.T @ Xp                                           # (6)
    if zero_diag:
        np.fill_diagonal(Hp, 0.0)
    G = -2.0 * (Xp - SC @ Hp)                               # (7)
    return E, G, X, HD, Xp, Hp


def rms_residual(G: np.ndarray) -> float:
    """r = ||G||_F / (2 sqrt(m)): the RMS column norm of H C - C H_C."""
    return float(np.linalg.norm(G) / (2.0 * math.sqrt(G.shape[1])))


# ----------------------------------------------------------------------------
# Polak-Ribiere (Sec. 2.1) and the preconditioner (Eq. PCEQ)
# ----------------------------------------------------------------------------
def diagonal_preconditioner(H, S=None) -> np.ndarray:
    """diag(M) = 1 / (H_jj - sigma), sigma = min_k H_kk - 1 (SPD, bounded);
    generalized: 1 / (H_jj - sigma S_jj), sigma = min_k H_kk / S_kk - 1."""
    d = np.asarray(H.diagonal(), dtype=np.float64)
    if S is None:
        sigma = d.min() - 1.0
        return 1.0 / (d - sigma)
    sd = np.asarray(S.diagonal(), dtype=np.float64)
    sigma = (d / sd).min() - 1.0
    return 1.0 / (d - sigma * sd)


def polak_ribiere(G, G_prev, MG, MG_prev) -> float:
    """gamma_i = tr((G_i - G_{i-1})^T M G_i) / tr(G_{i-1}^T M G_{i-1}); with M = I
    this is the printed Polak-Ribiere formula."""
    num = float(np.sum((G - G_prev) * MG))
    den = float(np.sum(G_prev * MG_prev))
    return num / den


# ----------------------------------------------------------------------------
# Line minimization along P (Fig. TMFIG, C_{i+1} = C_i + alpha_i P_i)
# ----------------------------------------------------------------------------
@dataclass
class LineMatrices:
    """m x m projections of the block pencil C + alpha P:
    S(alpha) = S0 + alpha (B + B^T) + alpha^2 Q   = (C + aP)^T S (C + aP)
    A(alpha) = A0 + alpha (K + K^T) + alpha^2 Ap  = (C + aP)^T H (C + aP)."""
    S0: np.ndarray
    B: np.ndarray
    Q: np.ndarray
    A0: np.ndarray
    K: np.ndarray
    Ap: np.ndarray


def line_matrices(C, P, X, HP, S=None) -> LineMatrices:
    """The Gram products C^T S C, C^T S P, P^T S P, C^T H C, C^T H P, P^T H P
    (S = None: the identity)."""
    SC, SP = _apply_s(S, C), _apply_s(S, P)
    return LineMatrices(S0=C.T @ SC, B=C.T @ SP, Q=P.T @ SP,
                        A0=C.T @ X, K=C.T @ HP, Ap=P.T @ HP)


def line_energy(alpha: float, M: LineMatrices) -> float:
    """E(alpha) = tr(S(alpha)^{-1} A(alpha)): the energy of orthonormalize(C + alpha P),
    since with C_out = (C + aP) L^{-T}, tr(C_out^T H C_out) = tr(L^{-1} A L^{-T})."""
    S = M.S0 + alpha * (M.B + M.B.T) + alpha * alpha * M.Q
    A = M.A0 + alpha * (M.K + M.K.T) + alpha * alpha * M.Ap
    S = 0.5 * (S + S.T)
    A = 0.5 * (A + A.T)
    try:
        cf = sla.cho_factor(S, lower=True)
    except np.linalg.LinAlgError:
        return math.inf
    return float(np.trace(sla.cho_solve(cf, A)))


def line_slope(alpha: float, M: LineMatrices) -> float:
    """dE/dalpha = tr(S^{-1} (A' - S' S^{-1} A)), S' = (B + B^T) + 2 alpha Q and
    A' = (K + K^T) + 2 alpha Ap. Near convergence E(alpha) - E(0) falls below the
    FP64 resolution of E itself, while this slope keeps its relative accuracy,
    so the minimum is located as the root of the slope."""
    S = M.S0 + alpha * (M.B + M.B.T) + alpha * alpha * M.Q
    A = M.A0 + alpha * (M.K + M.K.T) + alpha * alpha * M.Ap
    S1 = (M.B + M.B.T) + 2.0 * alpha * M.Q
    A1 = (M.K + M.K.T) + 2.0 * alpha * M.Ap
    S = 0.5 * (S + S.T)
    A = 0.5 * (A + A.T)
    cf = sla.cho_factor(S, lower=True)
    Y = sla.cho_solve(cf, A)
    return float(np.trace(sla.cho_solve(cf, A1 - S1 @ Y)))


def line_minimize(M: LineMatrices, alpha_guess: float, rtol: float = 1e-10):
    """alpha_i: the first minimum of E(alpha) along P for alpha > 0.

    E'(0) < 0 for a descent direction. The bracket [lo, hi] with E'(lo) < 0 <
    E'(hi) starts at alpha_guess and doubles; the root of E' inside it is then
    found by regula falsi with the Illinois modification (Dowell and Jarratt,
    1971) until |E'| <= rtol |E'(0)|. Returns (alpha, E'(0))."""
    g0 = line_slope(0.0, M)
    if not g0 < 0.0:
        return 0.0, g0
    lo, glo = 0.0, g0
    hi = float(alpha_guess)
    ghi = line_slope(hi, M)
    for _ in range(200):
        if ghi >= 0.0:
            break
        lo, glo = hi, ghi
        hi = 2.0 * hi
        ghi = line_slope(hi, M)
    else:
        return lo, g0
    side = 0
    c = lo
    for _ in range(200):
        c = (lo * ghi - hi * glo) / (ghi - glo)
        gc = line_slope(c, M)
        if abs(gc) <= rtol * abs(g0) or hi - lo <= 1e-15 * hi:
            break
        if gc < 0.0:
            lo, glo = c, gc
            if side == -1:
                ghi *= 0.5
            side = -1
        else:
            hi, ghi = c, gc
            if side == +1:
                glo *= 0.5
            side = +1
    return c, g0


# ----------------------------------------------------------------------------
# Closing diagonalisation of H (Sec. 2.1)
# ----------------------------------------------------------------------------
def rayleigh_ritz(H, C, S=None):
    """Diagonalise H = C^T H C on span(C): (C^T H C) y = theta (C^T S C) y.

    Returns (lambda ascending, C Y (S-orthonormal columns), column residual
    norms ||H c_j - lambda_j S c_j||). Each column's sign makes its
    largest-magnitude entry positive (presentation only)."""
    X = apply_h(H, C)
    SC = _apply_s(S, C)
    Hc = C.T @ X
    Hc = 0.5 * (Hc + Hc.T)
    Sc = C.T @ SC
    Sc = 0.5 * (Sc + Sc.T)
    lam, Y = sla.eigh(Hc, Sc)
    Cr = C @ Y
    Xr = X @ Y
    SCr = SC @ Y
    m = Cr.shape[1]
    piv = np.argmax(np.abs(Cr), axis=0)
    sgn = np.sign(Cr[piv, np.arange(m)])
    sgn[sgn == 0] = 1.0
    Cr *= sgn
    Xr *= sgn
    SCr *= sgn
    res = np.linalg.norm(Xr - SCr * lam[None, :], axis=0)
    return lam, Cr, res


def energy_sum(lam) -> float:
    """E_G = sum_j lambda_j (Eq. EGEQ), correctly rounded."""
    return math.fsum(float(x) for x in np.sort(lam))


# ----------------------------------------------------------------------------
# Fig. TMFIG: the trace-minimization loop
# ----------------------------------------------------------------------------
@dataclass
class Result:
    lam: np.ndarray
    E_G: float
    C: np.ndarray
    residuals: np.ndarray
    iterations: int
    converged: bool
    energies: list = field(default_factory=list)
    rms: list = field(default_factory=list)
    alphas: list = field(default_factory=list)


def solve(H, C0: np.ndarray, tol: float = 1e-10, max_iter: int = 20000,
          precond: bool = False, algorithm: int = 1, zero_diag: bool = False,
          cg: bool = True, callback=None, S=None) -> Result:
    """Fig. TMFIG. C_0 = orthonormalize(random guess); for i = 0, 1, ...:
    E_i, G_i (Fig. EGFIG); convergence check; P_i = G'_i + gamma_i P_{i-1} with
    G' = M G (Eq. PCEQ); C_{i+1} = C_i + alpha_i P_i; orthonormalize (Fig. ONFIG).
    Ends with the diagonalisation of H on span(C). ``cg=False`` keeps
    gamma_i = 0 (steepest descent), used only to show what the CG term buys.
    ``S``: the overlap of the generalized problem H e = lambda S e (None for
    the standard one)."""
    C = orthonormalize(np.array(C0, dtype=np.float64), S)
    m = C.shape[1]
    Mdiag = diagonal_preconditioner(H, S) if precond else None
    G_prev = MG_prev = P_prev = None
    alpha = None
    energies, rms, alphas = [], [], []
    converged = False
    it = 0
    for it in range(max_iter + 1):
        if algorithm == 1:
            E, G, X, _ = energy_gradient_alg1(H, C, S)
        else:
            E, G, X, _, _, _ = energy_gradient_alg2(H, C, zero_diag, S=S)
        r = rms_residual(G)
        energies.append(E)
        rms.append(r)
        if callback is not None:
            callback(it, E, r)
        if r <= tol:
            converged = True
            break
        if it == max_iter:
            break
        MG = G * Mdiag[:, None] if Mdiag is not None else G
        gamma = (0.0 if G_prev is None or not cg
                 else polak_ribiere(G, G_prev, MG, MG_prev))
        P = MG + gamma * P_prev if gamma != 0.0 else MG.copy()
        if float(np.sum(G * P)) <= 0.0:          # not a descent direction
            P = MG.copy()
        HP = apply_h(H, P)
        LM = line_matrices(C, P, X, HP, S)
        if alpha is None or alpha <= 0.0:
            alpha = 0.1 * math.sqrt(m) / max(np.linalg.norm(P), 1e-300)
        alpha, _ = line_minimize(LM, alpha)
        alphas.append(alpha)
        C = orthonormalize(C + alpha * P, S)
        G_prev, MG_prev, P_prev = G, MG, P
    lam, Cr, res = rayleigh_ritz(H, C, S)
    return Result(lam=lam, E_G=energy_sum(lam), C=Cr, residuals=res,
                  iterations=it, converged=converged, energies=energies,
                  rms=rms, alphas=alphas)


# ----------------------------------------------------------------------------
# Initial guess for the next of a chain of related problems
# ----------------------------------------------------------------------------
def procrustes(C_prev: np.ndarray, C_cur: np.ndarray) -> np.ndarray:
    """The orthogonal U minimising ||C_prev U - C_cur||_F: with the SVD
    C_prev^T C_cur = W diag(s) V^T, U = W V^T (orthogonal Procrustes)."""
    W, _, Vt = np.linalg.svd(C_prev.T @ C_cur)
    return W @ Vt


def extrapolate(C_prev: np.ndarray, C_cur: np.ndarray,
                alpha: float = 1.0) -> np.ndarray:
    """Block for the next problem of a chain from the converged blocks of the
    two before: C_prev rotated onto C_cur's basis (:func:`procrustes`), then
    C_cur + alpha (C_cur - C_prev U), orthonormalized (Fig. ONFIG). alpha = 1
    extrapolates linearly over equal steps."""
    U = procrustes(C_prev, C_cur)
    return orthonormalize(C_cur + alpha * (C_cur - C_prev @ U))


# ----------------------------------------------------------------------------
# Comparisons used by the tests
# ----------------------------------------------------------------------------
def sin_max_angle(A: np.ndarray, B: np.ndarray) -> float:
    """sin of the largest principal angle between span(A) and span(B):
    ||B - A (A^T B)||_2 after orthonormalising both (no arccos near 1)."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


def ritz_check(H, C):
    """A-posteriori FP64 check of any block C: Ritz values on span(C) and the
    residual norm of each Ritz pair (Sec. 2.1, HC = CH at convergence)."""
    lam, Cr, res = rayleigh_ritz(H, C)
    return lam, res
