"""Reference eigenpairs of large sparse H by Chebyshev-filtered subspace
iteration, plain FP64 (test infrastructure: only the tests and the scripts
that write stored expected values use it).

The trace-minimization oracle of :mod:`oracle.trm` is too slow at
N ~ 1e6, m ~ 1e3 (each of its ~1e3 iterations is ~1e13 flops), and ARPACK's
Lanczos needs a Krylov basis twice the wanted count, reorthogonalised by
matrix-vector sweeps over it. This module is an independent route to the
same numbers (the m lowest eigenvalues, their sum E_G of Eq. EGEQ and the gap
to lambda_{m+1} that Sec. 2.1 assumes), used to screen seeds by the gap rule
and to give the large workloads a reference E_G that does not come from the
trace minimization at all.

The method is the textbook one (Y. Zhou and Y. Saad, "A Chebyshev-Davidson
algorithm for large symmetric eigenproblems" / "Chebyshev-filtered subspace
iteration", 2007), in this order on a block X of b > k columns:

1. Rayleigh-Ritz on span(X): A = X^T H X, A = Q diag(theta) Q^T
   (ascending), X <- X Q, HX <- (H X) Q; residuals r_j = ||H x_j - theta_j x_j||.
2. Stop when max_{j < k} r_j <= tol.
3. Filter: with [a, b] = [theta_max of the block, an upper bound of the
   spectrum] mapped to [-1, 1] by t = (H - c) / e, c = (a + b) / 2,
   e = (b - a) / 2, replace X by T_d(t) X through the three-term recurrence
   Y_0 = X, Y_1 = t X, Y_{j+1} = 2 t Y_j - Y_{j-1}. T_d is bounded by 1 on
   [a, b] and grows fast below a, so the wanted (lowest) components are
   amplified relative to the rest.
4. Orthonormalize X (Cholesky, as in Fig. ONFIG, applied twice) and go to 1.

H X is formed by row blocks in threads: each row's sum is the one the plain
product forms, so the result is the same numbers; the blocks only spread the
work over the host's cores. The upper bound b is Gershgorin's,
max_i (H_ii + sum_{j != i} |H_ij|).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def gershgorin_upper(H) -> float:
    """max_i (H_ii + sum_{j != i} |H_ij|): no eigenvalue of H exceeds it."""
    H = sp.csr_matrix(H)
    d = H.diagonal()
    off = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)
    return float(np.max(d + off))


class RowBlockProduct:
    """Y = H X for a CSR H and a C-ordered N x b block X, by row blocks of H
    on a thread pool (the sparse kernel releases the interpreter lock)."""

    def __init__(self, H, threads: int | None = None):
        self.H = sp.csr_matrix(H)
        self.H.sort_indices()
        n = self.H.shape[0]
        self.threads = threads or min(8, os.cpu_count() or 1)
        cuts = np.linspace(0, n, 4 * self.threads + 1).astype(np.int64)
        self.rows = [(int(cuts[i]), int(cuts[i + 1]))
                     for i in range(len(cuts) - 1) if cuts[i + 1] > cuts[i]]
        self.parts = [self.H[lo:hi] for lo, hi in self.rows]
        self.pool = cf.ThreadPoolExecutor(self.threads)

    def __call__(self, X, out=None, combine=None):
        """out[rows] = H[rows] X, or combine(rows_slice, H[rows] X) when given
        (an in-place update that needs no second N x b array)."""
        X = np.ascontiguousarray(X)
        if out is None and combine is None:
            out = np.empty((self.H.shape[0], X.shape[1]))

        def one(i):
            lo, hi = self.rows[i]
            y = self.parts[i] @ X
            if combine is not None:
                combine(slice(lo, hi), y)
            else:
                out[lo:hi] = y

        list(self.pool.map(one, range(len(self.rows))))
        return out

    def close(self):
        self.pool.shutdown()


def _orthonormalize_rows(X, apply_rows):
    """X <- X L^{-T} with X^T X = L L^T (Fig. ONFIG), in place by row blocks."""
    S = X.T @ X
    L = np.linalg.cholesky(S)
    Rinv = sla.solve_triangular(L, np.eye(L.shape[0]), lower=True).T
    apply_rows(X, Rinv)


def filter_interval(theta, upper: float):
    """Centre c and half-width e of the damped interval [theta_max, upper]
    (theta: the block's Ritz values, ascending)."""
    a = float(theta[-1])
    return 0.5 * (a + upper), 0.5 * (upper - a)


@dataclass
class Eigenpairs:
    lam: np.ndarray        # the k lowest eigenvalues, ascending
    residuals: np.ndarray  # ||H x_j - lam_j x_j|| of the returned pairs
    X: np.ndarray | None   # N x k eigenvectors (C order), or None
    iterations: int
    converged: bool


def lowest_eigenpairs(H, k: int, block: int | None = None, degree: int = 16,
                      tol: float = 1e-9, max_iter: int = 200, seed: int = 0,
                      want_vectors: bool = False, threads: int | None = None,
                      callback=None) -> Eigenpairs:
    """The k lowest eigenpairs of the sparse symmetric H (steps 1-4 of the
    module docstring). block: columns iterated (default k + max(24, k // 8));
    tol: the largest residual norm accepted among the first k pairs."""
    N = H.shape[0]
    b = min(N, block or (k + max(24, k // 8)))
    if not 1 <= k <= b <= N:
        raise ValueError("need 1 <= k <= block <= N")
    prod = RowBlockProduct(H, threads)
    rows = prod.rows
    pool = prod.pool

    def apply_rows(X, M):
        # X[rows] <- X[rows] M for every row block (in place)
        def one(r):
            lo, hi = r
            X[lo:hi] = X[lo:hi] @ M
        list(pool.map(one, rows))

    upper = gershgorin_upper(H)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, b))
    for _ in range(2):
        _orthonormalize_rows(X, apply_rows)
    it = 0
    converged = False
    theta = res = None
    try:
        for it in range(max_iter + 1):
            # 1. Rayleigh-Ritz
            HX = prod(X)
            A = X.T @ HX
            A = 0.5 * (A + A.T)
            theta, Q = np.linalg.eigh(A)
            apply_rows(X, Q)
            apply_rows(HX, Q)
            R2 = np.zeros(b)

            def resid(r):
                lo, hi = r
                D = HX[lo:hi] - X[lo:hi] * theta[None, :]
                return np.einsum("ij,ij->j", D, D)

            for part in pool.map(resid, rows):
                R2 += part
            res = np.sqrt(R2)
            del HX
            if callback is not None:
                callback(it, theta[:k], res[:k])
            # 2. convergence
            if np.max(res[:k]) <= tol:
                converged = True
                break
            if it == max_iter:
                break
            # 3. Chebyshev filter on [theta_max, upper]
            c, e = filter_interval(theta, upper)
            Yp = X                          # Y_0
            Y = prod(X)                     # Y_1 = (H X - c X) / e
            Y -= c * X
            Y /= e
            for _ in range(2, degree + 1):
                # Y_{j+1} = 2 (H Y_j - c Y_j) / e - Y_{j-1}, written over Y_{j-1}
                Ycur = Y

                def comb(sl, HY, Yp=Yp, Ycur=Ycur):
                    Yp[sl] = (2.0 / e) * (HY - c * Ycur[sl]) - Yp[sl]

                prod(Ycur, combine=comb)
                Y, Yp = Yp, Ycur
            X = Y
            del Yp
            # 4. orthonormalize (twice: the filtered block is ill-conditioned)
            for _ in range(2):
                _orthonormalize_rows(X, apply_rows)
    finally:
        prod.close()
    return Eigenpairs(lam=np.array(theta[:k]), residuals=np.array(res[:k]),
                      X=np.ascontiguousarray(X[:, :k]) if want_vectors else None,
                      iterations=it, converged=converged)
