"""Grid Hamiltonians, the test matrix of Sec. 3 and their exact spectra (FP64).

The sparse symmetric H of Sec. 2.1 (Eq. BASICEQ, O(N) nonzeros) is built here as
a Kronecker sum of one-dimensional Dirichlet difference operators plus a
diagonal potential:

    H = t * (T_x (+) T_y (+) T_z) + diag(V),   t = 1 / (2 h^2),

so that t*T_d is -1/2 d^2/dx_d^2 on a grid of spacing h. T_d is the 3-point rule
tridiag(-1, 2, -1) (order 2) or the 5-point rule (1, -16, 30, -16, 1)/12
(order 4), with neighbours outside the grid dropped. Grid points are ordered
x fastest: idx = x + nx*(y + ny*z). An axis of length 1 is absent, so the 2-D
matrix H_N of Eq. LAPLACE is order 2, nz = 1, t = 1 (diagonal 4, neighbours -1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp

# One-dimensional -d^2/dx^2 * h^2 weights for offsets 0, 1, 2.
_WEIGHTS = {2: (2.0, -1.0), 4: (2.5, -4.0 / 3.0, 1.0 / 12.0)}


def axis_operator(n: int, order: int) -> sp.csr_matrix:
    """T: the n x n one-dimensional Dirichlet difference matrix of the given order."""
    w = _WEIGHTS[order]
    offsets, bands = [], []
    for s, ws in enumerate(w):
        if s >= n:
            break
        offsets.append(s)
        bands.append(np.full(n - s, ws))
        if s:
            offsets.append(-s)
            bands.append(np.full(n - s, ws))
    return sp.diags(bands, offsets, shape=(n, n), format="csr")


def kinetic_scale(h: float) -> float:
    """t = 1/(2 h^2): the factor that turns T into -1/2 d^2/dx^2."""
    return 0.5 / (h * h)


def grid_hamiltonian(shape, order: int, h: float, V=None) -> sp.csr_matrix:
    """H = t (T_x (+) T_y (+) T_z) + diag(V) as a CSR matrix (Sec. 2.1; Eq. LAPLACE).

    The Kronecker sum puts x on the fastest index: the term for axis d is
    I_z (x) I_y (x) T_x, I_z (x) T_y (x) I_x and T_z (x) I_y (x) I_x.
    """
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    dims = [nx, ny, nz]
    N = nx * ny * nz
    t = kinetic_scale(h)
    H = sp.csr_matrix((N, N))
    for d in range(3):
        if dims[d] == 1:
            continue
        factors = []
        for e in (2, 1, 0):            # z, y, x from slowest to fastest
            factors.append(axis_operator(dims[e], order) if e == d
                           else sp.identity(dims[e], format="csr"))
        term = sp.kron(factors[0], sp.kron(factors[1], factors[2]),
                       format="csr")
        H = H + t * term
    if V is not None:
        H = H + sp.diags(np.asarray(V, dtype=np.float64).reshape(-1))
    H = H.tocsr()
    H.sort_indices()
    return H


def apply_h(H, C: np.ndarray) -> np.ndarray:
    """X = H C (Fig. EGFIG, step (1)), as a sparse-times-dense product."""
    return np.asarray(H @ C)


def laplace2d(n: int) -> sp.csr_matrix:
    """H_N of Eq. LAPLACE written out block by block: D_n on the diagonal
    (tridiag(-1, 4, -1)) and -I_n on the first block off-diagonals."""
    Dn = sp.diags([np.full(n, 4.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)],
                  [0, 1, -1], shape=(n, n))
    off = sp.diags([np.ones(n - 1), np.ones(n - 1)], [1, -1], shape=(n, n))
    H = sp.kron(sp.identity(n), Dn) - sp.kron(off, sp.identity(n))
    H = H.tocsr()
    H.sort_indices()
    return H


def laplace2d_spectrum(n: int) -> np.ndarray:
    """All eigenvalues of Eq. LAPLACE from the closed form printed after it:
    lambda_{p,q} = 4 (sin^2(p pi / 2(n+1)) + sin^2(q pi / 2(n+1))), ascending."""
    k = np.arange(1, n + 1)
    s = np.sin(k * np.pi / (2.0 * (n + 1))) ** 2
    lam = 4.0 * (s[:, None] + s[None, :])
    return np.sort(lam.reshape(-1))


def order2_spectrum(shape, h: float) -> np.ndarray:
    """Exact eigenvalues of the order-2 (7-point in 3-D) grid operator with V = 0:
    lambda = t * sum_d (2 - 2 cos(k_d pi / (n_d + 1))), k_d = 1..n_d, ascending."""
    dims = [n for n in (tuple(shape) + (1, 1))[:3] if n > 1]
    t = kinetic_scale(h)
    lam = np.zeros(1)
    for n in dims:
        k = np.arange(1, n + 1)
        mu = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
        lam = (lam[:, None] + mu[None, :]).reshape(-1)
    return np.sort(t * lam)


def kron_sum_spectrum(shape, order: int, h: float) -> np.ndarray:
    """Exact eigenvalues of t (T_x (+) T_y (+) T_z) with V = 0 for any order:
    the sums mu_a + mu_b + mu_c of the 1-D eigenvalues (dense, FP64), ascending.
    Zero-ghost Dirichlet breaks the sine basis of the 5-point rule, so the 1-D
    spectra are computed densely; the Kronecker sum identity is exact."""
    dims = [n for n in (tuple(shape) + (1, 1))[:3] if n > 1]
    t = kinetic_scale(h)
    lam = np.zeros(1)
    for n in dims:
        mu = scipy.linalg.eigvalsh(axis_operator(n, order).toarray())
        lam = (lam[:, None] + mu[None, :]).reshape(-1)
    return np.sort(t * lam)


def dense_spectrum(H) -> np.ndarray:
    """Brute force: all eigenvalues of H by dense symmetric diagonalisation."""
    A = H.toarray() if sp.issparse(H) else np.asarray(H)
    return scipy.linalg.eigvalsh(A)


def lowest_eigenvalues(H, k: int) -> np.ndarray:
    """The k lowest eigenvalues of a sparse H by Lanczos (ARPACK), ascending.
    Used only to screen seeds by the spectral gap of Sec. 2.1 at sizes where the
    dense route is too slow; the trace-minimization oracle does not use it."""
    import scipy.sparse.linalg as sla
    if H.shape[0] <= 3000:
        return dense_spectrum(H)[:k]
    vals = sla.eigsh(H, k=k, which="SA", tol=0, maxiter=200000,
                     ncv=min(H.shape[0], max(2 * k + 1, k + 64)),
                     return_eigenvectors=False)
    return np.sort(vals)
