"""Plain FP64 CPU oracle of the trace-minimization eigensolver (test infrastructure).

This package is the checker, not the product. Only the test suite, the smoke
check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import
it. The CUDA library never calls into it and shares no code with it: the two
meet only through the seeded inputs of :mod:`trm_inputs`.

Contents (each function cites the passage of Tsuchida and Choe, "Iterative
diagonalization of symmetric matrices in mixed precision", that it follows):

* :mod:`oracle.operator` - the grid Hamiltonians as Kronecker sums, the test
  matrix of Sec. 3 (Eq. LAPLACE), closed-form spectra and brute-force dense
  diagonalisation.
* :mod:`oracle.trm` - Fig. TMFIG (nonlinear CG trace minimization), Fig. EGFIG
  (energy and gradient, Algorithm-1 and Algorithm-2), Fig. ONFIG (Cholesky
  orthonormalization), the Polak-Ribiere gamma, the preconditioned gradient of
  Eq. PCEQ, the line minimization along P and the closing diagonalisation of H.

Every function is pinned by a CPU test against something other than itself
(closed forms, values printed in Table RESTBL, brute-force dense eigenvalues,
invariants); none is "parity unpinned".
"""
from . import operator, trm  # noqa: F401
