"""CPU checks of the seeded input generators (no GPU, no method arithmetic)."""
import json
import os

import numpy as np

import trm_inputs as ti
from oracle import operator as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_first_output():
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    assert int(ti.splitmix64(np.uint64(0))) == int(ref["state0_first_output"], 16)


def test_splitmix64_matches_python_integer_arithmetic():
    mask = (1 << 64) - 1

    def mix(x):
        z = (x + 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    xs = np.array([0, 1, 2, 12345, 2**63 + 7, 2**64 - 1], dtype=np.uint64)
    got = ti.splitmix64(xs)
    for x, g in zip(xs, got):
        assert int(g) == mix(int(x))


def test_random_block_layout_and_range():
    C = ti.random_block(1000, 7, seed=3)
    assert C.shape == (1000, 7) and C.flags["F_CONTIGUOUS"]
    assert C.min() >= -0.5 and C.max() < 0.5
    # entry (i, j) uses counter i + N j
    i, j = 123, 5
    assert C[i, j] == ti.uniform01(3, np.uint64(i + 1000 * j)) - 0.5
    # roughly uniform: mean ~ 0, variance ~ 1/12
    assert abs(C.mean()) < 0.02
    assert abs(C.var() - 1.0 / 12.0) < 0.005
    assert not np.array_equal(C, ti.random_block(1000, 7, seed=4))


def test_gaussian_wells_deterministic_and_bounded():
    V1 = ti.gaussian_wells((10, 9, 8), 5, seed=11)
    V2 = ti.gaussian_wells((10, 9, 8), 5, seed=11)
    assert np.array_equal(V1, V2)
    assert V1.shape == (720,)
    assert V1.max() <= 0.0 and V1.min() >= -2.0 * 5
    # a single well at its centre reaches its depth when the centre is on a node
    V = ti.gaussian_wells((1, 1, 1), 1, seed=2)
    assert -2.0 <= V[0] <= -0.5


def test_grid_csr_equals_kronecker_operator():
    """The CSR builder and the oracle's Kronecker sum are written independently;
    indices must agree bit for bit, values to rounding."""
    for shape, order in [((7, 6, 5), 2), ((7, 6, 5), 4), ((9, 8, 1), 2),
                         ((5, 5, 5), 4), ((3, 4, 2), 4)]:
        V = ti.gaussian_wells(shape, 3, seed=1)
        rp, cols, vals = ti.grid_csr(shape, order, 1.0, V)
        H = op.grid_hamiltonian(shape, order, 1.0, V)
        assert np.array_equal(rp, H.indptr)
        assert np.array_equal(cols, H.indices)
        assert np.allclose(vals, H.data, rtol=4e-16, atol=4e-16)


def test_grid_csr_13_point_coefficients():
    """-1/2 nabla^2 with the 5-point 4th-order rule per axis at h = 1:
    diagonal 3.75 + V, first neighbours -2/3, second neighbours 1/24."""
    shape = (6, 6, 6)
    V = np.zeros(216)
    rp, cols, vals = ti.grid_csr(shape, 4, 1.0, V)
    r = 2 + 6 * (2 + 6 * 2)  # interior point (2,2,2)
    row = dict(zip(cols[rp[r]:rp[r + 1]], vals[rp[r]:rp[r + 1]]))
    assert len(row) == 13
    assert abs(row[r] - 3.75) < 1e-15
    for off in (1, 6, 36):
        assert abs(row[r + off] + 2.0 / 3.0) < 1e-15
        assert abs(row[r - off] + 2.0 / 3.0) < 1e-15
        assert abs(row[r + 2 * off] - 1.0 / 24.0) < 1e-15
        assert abs(row[r - 2 * off] - 1.0 / 24.0) < 1e-15


def test_random_block_column_matches_block():
    B = ti.random_block(1000, 5, 7)
    for j in range(5):
        assert np.array_equal(B[:, j], ti.random_block_column(1000, j, 7))


def test_hat_overlap_csr_in_two_and_one_dimensions():
    """An axis of length 1 is absent: a 2-D grid gives the 9-point tensor
    product, a 1-D grid the tridiagonal (1, 4, 1)/6; columns ascend."""
    import scipy.sparse as sp
    T = lambda n: (np.diag(np.full(n, 4 / 6))                 # noqa: E731
                   + np.diag(np.full(n - 1, 1 / 6), 1)
                   + np.diag(np.full(n - 1, 1 / 6), -1))
    for shape, want in (((5, 4, 1), np.kron(T(4), T(5))), ((7, 1, 1), T(7))):
        rp, ci, v = ti.hat_overlap_csr(shape)
        N = int(np.prod(shape))
        S = sp.csr_matrix((v, ci, rp), shape=(N, N)).toarray()
        assert np.array_equal(S, want)
        for r in range(N):
            assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)
        assert rp.dtype == np.int32 and ci.dtype == np.int32
