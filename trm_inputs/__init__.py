"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the trace-minimization method. It only makes
the *inputs* the method is run on:

* a counter-based random generator (SplitMix64, Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014), used for the
  random initial guess C0 (Sec. 3: "generated from random numbers, followed by
  orthonormalization") and for the well positions and depths;
* the Gaussian-well potential V on a grid;
* an explicit CSR copy of a grid Hamiltonian -1/2 nabla^2 + V, for callers that
  hand the solver a sparse matrix instead of a stencil description;
* the overlap matrix S of trilinear finite-element hat functions on the same
  grid, an SPD matrix for the generalized problem H e = lambda S e;
* the named synthetic workloads (grid size, stencil order, well count, m).

The CUDA path draws C0 on the device with its own implementation of the same
generator; a GPU test checks the two bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "splitmix64", "u64", "uniform01", "random_block", "gaussian_wells",
    "grid_csr", "hat_overlap_csr", "Workload", "WORKLOADS", "workload",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_WELL_TAG = 0x57454C4C53  # "WELLS"


def splitmix64(x):
    """SplitMix64 output function applied to a counter value (vectorised).

    Returns mix(x + 0x9E3779B97F4A7C15) with the two published xor-shift-multiply
    rounds; all arithmetic is modulo 2**64.
    """
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u64(seed, idx):
    """Counter-based 64-bit draw: splitmix64(seed ^ splitmix64(idx))."""
    s = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
    return splitmix64(s ^ splitmix64(idx))


def uniform01(seed, idx):
    """Uniform double in [0, 1) from the top 53 bits of u64(seed, idx)."""
    return (u64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_block(N: int, m: int, seed: int) -> np.ndarray:
    """Random N x m block, column-major, entries uniform in [-0.5, 0.5).

    Entry (i, j) uses counter idx = i + N*j. Returned with Fortran order so that
    column j is contiguous, the layout the solver uses.
    """
    idx = np.arange(N * m, dtype=np.uint64)
    vals = uniform01(seed, idx) - 0.5
    return vals.reshape((m, N)).T.copy(order="F")


def random_block_column(N: int, j: int, seed: int) -> np.ndarray:
    """Column j of random_block(N, m, seed) alone (same counters i + N*j)."""
    idx = np.arange(N, dtype=np.uint64) + np.uint64(N) * np.uint64(j)
    return uniform01(seed, idx) - 0.5


def gaussian_wells(shape, nwells: int, seed: int, h: float = 1.0,
                   depth=(-2.0, -0.5), width: float = 1.5) -> np.ndarray:
    """Sum of `nwells` Gaussian wells sampled on a grid, FP64, x fastest.

    V(r) = sum_k d_k exp(-|r - c_k|^2 / (2 w^2)), with w the standard
    deviation `width`, d_k uniform in `depth` and c_k uniform in the box
    [0, n_x-1] x [0, n_y-1] x [0, n_z-1] (grid units times h). For well k the
    four draws (d, cx, cy, cz) use counters 4k .. 4k+3 of the stream keyed by
    splitmix64(seed ^ "WELLS").
    """
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    key = int(splitmix64(np.uint64(int(seed) ^ _WELL_TAG)))
    k = np.arange(nwells, dtype=np.uint64)
    u = [uniform01(key, 4 * k + f) for f in range(4)]
    d = depth[0] + (depth[1] - depth[0]) * u[0]
    cx = u[1] * (nx - 1) * h
    cy = u[2] * (ny - 1) * h
    cz = u[3] * (nz - 1) * h
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = np.arange(nz) * h
    V = np.zeros((nz, ny, nx))
    inv = 1.0 / (2.0 * width * width)
    for w in range(nwells):
        ex = np.exp(-((x - cx[w]) ** 2) * inv)
        ey = np.exp(-((y - cy[w]) ** 2) * inv)
        ez = np.exp(-((z - cz[w]) ** 2) * inv)
        V += d[w] * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
    return V.reshape(-1)


# Per-axis finite-difference weights of -d^2/dx^2 (times h^2): order 2 is the
# 3-point rule, order 4 the 5-point rule (-1, 16, -30, 16, -1)/12 negated.
_AXIS_WEIGHTS = {2: (2.0, -1.0), 4: (30.0 / 12.0, -16.0 / 12.0, 1.0 / 12.0)}


def grid_csr(shape, order: int, h: float, V, vals_dtype=np.float64):
    """Explicit CSR of H = -1/2 nabla^2_h + diag(V) on a Dirichlet grid.

    Rows and columns are grid points idx = x + nx*(y + ny*z). Axes of length 1
    are absent (a 2-D grid is nz = 1). Neighbours outside the grid are dropped
    (zero Dirichlet ghosts). Columns of each row are in ascending order.
    Returns (rowptr int32[N+1], cols int32[nnz], vals[nnz]).
    """
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    N = nx * ny * nz
    if N >= 2 ** 31:
        raise ValueError("grid too large for int32 CSR")
    w = _AXIS_WEIGHTS[order]
    t = 0.5 / (h * h)
    V = np.asarray(V, dtype=np.float64).reshape(-1)
    idx = np.arange(N, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    axes = [(x, nx, 1), (y, ny, nx), (z, nz, nx * ny)]
    diag = V.copy()
    ndim_active = sum(1 for _, n, _ in axes if n > 1)
    diag += t * w[0] * ndim_active
    # candidate entries as (offset, coefficient, valid mask), ascending offsets
    entries = []
    for coord, n, stride in reversed(axes):
        if n == 1:
            continue
        for s in range(len(w) - 1, 0, -1):
            entries.append((-s * stride, t * w[s], coord - s >= 0))
    entries.append((0, None, np.ones(N, dtype=bool)))
    for coord, n, stride in axes:
        if n == 1:
            continue
        for s in range(1, len(w)):
            entries.append((s * stride, t * w[s], coord + s < n))
    counts = np.zeros(N, dtype=np.int64)
    for _, _, mask in entries:
        counts += mask
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    cols = np.empty(nnz, dtype=np.int64)
    vals = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    for off, coef, mask in entries:
        r = idx[mask]
        pos = fill[mask]
        cols[pos] = r + off
        vals[pos] = diag[mask] if coef is None else coef
        fill[mask] += 1
    return (rowptr.astype(np.int32), cols.astype(np.int32),
            vals.astype(vals_dtype))


def hat_overlap_csr(shape):
    """Explicit CSR of the overlap S_ij = <phi_i, phi_j> of the trilinear hat
    functions of a uniform Dirichlet grid, in units of the cell volume: the
    tensor product over the grid's axes of the 1-D overlap tridiag(1, 4, 1)/6
    (27 points in 3-D). S is symmetric positive definite, the basis being
    non-orthogonal. Same row order, layout and return types as
    :func:`grid_csr` (float64 values)."""
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    N = nx * ny * nz
    if N >= 2 ** 31:
        raise ValueError("grid too large for int32 CSR")
    idx = np.arange(N, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    axes = [(x, nx, 1), (y, ny, nx), (z, nz, nx * ny)]
    # per axis: offsets -1, 0, +1 with weights 1/6, 4/6, 1/6 (an axis of
    # length 1 contributes the single weight 1)
    per_axis = []
    for coord, n, stride in axes:
        if n == 1:
            per_axis.append([(0, 1.0, np.ones(N, dtype=bool))])
        else:
            per_axis.append([(-stride, 1.0 / 6.0, coord - 1 >= 0),
                             (0, 4.0 / 6.0, np.ones(N, dtype=bool)),
                             (stride, 1.0 / 6.0, coord + 1 < n)])
    entries = []
    for oz, wz, mz in per_axis[2]:
        for oy, wy, my in per_axis[1]:
            for ox, wx, mx in per_axis[0]:
                entries.append((oz + oy + ox, wx * wy * wz, mx & my & mz))
    entries.sort(key=lambda e: e[0])        # ascending columns in each row
    counts = np.zeros(N, dtype=np.int64)
    for _, _, mask in entries:
        counts += mask
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    cols = np.empty(nnz, dtype=np.int64)
    vals = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    for off, w, mask in entries:
        r = idx[mask]
        pos = fill[mask]
        cols[pos] = r + off
        vals[pos] = w
        fill[mask] += 1
    return rowptr.astype(np.int32), cols.astype(np.int32), vals


@dataclass(frozen=True)
class Workload:
    """A named synthetic eigenproblem: grid, stencil order, wells, m."""
    name: str
    shape: tuple
    order: int
    nwells: int
    m: int
    h: float = 1.0
    precond: int = 0          # 0 none, 1 diagonal
    seed: int = 0             # well seed (accepted by the gap rule)

    @property
    def N(self) -> int:
        return int(np.prod(self.shape))

    def potential(self) -> np.ndarray:
        if self.nwells == 0:
            return np.zeros(self.N)
        return gaussian_wells(self.shape, self.nwells, self.seed, h=self.h)


# h for the 2-D Laplacian of Sec. 3 (diagonal 4, off-diagonal -1): 1/(2h^2) = 1.
_H_LAPLACE = math.sqrt(0.5)

WORKLOADS = {
    w.name: w for w in [
        Workload("grid16_o2_w8_m16", (16, 16, 16), 2, 8, 16),
        Workload("grid48_o4_w64_m128", (48, 48, 48), 4, 64, 128, precond=1),
        Workload("grid96_o4_w512_m512", (96, 96, 96), 4, 512, 512, precond=1),
        Workload("grid100_o4_w1000_m1024", (100, 100, 100), 4, 1000, 1024,
                 precond=1),
        Workload("laplace2d_96_m220", (96, 96, 1), 2, 0, 220, h=_H_LAPLACE),
        Workload("laplace2d_192_m220", (192, 192, 1), 2, 0, 220, h=_H_LAPLACE),
        Workload("laplace2d_192_m534", (192, 192, 1), 2, 0, 534, h=_H_LAPLACE),
    ]
}


def workload(name: str, seed: int | None = None) -> Workload:
    w = WORKLOADS[name]
    if seed is not None:
        w = Workload(w.name, w.shape, w.order, w.nwells, w.m, w.h, w.precond,
                     seed)
    return w
