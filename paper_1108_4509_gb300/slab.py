"""Z-slab sharding of the block steps over several processes, one GPU each.

Every O(m N) and O(m^2 N) step of the trace minimization is a loop over the
N grid points (Sec. 2.1; Fig. EGFIG, Fig. ONFIG), so rank r keeps only the
rows of its z-slab of every N x m block (:func:`trm_slab_plan`). Two steps
cross slabs:

* applying H: the stencil reaches `radius` planes (1 for the 7-point rule, 2
  for the 13-point rule) into the neighbouring slabs, so before each
  application the boundary planes of the block go to the two neighbours
  (:meth:`Slab.exchange`), and H is applied on the rank's extended grid
  (halo planes + owned planes), of which the owned rows are exact;
* the N-deep sums (the Gram products C^T X', C^T P, P^T P, ..., the energy,
  the norms of the conjugate-gradient scalars) are sums over ranks of the
  partial sums over owned rows: one all-reduce of each m x m (or smaller)
  result (:meth:`Slab.allreduce`).

The m x m work (line step, Cholesky, Rayleigh-Ritz) is the same on every
rank. This module is partition and communication only (torch.distributed:
NCCL between GPUs, gloo between host processes); the local arithmetic is
passed in -- on a GPU the library's kernels (:class:`LibraryOps`: trm_apply_h
on a stencil handle for the extended grid, trm_gram on the owned rows).

Blocks are torch tensors of shape (m, rows): row j of the tensor is column j
of the library's column-major N x m block.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import (TRM_F32, TRM_F64, trm_apply_h, trm_gram, trm_slab_plan)


class Slab:
    """Rank `rank` of `ranks` on an nx x ny x nz stencil grid of the given
    order (2: 7-point, 4: 13-point)."""

    def __init__(self, nx, ny, nz, order, ranks=None, rank=None, group=None):
        self.group = group
        self.ranks = dist.get_world_size(group) if ranks is None else ranks
        self.rank = dist.get_rank(group) if rank is None else rank
        self.nx, self.ny, self.nz, self.order = nx, ny, nz, order
        self.plan = trm_slab_plan(nx, ny, nz, order, self.ranks, self.rank)
        self.plane = nx * ny
        self.radius = 1 if order == 2 else 2
        p = self.plan
        self.rows = int(p.rows)
        self.row0 = int(p.row0)
        self.ext_rows = int(p.ext_rows)
        self.lo = p.halo_lo * self.plane   # rows of the lower halo
        self.hi = p.halo_hi * self.plane   # rows of the upper halo

    # -- layout -------------------------------------------------------------
    def owned_slice(self):
        """Rows [row0, row0 + rows) of the global grid."""
        return slice(self.row0, self.row0 + self.rows)

    def extend(self, X):
        """An (m, ext_rows) block with X's rows in the middle, halos empty."""
        m = X.shape[0]
        Xe = torch.zeros((m, self.ext_rows), dtype=X.dtype, device=X.device)
        Xe[:, self.lo:self.lo + self.rows] = X
        return Xe

    def owned(self, Xe):
        """The owned rows of an extended block, contiguous."""
        return Xe[:, self.lo:self.lo + self.rows].contiguous()

    # -- communication ------------------------------------------------------
    def exchange(self, Xe):
        """Fill the halo rows of the extended block Xe from the neighbours:
        the lowest `radius` owned planes go to rank - 1 (its upper halo), the
        highest to rank + 1 (its lower halo)."""
        k = self.radius * self.plane
        ops, recv = [], []
        lo, rows = self.lo, self.rows
        if self.rank > 0:
            send = Xe[:, lo:lo + k].contiguous()
            buf = torch.empty_like(send)
            ops.append(dist.P2POp(dist.isend, send, self._peer(-1), self.group))
            ops.append(dist.P2POp(dist.irecv, buf, self._peer(-1), self.group))
            recv.append((slice(0, lo), buf))
        if self.rank + 1 < self.ranks:
            send = Xe[:, lo + rows - k:lo + rows].contiguous()
            buf = torch.empty_like(send)
            ops.append(dist.P2POp(dist.isend, send, self._peer(+1), self.group))
            ops.append(dist.P2POp(dist.irecv, buf, self._peer(+1), self.group))
            recv.append((slice(lo + rows, lo + rows + self.hi), buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for sl, buf in recv:
            Xe[:, sl] = buf
        return Xe

    def allreduce(self, t):
        """Sum of t over the ranks, in place (the N-deep partial sums)."""
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def _peer(self, d):
        r = self.rank + d
        return dist.get_global_rank(self.group, r) if self.group else r

    # -- sharded steps ------------------------------------------------------
    def apply_h(self, ops, X):
        """H X on the owned rows: halo exchange, then the local operator on
        the extended grid (ops.apply_ext)."""
        Xe = self.exchange(self.extend(X))
        return self.owned(ops.apply_ext(Xe))

    def gram(self, ops, A, B):
        """A^T B over all N rows: local partial, then the all-reduce."""
        return self.allreduce(ops.gram(A, B))

    def dot(self, ops, A, B):
        """sum(A * B) over all N rows (a trace of a block product)."""
        t = ops.dot(A, B).reshape(1)
        return float(self.allreduce(t).item())


class LibraryOps:
    """The local arithmetic of a slab on the GPU, through the C ABI: a stencil
    handle created for the slab's extended grid (nx x ny x ext_nz, the
    potential of those planes) applies H, trm_gram forms the partial Grams
    over owned rows, and the traces are sums of products on the device."""

    def __init__(self, handle, stream):
        self.h = handle
        self.stream = stream

    def apply_ext(self, Xe):
        dt = TRM_F64 if Xe.dtype == torch.float64 else TRM_F32
        Y = torch.empty_like(Xe)
        trm_apply_h(self.h, dt, Xe.data_ptr(), dt, Y.data_ptr(), Xe.shape[0])
        return Y

    def gram(self, A, B):
        dt = TRM_F64 if A.dtype == torch.float64 else TRM_F32
        m, N = A.shape
        n = B.shape[0]
        out = torch.empty((n, m), dtype=torch.float64, device=A.device)
        trm_gram(N, m, n, dt, A.data_ptr(), B.data_ptr(), out.data_ptr(),
                 self.stream)
        return out  # out[j, i] = (A^T B)(i, j)

    def dot(self, A, B):
        return self.gram(A.reshape(1, -1), B.reshape(1, -1)).reshape(1)
