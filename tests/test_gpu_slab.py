"""The z-slab partition on one GPU: every rank's local arithmetic runs
through the library (paper_1108_4509_gb300.slab.LibraryOps: a stencil handle
for the rank's extended grid, trm_gram on its owned rows), the ranks one after
another in this process, with each rank's halo planes filled from the full
block -- what the exchange between ranks delivers. The owned rows of H C must
equal the full-grid product bit for bit (the same terms in the same order per
point), and the per-rank Gram partials must sum to the single-GPU Gram within
the FP64 rounding of a split sum."""
import numpy as np
import pytest

import trm_inputs as ti

from . import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


@pytest.mark.parametrize("shape,order,ranks", [((20, 16, 24), 2, 2),
                                               ((20, 16, 24), 4, 3),
                                               ((32, 12, 21), 4, 4)])
def test_slabs_reproduce_the_full_grid(trm, shape, order, ranks):
    torch = gu.torch_mod()
    from paper_1108_4509_gb300.slab import LibraryOps, Slab
    nx, ny, nz = shape
    N, m = nx * ny * nz, 6
    V = ti.gaussian_wells(shape, 7, seed=5)
    C = ti.random_block(N, m, seed=8)
    Ct = gu.to_dev(C)                       # (m, N)
    full = gu.empty(N, m, np.float64)
    opt = trm.trm_default_options(stream=gu.stream())
    hf = trm.trm_create_stencil(nx, ny, nz, order, 1.0, V, 1, 1e-8, opt)
    try:
        trm.trm_apply_h(hf, trm.TRM_F64, Ct.data_ptr(), trm.TRM_F64,
                        full.data_ptr(), m)
        gram_full = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        trm.trm_gram(N, m, m, trm.TRM_F64, Ct.data_ptr(), Ct.data_ptr(),
                     gram_full.data_ptr(), gu.stream())
    finally:
        trm.trm_destroy(hf)
    plane = nx * ny
    gram_sum = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    rows = 0
    for r in range(ranks):
        slab = Slab(nx, ny, nz, order, ranks=ranks, rank=r)
        p = slab.plan
        Ve = V[p.ext_z0 * plane:(p.ext_z0 + p.ext_nz) * plane]
        h = trm.trm_create_stencil(nx, ny, p.ext_nz, order, 1.0, Ve, 1, 1e-8,
                                   opt)
        try:
            ops = LibraryOps(h, gu.stream())
            own = slab.owned_slice()
            X = Ct[:, own].contiguous()
            Xe = slab.extend(X)
            # the halo planes as the neighbours' exchange delivers them
            lo = p.ext_z0 * plane
            Xe[:, :slab.lo] = Ct[:, lo:lo + slab.lo]
            hi0 = p.z1 * plane
            Xe[:, slab.lo + slab.rows:] = Ct[:, hi0:hi0 + slab.hi]
            Y = slab.owned(ops.apply_ext(Xe))
            assert torch.equal(Y, full[:, own]), r
            gram_sum += ops.gram(X, X)
            rows += slab.rows
        finally:
            trm.trm_destroy(h)
    torch.cuda.synchronize()
    assert rows == N
    scale = np.abs(C).T @ np.abs(C)
    diff = (gram_sum - gram_full).cpu().numpy()
    assert np.all(np.abs(diff) <= 4 * N * 2.0 ** -53 * scale)
