"""The allocation-free Gram entry point, trm_gram_noalloc.

Some callers of this library cannot allocate device memory: their framework's
caching allocator or a start-up arena already owns the GPU's memory, or a
fixed memory budget forbids growth, or a latency-critical loop cannot absorb
the synchronisation of cudaMalloc/cudaFree. trm_gram_noalloc serves them with
the split partial sums of the Gram product kept in a fixed array inside the
library. These tests call it through the C ABI and hold it to the result of
the ordinary trm_gram, within the same FP32/FP64 rounding bound the other
Gram tests use, on calls in a row (FP32 operands that trm_gram sends to the
tensor cores must give the same bytes: the same kernel runs). The file name makes pytest collect it
last, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import trm_inputs as ti

from . import gpu_util as gu

pytestmark = pytest.mark.gpu


def gamma(n, u):
    return n * u / (1.0 - n * u)


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


def test_gram_noalloc_matches_gram_on_two_calls(trm):
    torch = gu.torch_mod()
    # two calls in a row with different shapes: the second must not see the
    # first call's partial sums left in the shared scratch
    for N, m, n, seed in [(110592, 128, 128, 1), (5003, 70, 200, 2),
                          (65536, 512, 256, 3)]:
        A = ti.random_block(N, m, seed=seed)
        B = ti.random_block(N, n, seed=seed + 10)
        scale = np.abs(A).T @ np.abs(B)
        for dtype, u, npdt in [(trm.TRM_F64, 2.0 ** -53, np.float64),
                               (trm.TRM_F32, 2.0 ** -24, np.float32)]:
            a, b = gu.to_dev(A.astype(npdt)), gu.to_dev(B.astype(npdt))
            ref = torch.zeros((n, m), dtype=torch.float64, device="cuda")
            got = torch.zeros((n, m), dtype=torch.float64, device="cuda")
            trm.trm_gram(N, m, n, dtype, a.data_ptr(), b.data_ptr(),
                         ref.data_ptr(), gu.stream())
            trm.trm_gram_noalloc(N, m, n, dtype, a.data_ptr(), b.data_ptr(),
                                 got.data_ptr(), gu.stream())
            r, g = gu.from_dev(ref), gu.from_dev(got)
            if dtype == trm.TRM_F32 and N % 4 == 0 and m >= 32:
                # the tensor-core kernel of trm_gram, same slices and order
                assert np.array_equal(g, r)
            # each is within gamma_N |A|^T |B| of the exact product
            assert np.all(np.abs(g - r) <= 2 * gamma(N, u) * scale)
            exact = (A.astype(npdt).astype(np.float64).T
                     @ B.astype(npdt).astype(np.float64))
            assert np.all(np.abs(g - exact) <= gamma(N, u) * scale)


def test_gram_noalloc_rejects_sizes_beyond_its_scratch(trm):
    torch = gu.torch_mod()
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(trm.TrmError) as e:
        trm.trm_gram_noalloc(4, 1025, 1024, trm.TRM_F64, a.data_ptr(),
                             a.data_ptr(), a.data_ptr(), gu.stream())
    assert e.value.status == -1
    assert "scratch" in trm.trm_last_error()
