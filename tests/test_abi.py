"""CPU checks of the C ABI: the library builds, loads and exports every entry
point that include/trm.h declares, and host-side argument checks reject bad
input without touching a GPU."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "trm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def trm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as mod
    return mod


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("trm_create_stencil", "trm_create_csr", "trm_solve",
                     "trm_destroy", "trm_apply_h", "trm_gram",
                     "trm_orthonormalize", "trm_rayleigh_ritz"):
        assert required in names


def test_library_exports_every_declared_symbol(trm):
    lib = ct.CDLL(trm.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(trm):
    assert trm.trm_strerror(0) == "success"
    assert trm.trm_strerror(-1) == "invalid argument"
    assert trm.trm_strerror(-4).startswith("no convergence")


def test_default_options(trm):
    o = trm.trm_default_options()
    assert o.precision == trm.TRM_MIXED and o.max_iter > 0 and o.lag >= 1
    assert o.graphs == 1
    # the C layout: 3 ints + pad, uint64, 2 doubles, 3 ints + pad, pointer,
    # int + pad
    assert ct.sizeof(trm.trm_options) == 72


def test_invalid_arguments_rejected_on_host(trm):
    """Argument validation happens before any CUDA call."""
    bad = [
        dict(nx=0, ny=4, nz=4, order=2, h=1.0, m=2),
        dict(nx=4, ny=4, nz=4, order=3, h=1.0, m=2),
        dict(nx=4, ny=4, nz=4, order=2, h=-1.0, m=2),
        dict(nx=4, ny=4, nz=4, order=2, h=1.0, m=0),
        dict(nx=2, ny=2, nz=1, order=2, h=1.0, m=4),
    ]
    for kw in bad:
        with pytest.raises(trm.TrmError) as e:
            trm.trm_create_stencil(kw["nx"], kw["ny"], kw["nz"], kw["order"],
                                   kw["h"], None, kw["m"], 1e-8)
        assert e.value.status == -1
    opt = trm.trm_default_options(precision=9)
    with pytest.raises(trm.TrmError):
        trm.trm_create_stencil(4, 4, 4, 2, 1.0, None, 2, 1e-8, opt)
    import numpy as np
    with pytest.raises(trm.TrmError) as e:
        trm.trm_create_csr(3, np.array([0, 1, 2, 3]), np.array([0, 5, 2]),
                           np.ones(3), 1, 1e-8)
    assert e.value.status == -1


def test_footprint_estimate(trm):
    """The admission estimate grows with N m and covers the N x m blocks the
    solver keeps (92 bytes per entry across FP64, FP32 and pair copies)."""
    a = trm.trm_footprint_bytes(4096, 16)
    b = trm.trm_footprint_bytes(110592, 128)
    assert 92 * 4096 * 16 < a < b
    assert 92 * 110592 * 128 <= b < 130 * 110592 * 128
    assert trm.trm_footprint_bytes(1, 1) == 0


def test_extrapolate_rejects_invalid_arguments_on_the_host(trm):
    # m > N, and an output aliasing an input: refused before any CUDA call
    for args in ((10, 20, 8, 16, 1.0, 24), (100, 4, 8, 16, 1.0, 16)):
        with pytest.raises(trm.TrmError) as e:
            trm.trm_extrapolate(*args)
        assert e.value.status == -1


def test_history_rejects_a_null_handle(trm):
    assert trm.lib.trm_history(None, None, 0) == -1
    with pytest.raises(trm.TrmError):
        trm.trm_history(None)
