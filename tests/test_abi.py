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


def test_header_is_plain_c_and_a_c_program_links(trm, tmp_path):
    """include/trm.h compiles as strict C99 and a C program linked against
    the library calls it (host-only entry points; no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(
        "#include <stdio.h>\n#include \"trm.h\"\n"
        "int main(void) {\n"
        "  trm_options o;\n"
        "  trm_iter_record r;\n"
        "  trm_problem p;\n"
        "  (void)r; (void)p;\n"
        "  if (trm_default_options(&o) != TRM_OK) return 1;\n"
        "  if (o.precision != TRM_MIXED || o.graphs != 1) return 2;\n"
        "  if (trm_history(NULL, NULL, 0) != TRM_EINVAL) return 3;\n"
        "  if (trm_footprint_bytes(1000, 8) == 0) return 4;\n"
        "  printf(\"%s\\n\", trm_strerror(TRM_ENOTPD));\n"
        "  return 0;\n}\n")
    libdir = os.path.dirname(trm.LIB_PATH)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror",
                    "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-ltrm", "-Wl,-rpath," + libdir, "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    assert out.stdout.strip() == trm.trm_strerror(-3)
