"""The request server's native scheduler under the host sanitizers (CPU, no
GPU): csrc/server.cu is compiled alone with ThreadSanitizer, and again with
AddressSanitizer + UndefinedBehaviorSanitizer, linked with stand-ins for the
solver entry points (tests/native/server_stubs.cu) and driven by
tests/native/server_harness.cpp: six client threads submitting and waiting
on one server whose requests run a host function. Any report fails the run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1108_4509_gb300", "csrc")
NATIVE = os.path.join(ROOT, "tests", "native")
CUDA = "/usr/local/cuda"


def _tool(name):
    return shutil.which(name) or (os.path.join(CUDA, "bin", name)
                                  if os.path.exists(os.path.join(CUDA, "bin", name))
                                  else None)


@pytest.mark.parametrize("sanitizers", [["thread"], ["address", "undefined"]])
def test_scheduler_is_clean_under_sanitizers(tmp_path, sanitizers):
    nvcc, gxx = _tool("nvcc"), shutil.which("g++")
    if nvcc is None or gxx is None:
        pytest.skip("needs nvcc and g++")
    san = [f"-fsanitize={s}" for s in sanitizers]
    xsan = [a for s in san for a in ("-Xcompiler", s)]
    common = ["-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-g",
              "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    objs = []
    for src in (os.path.join(CSRC, "server.cu"),
                os.path.join(NATIVE, "server_stubs.cu")):
        obj = str(tmp_path / (os.path.basename(src) + ".o"))
        subprocess.run([nvcc, *common, *xsan, "-c", src, "-o", obj],
                       check=True)
        objs.append(obj)
    exe = str(tmp_path / "harness")
    libdir = os.path.join(CUDA, "lib64")
    subprocess.run([gxx, "-std=c++17", "-O1", "-g", *san,
                    "-I" + os.path.join(ROOT, "include"),
                    os.path.join(NATIVE, "server_harness.cpp"), *objs,
                    "-L" + libdir, "-lcudart", "-Wl,-rpath," + libdir,
                    "-lpthread", "-o", exe], check=True)
    env = dict(os.environ,
               TSAN_OPTIONS="halt_on_error=1 exitcode=66",
               ASAN_OPTIONS="detect_leaks=1",
               UBSAN_OPTIONS="halt_on_error=1 print_stacktrace=1")
    out = subprocess.run([exe], capture_output=True, text=True, env=env,
                         timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "bad 0" in out.stdout
