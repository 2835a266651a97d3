"""Host logic of bench.py: the seeded serving trace and the roofline's use of
the committed ncu summaries (no GPU)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_serving_trace_is_seeded_and_in_range():
    a = bench.serving_trace(2.0, 25)
    b = bench.serving_trace(2.0, 25)
    assert len(a) == len(b) > 10
    times = [t for t, *_ in a]
    assert all(0 < t < 2.0 for t in times) and times == sorted(times)
    for (ta, shape, order, V, m), (tb, shape_b, order_b, Vb, mb) in zip(a, b):
        assert ta == tb and shape == shape_b and order == order_b and m == mb
        assert np.array_equal(V, Vb)
        n = shape[0]
        assert shape == (n, n, n) and 12 <= n <= 40
        assert order in (2, 4) and 8 <= m <= 96 and V.size == n ** 3
    # Poisson arrivals: the mean gap is about 1 / rate
    gaps = np.diff([0.0] + times)
    assert 0.5 / 25 < gaps.mean() < 2.0 / 25


def test_profile_traffic_checks_the_source_hash(tmp_path, monkeypatch):
    # every class mapped to a summary parses while its kernel source matches
    for cls in bench.PROFILE_OF_CLASS:
        tr = bench.traffic_from_profile(cls)
        if tr is None:  # stale summary: the kernel changed since the capture
            continue
        assert tr["bytes_per_launch"] > 0 and tr["algorithmic_bytes"] > 0
    # a summary whose recorded hash does not match the source gives None
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(
        "Algorithmic bytes of the captured launch: 100\n\n"
        "Kernel source at capture: `bench.py` sha256 0000000000000000\n\n"
        "| `dram__bytes_read.sum` | 1.0 Mbyte |\n"
        "| `dram__bytes_write.sum` | 1.0 Mbyte |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "bench.py").write_text("print(1)\n")
    monkeypatch.setitem(bench.PROFILE_OF_CLASS, "gram_f32", "x.md")
    assert bench.traffic_from_profile("gram_f32") is None


def test_roofline_scales_traffic_to_the_class_launch():
    prof = {"gram_f32": {"ms": 100.0, "launches": 10, "bytes": 10 * 1.0e8,
                         "flops": 0.0},
            "small_mm": {"ms": 5.0, "launches": 10, "bytes": 0.0,
                         "flops": 1e9}}
    r, every = bench.roofline(prof, {"hbm_gbs": 6700.0}, "measured")
    assert r["kernel"] == "gram_f32" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 1.0e8 / 10e-3 / 1e9) < 1e-9  # GB/s
    assert abs(r["frac"] - r["achieved"] / 6700.0) < 1e-12
    tr = bench.traffic_from_profile("gram_f32")
    if tr is not None:  # captured bytes x (class bytes / captured algorithmic)
        expect = tr["bytes_per_launch"] * 1.0e8 / tr["algorithmic_bytes"]
        assert abs(r["traffic"] - expect) < 1e-3 * expect
    assert every["small_mm"]["bound"] == "alu"


def test_double_float_classes_use_the_fp32_pipe_ceiling():
    # the mixed ladder's gram_f64 runs in double-float on the FP32 pipe: its
    # ceiling is FP32 SIMT / 12, not the FP64 unit rate
    prof = {"gram_f64": {"ms": 9.0, "launches": 9, "bytes": 0.0,
                         "flops": 9 * 3.6e9},
            "eig": {"ms": 1.0, "launches": 1, "bytes": 0.0, "flops": 1e8}}
    _, every = bench.roofline(prof, {"hbm_gbs": 6700.0}, "measured")
    g = every["gram_f64"]
    assert g["bound"] == "alu" and g["peak"] == bench.DF_TFLOPS
    assert 0.0 < g["frac"] < 1.0
    assert every["eig"]["peak"] == bench.FP64_TFLOPS
    _, fp64 = bench.roofline(prof, {"hbm_gbs": 6700.0}, "measured",
                             double_float=False)
    assert fp64["gram_f64"]["peak"] == bench.FP64_TFLOPS


def test_tensor_core_classes_take_the_binding_roof():
    # m = 512 line Grams: 5 m^2 N flops against 3 blocks of FP32 (12 N m
    # bytes); the TF32 roof / 3 binds, so the class is rated in TFLOP/s
    peaks = {"hbm_gbs": 6700.0, "bf16_tflops": 1900.0,
             "bf16_tflops_sustained": 1700.0}
    N, m = 884736, 512
    fl, by = 5.0 * m * m * N, 12.0 * N * m
    prof = {"gram_f32": {"ms": 6.0, "launches": 1, "bytes": by, "flops": fl}}
    r, _ = bench.roofline(prof, peaks, "measured")
    pk = 1700.0 * bench.TF32_OVER_BF16 / bench.TC_SPLIT
    assert r["bound"] == "tensor" and abs(r["peak"] - pk) < 1e-9
    assert abs(r["achieved"] - fl / 6e-3 / 1e12) < 1e-6
    assert abs(r["frac"] - r["achieved"] / pk) < 1e-12
    assert 0.0 < r["hbm_frac"] < r["frac"]
    # m = 16: the same kind of launch is bound by its bytes
    m = 16
    fl, by = 5.0 * m * m * N, 12.0 * N * m
    prof = {"gram_f32": {"ms": 0.1, "launches": 1, "bytes": by, "flops": fl}}
    r, _ = bench.roofline(prof, peaks, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert 0.0 < r["tensor_frac"] < r["frac"]
