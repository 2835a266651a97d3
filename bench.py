#!/usr/bin/env python
"""Benchmark: time to E_G at 1e-10 relative error on one GB300.

One timed step is one complete trace-minimization solve (Fig. TMFIG to the
stopping tolerance, then the FP64 Rayleigh-Ritz step) of the workload
"48^3 grid, 13-point 4th-order -1/2 nabla^2 + 64 Gaussian wells, m = 128,
diagonal preconditioner", in the mixed-precision ladder, with the operator
already resident in HBM. Every step's E_G is checked against the stored
reference; a step that misses 1e-10 relative error is reported.

The headline steps replay each kind of iteration as a CUDA graph with no
per-launch events. A second, profiled pass (--profile-steps solves, plain
launches with CUDA events around each) gives the per-class timing; its
slowdown over the headline is reported (profiled_pass.over_headline).

Printed JSON keys beyond the base contract: roofline (dominant kernel class,
from the profiled pass), classes (the same for every kernel class), fp64_path
(the same solve with every operation in FP64), e2e (the solve through the C
ABI from host buffers, copies included), clocks (nvidia-smi sampled during
the headline steps), large (one timed mixed solve of the 96^3, m = 512
workload, its E_G error against the oracle's reference, its per-class
roofline from a short profiled solve, and the FP64 path's time per iteration
extrapolated to a solve), cpu_baseline (the FP64 oracle on all host cores and
on one, bounded samples scaled to a solve, with the host's nproc and CPU);
with --xlarge 1, xlarge (a cold mixed solve of the 100^3, m = 1024 stencil
and the same operator as an FP32/int32 CSR matrix warm-started from it).

--impl reference times the oracle itself (the CPU program), bounded samples.

--serving T replaces the solve benchmark with a serving run: T seconds of
seeded Poisson arrivals of stencil problems (grids 12^3 to 40^3, orders 2 and
4, 4 to 64 Gaussian wells, m = 8 to 96) submitted to the request server; the
same arrival trace is then replayed with one solve at a time for comparison.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grid48_o4_w64_m128"
GOLDEN = os.path.join(ROOT, "tests", "golden", "workloads.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Fallback peaks when the measured file is absent (one earlier GB300 run).
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# Peaks derived from unit counts and the 2070 MHz maximum SM clock:
# FP32 SIMT = 152 SMs x 128 FMA lanes x 2 flops; FP64 = 152 SMs x 2 FMA
# lanes x 2 flops (1.26 TFLOP/s, the nominal 1.25).
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# The mixed ladder's FP64-class Grams and block products run in double-float
# on the FP32 pipe: one pair multiply-add (TwoProduct by FMA with the two
# cross terms, TwoSum into the accumulator, one add) is 12 FP32 instructions
# for 2 algorithmic flops, so their ceiling is the FP32 SIMT rate / 12.
DF_TFLOPS = FP32_SIMT_TFLOPS / 12
DF_CLASSES = ("gram_f64", "rotate_f64")
# Kernel classes whose bound is HBM traffic (algorithmic bytes); the others
# are bound by FP64 (or FP32 SIMT) arithmetic; the tensor-core classes below
# take whichever roof binds them. spmm_df and rotate_df are MP2's
# double-float stencil and split rotation (FP32 pairs, 8 bytes per element
# like FP64).
HBM_CLASSES = ("spmm_f32", "spmm_f64", "spmm_df", "gram_f32", "grad_f32",
               "rotate_f32", "rotate_df", "rowops")
# The classes on the tensor cores: each algorithmic flop is three TF32
# products (hi.hi + hi.lo + lo.hi), so their compute roof is the TF32 rate
# / 3. The TF32 rate is the measured BF16 rate times the nominal TF32/BF16
# ratio (1.1 / 2.25 PFLOP/s dense). A launch is rated against the roof that
# binds it: the larger of its HBM floor (bytes / copy bandwidth) and its
# tensor floor (flops / (TF32 rate / 3)).
TC_CLASSES = ("gram_f32", "grad_f32", "rotate_f32", "rotate_df")
TF32_OVER_BF16 = 1.1 / 2.25
TC_SPLIT = 3
METRIC = "time-to-E_G at 1e-10 rel err (mixed precision)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="RMS residual at which a solve stops")
    ap.add_argument("--fp64", type=int, default=1,
                    help="also time one solve of the all-FP64 path")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="budget of the oracle CPU sample")
    ap.add_argument("--serving", type=float, default=0.0,
                    help="instead of the solve benchmark: seconds of seeded "
                         "Poisson arrivals of mixed problems through the "
                         "request server; prints latency p50/p99 and solves/s")
    ap.add_argument("--rate", type=float, default=20.0,
                    help="serving: mean arrivals per second")
    ap.add_argument("--max-live", type=int, default=16,
                    help="serving: concurrent solves")
    ap.add_argument("--serving-leg", type=float, default=4.0,
                    help="seconds of Poisson arrivals at 50/s served after "
                         "the solve benchmark (the serving key: p50/p99 "
                         "latency and solves/s; 0 leaves it out)")
    ap.add_argument("--compare", type=int, default=1,
                    help="serving: also replay the trace one request at a "
                         "time and compare every result")
    ap.add_argument("--generalized", type=int, default=0,
                    help="instead of the solve benchmark: grid edge n of a "
                         "generalized problem H e = lambda S e (S the hat-"
                         "function overlap) solved in the FP64 mode, timed "
                         "beside the standard problem of the same H")
    ap.add_argument("--chain", type=int, default=0,
                    help="instead of the solve benchmark: grid edge n of a "
                         "chain of related problems V0 + t V1, the third "
                         "solved from a cold, the previous and the "
                         "extrapolated block")
    ap.add_argument("--gen-m", type=int, default=48,
                    help="--generalized: eigenpairs m (at n = 32 the gap "
                         "lambda_49 - lambda_48 is 0.013)")
    ap.add_argument("--chain-m", type=int, default=44,
                    help="--chain: eigenpairs m (at n = 32 the smallest gap "
                         "lambda_45 - lambda_44 along the chain is 0.021)")
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="solves timed again with per-launch events for the "
                         "per-class roofline (after the headline steps)")
    ap.add_argument("--large", type=int, default=1,
                    help="also time one mixed solve of the 96^3, m = 512 "
                         "workload and the FP64 path's time per iteration")
    ap.add_argument("--xlarge", type=int, default=0,
                    help="also time the 100^3, m = 1024 workload: a cold mixed "
                         "solve of the stencil (about five minutes) and the "
                         "same operator as an FP32/int32 CSR matrix solved "
                         "from the stencil's converged block")
    ap.add_argument("--table", type=int, default=0,
                    help="instead of the benchmark: the paper's own 2-D "
                         "Laplacian cases of Table RESTBL (96^2 and 192^2, "
                         "m = 220 and 534), mixed and FP64, time and "
                         "iterations per solve")
    ap.add_argument("--accuracy", type=int, default=0,
                    help="instead of the benchmark: each precision mode's "
                         "accuracy against the oracle's references at "
                         "m = 16, 128, 512")
    ap.add_argument("--clocks", type=int, default=1,
                    help="sample nvidia-smi clocks during the timed region "
                         "(0 under a profiler, which should see no other "
                         "GPU client)")
    return ap.parse_args()


def load_json(path, default=None):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return default


def workload():
    import trm_inputs as ti
    g = load_json(GOLDEN, {}).get(WORKLOAD, {})
    seed = int(g.get("seed", 1))
    return ti.workload(WORKLOAD, seed=seed), g


def describe(w, g, tol):
    return {"workload": (f"{w.name}: {w.shape[0]}^3 grid, 13-point 4th-order "
                         f"-1/2 nabla^2 + {w.nwells} Gaussian wells (seed "
                         f"{w.seed}), m={w.m}, diagonal preconditioner"),
            "N": w.N, "m": w.m, "tol_rms": tol,
            "E_G_ref": g.get("E_G"), "gap": g.get("gap"),
            "inputs": "synthetic, seeded",
            "l2": "256 MB buffer written between timed steps",
            "parallelism": "replicas (one independent solve per GPU)"}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, bounded sample
# ---------------------------------------------------------------------------
_CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import trm_inputs as ti
from oracle import operator as op, trm
w = ti.workload(%(name)r, seed=%(seed)d)
H = op.grid_hamiltonian(w.shape, w.order, w.h, w.potential())
C0 = ti.random_block(w.N, w.m, seed=1)
budget = %(budget)f
t0 = time.time()
stamps = []
def cb(it, E, r):
    stamps.append(time.time())
    if stamps[-1] - t0 > budget:
        raise StopIteration
try:
    trm.solve(H, C0, tol=0.0, max_iter=100000, precond=True, callback=cb)
except StopIteration:
    pass
n = len(stamps) - 1
per = (stamps[-1] - stamps[0]) / max(n, 1)
print(json.dumps({"per_iter_s": per, "iters": n, "wall": time.time() - t0}))
"""


def cpu_sample(w, budget, threads):
    env = dict(os.environ)
    env["OPENBLAS_NUM_THREADS"] = str(threads)
    env["OMP_NUM_THREADS"] = str(threads)
    code = _CPU_SNIPPET % {"root": ROOT, "name": w.name, "seed": w.seed,
                           "budget": budget}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True,
                       text=True, env=env, timeout=budget * 10 + 300)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_description():
    """nproc and the CPU model of the host the oracle runs on."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20)
        for ln in r.stdout.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Vendor ID") and v.strip():
                model = v.strip() if model is None else model + ", " + v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu": model or platform.processor(),
            "machine": platform.machine()}


def cpu_baseline(w, g, budget, iters_to_solve):
    """The oracle on all host cores (its BLAS threaded) and on one core, each
    for half the budget, scaled by the oracle's iterations per solve."""
    host = host_description()
    cores = host["nproc"] or 1
    s_all = cpu_sample(w, budget / 2, cores)
    s_one = cpu_sample(w, budget / 2, 1)
    value = s_all["per_iter_s"] * iters_to_solve
    return {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
            "host": host,
            "sample": (f"{s_all['iters']} FP64 oracle iterations (numpy, "
                       f"{cores} BLAS threads) of the same workload, "
                       f"{s_all['per_iter_s']:.3f} s each, scaled by "
                       f"{iters_to_solve} iterations per solve"),
            "single_core": {"value": s_one["per_iter_s"] * iters_to_solve,
                            "per_iter_s": s_one["per_iter_s"],
                            "iters": s_one["iters"], "cores": 1}}


def iterations_to_solve(g, fallback):
    it = g.get("oracle_iterations_tol_1e-8")
    return int(it) if it else int(fallback)


# ---------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# DRAM traffic of a kernel class from its committed ncu summary (profiles/),
# per launch; None when there is none or the kernel source has changed since
# the capture (the summary records the source file and its sha256 prefix).
# ---------------------------------------------------------------------------
# Each profiler class is one kernel family (the solver keeps MP2's
# double-float stencil and split rotation in classes of their own), so the
# DRAM counters of a capture apply to its class alone.
PROFILE_OF_CLASS = {
    "grad_f32": "k_mul_tc_grad_grid48_m128.md",
    "gram_f32": "k_gram_tc_line_grams_grid48_m128.md",
    "spmm_df": "k_stencil_df_v4_mp2_grid48_m128.md",
    "rotate_df": "k_mul_tc_splitdf_mp2_grid48_m128.md",
    "spmm_f32": "k_stencil_zm_f32_grid48_m128.md",
}


def traffic_from_profile(cls):
    import hashlib
    import re
    name = PROFILE_OF_CLASS.get(cls)
    if not name:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    m = re.search(r"Kernel source at capture: `([^`]+)` sha256 ([0-9a-f]+)", text)
    if not m:
        return None
    try:
        src = open(os.path.join(ROOT, m.group(1)), "rb").read()
    except OSError:
        return None
    if not hashlib.sha256(src).hexdigest().startswith(m.group(2)):
        return None
    total = 0.0
    for metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        mm = re.search(r"`%s` \| ([0-9.]+) (\w+)" % re.escape(metric), text)
        if not mm:
            return None
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[mm.group(2)]
        total += float(mm.group(1)) * scale
    ab = re.search(r"Algorithmic bytes of the captured launch: (\d+)", text)
    return {"bytes_per_launch": total, "source": "profiles/" + name,
            "algorithmic_bytes": int(ab.group(1)) if ab else None}


# ---------------------------------------------------------------------------
# roofline of the dominant kernel class
# ---------------------------------------------------------------------------
def roofline(prof, peaks, src, double_float=True):
    classes = {k: v for k, v in prof.items() if v["launches"] > 0 and v["ms"] > 0}
    if not classes:
        return None, None

    def entry(cname, cc):
        pl = cc["ms"] / 1e3 / cc["launches"]
        if cname in TC_CLASSES and cc["bytes"] > 0 and cc["flops"] > 0:
            bf16 = peaks.get("bf16_tflops_sustained") or peaks["bf16_tflops"]
            tc_pk = bf16 * TF32_OVER_BF16 / TC_SPLIT
            t_hbm = cc["bytes"] / cc["launches"] / (peaks["hbm_gbs"] * 1e9)
            t_tc = cc["flops"] / cc["launches"] / (tc_pk * 1e12)
            hbm = cc["bytes"] / cc["launches"] / pl / 1e9
            tcv = cc["flops"] / cc["launches"] / pl / 1e12
            if t_tc > t_hbm:
                e = {"bound": "tensor", "achieved": tcv, "peak": tc_pk,
                     "unit": "TFLOP/s", "frac": tcv / tc_pk,
                     "peak_source": src + " (BF16 sustained x 1.1/2.25 for "
                     "TF32, / 3 products per algorithmic flop)",
                     "hbm_frac": hbm / peaks["hbm_gbs"]}
            else:
                e = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
                     "peak_source": src + " (copy bandwidth)",
                     "tensor_frac": tcv / tc_pk}
        elif cname in HBM_CLASSES and cc["bytes"] > 0:
            ach = cc["bytes"] / cc["launches"] / pl / 1e9
            e = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                 "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                 "peak_source": src + " (copy bandwidth)"}
        else:
            ach = cc["flops"] / cc["launches"] / pl / 1e12
            if double_float and cname in DF_CLASSES:
                pk, ps = DF_TFLOPS, ("derived double-float on the FP32 pipe "
                                     "(152 SMs x 128 lanes x 2070 MHz / 12 "
                                     "instructions per pair multiply-add)")
            elif cname.endswith("f64") or cname in ("small_mm", "eig"):
                pk, ps = FP64_TFLOPS, "derived FP64 (152 SMs x 2 FMA x 2070 MHz)"
            else:
                pk, ps = FP32_SIMT_TFLOPS, "derived FP32 SIMT (152 SMs x 128 FMA x 2070 MHz)"
            e = {"bound": "alu", "achieved": ach, "peak": pk,
                 "unit": "TFLOP/s", "frac": ach / pk, "peak_source": ps}
        e.update({"launches": cc["launches"], "avg_launch_ms": pl * 1e3})
        return e

    def with_traffic(cname, e):
        # DRAM bytes of the captured launch, scaled to this class's average
        # launch by the ratio of algorithmic bytes (a class mixes launch
        # sizes, e.g. the n = m and n = 3m Grams)
        tr = traffic_from_profile(cname)
        cc = classes[cname]
        if tr and tr["algorithmic_bytes"] and cc["bytes"] > 0:
            per = cc["bytes"] / cc["launches"]
            e.update({"traffic": tr["bytes_per_launch"] * per / tr["algorithmic_bytes"],
                      "traffic_captured": tr["bytes_per_launch"],
                      "traffic_captured_algorithmic": tr["algorithmic_bytes"],
                      "traffic_source": tr["source"]})
        else:
            e.update({"traffic": None, "traffic_source": None})
        return e

    name = max(classes, key=lambda k: classes[k]["ms"])
    r = with_traffic(name, entry(name, classes[name]))
    r.update({"kernel": name,
              "share_of_timed": classes[name]["ms"] / sum(v["ms"] for v in classes.values())})
    every = {k: with_traffic(k, entry(k, v)) for k, v in classes.items()}
    return r, every


# ---------------------------------------------------------------------------
# multi-rank: one independent solve per rank (replicas, weak scaling); the
# job's time per step is the slowest rank's
# ---------------------------------------------------------------------------
def job_seconds(t_local, dist=None, device="cpu"):
    if dist is None:
        return float(t_local)
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, g = workload()
    its = iterations_to_solve(g, g.get("gpu_iterations_hint", 2000))
    budget = max(5.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_sample(w, min(budget, 5.0), 1)
    vals, samples = [], []
    for _ in range(args.steps):
        s = cpu_sample(w, budget, 1)
        samples.append(s)
        vals.append(s["per_iter_s"] * its)
    v = statistics.mean(vals)
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": describe(w, g, args.tol),
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1,
                            "kind": "oracle",
                            "sample": (f"per step: FP64 oracle iterations for "
                                       f"{budget:.0f} s, scaled by {its} "
                                       f"iterations per solve")},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def serving_trace(seconds, rate, seed=2024):
    """Seeded arrival times and problems of the serving run."""
    import numpy as np
    import trm_inputs as ti
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        n = int(rng.integers(12, 41))
        order = int(rng.choice([2, 4]))
        wells = int(rng.integers(4, 65))
        m = int(rng.integers(8, 97))
        V = ti.gaussian_wells((n, n, n), wells, seed=int(rng.integers(1 << 30)))
        out.append((t, (n, n, n), order, V, m))


def serve(trm, trace, max_live, tol, budget, index=None):
    """Replays the trace through a server; returns the per-request results
    and the wall time from the first arrival to the last completion.
    Request k's starting block is seeded by its index in the full trace
    (index[k], default k)."""
    srv = trm.trm_server_create(budget, max_live)
    tickets = []
    t0 = time.perf_counter()
    try:
        for i, (ta, shape, order, V, m) in enumerate(trace):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            opt = trm.trm_default_options(
                precision=trm.TRM_MIXED, precond=1,
                seed=1000 + (i if index is None else index[i]))
            tickets.append(trm.trm_server_submit(srv, shape, order, 1.0, V, m,
                                                 tol, opt))
        res = [trm.trm_server_wait(srv, tk, tr[4])
               for tk, tr in zip(tickets, trace)]
        wall = time.perf_counter() - t0 - trace[0][0]
    finally:
        trm.trm_server_destroy(srv)
    return res, wall


def serving_run(trm, torch, seconds, rate, max_live, tol, compare,
                clocks=True, sample_alone=0):
    """One serving measurement: the seeded trace replayed through a server.
    compare: replay the whole trace one request at a time and compare every
    result; sample_alone > 0: re-solve that many requests (spread over the
    trace) one at a time and compare those."""
    import numpy as np
    trace = serving_trace(seconds, rate)
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    # warm-up: one small solve through a server (module load, attributes)
    serve(trm, trace[:2], 2, tol, budget)
    sampler = ClockSampler(0)
    if clocks:
        sampler.start()
    launches0 = trm.trm_launch_count()
    res, wall = serve(trm, trace, max_live, tol, budget)
    launches = trm.trm_launch_count() - launches0
    clk = sampler.stop()
    lat = np.array([r[4] for r in res])
    seq = None
    if compare:
        seq, wall1 = serve(trm, trace, 1, tol, budget)
        lat1 = np.array([r[4] for r in seq])
    same = None
    if seq is not None:
        same = bool(all(np.array_equal(a[0], b[0]) and a[1] == b[1]
                        for a, b in zip(res, seq)))
    elif sample_alone > 0:
        idx = sorted(set(np.linspace(0, len(trace) - 1,
                                     min(sample_alone, len(trace))).astype(int)))
        alone, _ = serve(trm, [(0.0,) + tuple(trace[i][1:]) for i in idx], 1,
                         tol, budget, index=idx)
        same = bool(all(np.array_equal(res[i][0], a[0]) and res[i][1] == a[1]
                        for i, a in zip(idx, alone)))
        same_how = "%d requests spread over the trace re-solved alone" % len(idx)
    out = {"value": len(trace) / wall, "unit": "solves/s",
           "config": {"workload": "Poisson arrivals of stencil problems",
                      "rate_per_s": rate, "seconds": seconds,
                      "requests": len(trace), "grid": "12^3..40^3",
                      "order": [2, 4], "wells": "4..64", "m": "8..96",
                      "tol": tol, "max_live": max_live},
           "latency_s": {"p50": float(np.percentile(lat, 50)),
                         "p99": float(np.percentile(lat, 99)),
                         "max": float(lat.max())},
           "one_at_a_time": None if seq is None else {
               "solves_per_s": len(trace) / wall1,
               "p50": float(np.percentile(lat1, 50)),
               "p99": float(np.percentile(lat1, 99))},
           "status": sorted({int(r[3]) for r in res}),
           "same_bytes_as_alone": same,
           "gpu_launches": launches, "clocks": clk}
    if seq is None and sample_alone > 0:
        out["same_bytes_checked"] = same_how
    return out


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as trm
    r = serving_run(trm, torch, args.serving, args.rate, args.max_live,
                    args.tol, args.compare, clocks=args.clocks)
    out = {"metric": "serving latency p50/p99 and throughput (mixed precision)",
           "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64",
           "data": "synthetic", **r}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# next rows: the generalized problem and chains of related problems
# ---------------------------------------------------------------------------
def _timed_solve(torch, trm, h, N, m, stream, C0=None, C_out=None):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lam, eg, st, status = trm.trm_solve(h, N, m, C_out=C_out, C0=C0)
    e1.record(stream)
    e1.synchronize()
    return lam, eg, st, status, e0.elapsed_time(e1) / 1e3


def run_generalized(args, torch, trm, stream):
    """FP64 solve of H e = lambda S e (13-point H with wells, S the 27-point
    hat-function overlap) and of H e = lambda e on the same grid; then the
    generalized problem in the mixed ladder (full SP with S in FP32, then
    FP64)."""
    import numpy as np
    import trm_inputs as ti
    n, m = args.generalized, args.gen_m
    shape, N = (n, n, n), n ** 3
    wells = max(4, N // 1024)
    V = ti.gaussian_wells(shape, wells, seed=1)
    S = ti.hat_overlap_csr(shape)
    sptr = stream.cuda_stream

    def make(gen, prec=None):
        opt = trm.trm_default_options(
            precision=trm.TRM_FP64 if prec is None else prec, precond=1,
            stream=sptr, seed=7)
        h = trm.trm_create_stencil(n, n, n, 4, 1.0, V, m, args.tol, opt)
        if gen:
            trm.trm_set_overlap_csr(h, *S)
        return h

    hg, hs = make(True), make(False)
    try:
        for _ in range(args.warmup):
            _timed_solve(torch, trm, hg, N, m, stream)
        trm.trm_profile(hg, True)
        sampler = ClockSampler(torch.cuda.current_device())
        if args.clocks:
            sampler.start()
        launches0 = trm.trm_launch_count()
        times = []
        for _ in range(args.steps):
            lam, eg, st, status, t = _timed_solve(torch, trm, hg, N, m, stream)
            times.append(t)
        launches = (trm.trm_launch_count() - launches0) / max(1, args.steps)
        clocks = sampler.stop()
        prof = trm.trm_profile_read(hg)
        trm.trm_profile(hg, False)
        for _ in range(args.warmup):
            _timed_solve(torch, trm, hs, N, m, stream)
        _, eg_s, st_s, status_s, t_s = _timed_solve(torch, trm, hs, N, m,
                                                    stream)
        hm = make(True, trm.TRM_MIXED)
        try:
            for _ in range(args.warmup):
                _timed_solve(torch, trm, hm, N, m, stream)
            tm = []
            for _ in range(args.steps):
                lam_m, eg_m, st_m, status_m, t = _timed_solve(torch, trm, hm,
                                                              N, m, stream)
                tm.append(t)
        finally:
            trm.trm_destroy(hm)
    finally:
        trm.trm_destroy(hg)
        trm.trm_destroy(hs)
    peaks_file = load_json(PEAKS)
    peaks = peaks_file if peaks_file else FALLBACK
    roof, per_class = roofline(prof, peaks,
                               "measured" if peaks_file else "fallback",
                               double_float=False)
    out = {"metric": "generalized H e = lambda S e: time to tol (FP64 mode)",
           "value": statistics.mean(times), "unit": "s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": False, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{n}^3 grid, 13-point -1/2 nabla^2 + "
                                  f"{wells} Gaussian wells (seed 1), S = "
                                  "trilinear hat-function overlap (27-point "
                                  f"CSR), m={m}, diagonal preconditioner",
                      "N": N, "m": m, "tol_rms": args.tol,
                      "l2": "working set L2-resident (blocks of "
                            f"{N * m * 8 / 1e6:.1f} MB)"},
           "iterations": st.iterations, "status": status,
           "max_residual": st.max_residual, "E_G": eg,
           "standard_same_H": {"seconds": t_s, "iterations": st_s.iterations,
                               "status": status_s, "E_G": eg_s},
           "mixed": {"seconds": statistics.mean(tm),
                     "iterations": st_m.iterations,
                     "iterations_sp_fp64": [st_m.iterations_phase[0],
                                            st_m.iterations_phase[1]],
                     "status": status_m, "max_residual": st_m.max_residual,
                     "E_G": eg_m, "rel_diff_E_G_vs_fp64": abs(eg_m - eg) / abs(eg),
                     "max_abs_diff_lambda_vs_fp64":
                         float(np.max(np.abs(np.asarray(lam_m) - np.asarray(lam)))),
                     "ladder": "full SP (S in FP32, Y = S C in FP32) until its "
                               "floor, then FP64 iterations, then the FP64 "
                               "Rayleigh-Ritz step"},
           "roofline": roof, "classes": per_class,
           "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out))


def run_chain(args, torch, trm, stream):
    """V(t) = V0 + t V1 at t = 0, dt, 2 dt (mixed precision): the third
    problem from a cold start, from the second's block, and from the block
    trm_extrapolate forms from the first two."""
    import numpy as np
    import trm_inputs as ti
    n, m, dt = args.chain, args.chain_m, 0.02
    shape, N = (n, n, n), n ** 3
    wells = max(4, N // 1024)
    V0 = ti.gaussian_wells(shape, wells, seed=31)
    V1 = ti.gaussian_wells(shape, wells, seed=32)
    sptr = stream.cuda_stream

    def solve(t, C0=None):
        opt = trm.trm_default_options(precision=trm.TRM_MIXED, precond=1,
                                      stream=sptr, seed=3)
        h = trm.trm_create_stencil(n, n, n, 4, 1.0, V0 + t * V1, m, args.tol,
                                   opt)
        C = np.zeros((N, m), order="F")
        try:
            _, eg, st, status, secs = _timed_solve(torch, trm, h, N, m, stream,
                                                   C0=C0, C_out=C)
        finally:
            trm.trm_destroy(h)
        return {"seconds": secs, "iterations": st.iterations,
                "status": status, "E_G": eg}, C

    for _ in range(args.warmup):
        solve(0.0)
    _, Ca = solve(0.0)
    _, Cb = solve(dt)
    dA = torch.from_numpy(np.ascontiguousarray(Ca.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(Cb.T)).cuda()
    dX = torch.empty((m, N), dtype=torch.float64, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    trm.trm_extrapolate(N, m, dA.data_ptr(), dB.data_ptr(), 1.0,
                        dX.data_ptr(), sptr)
    e1.record(stream)
    e1.synchronize()
    t_x = e0.elapsed_time(e1) / 1e3
    Cx = np.asfortranarray(dX.cpu().numpy().T)
    cold, _ = solve(2 * dt)
    prev, _ = solve(2 * dt, Cb)
    extr, _ = solve(2 * dt, Cx)
    extr["extrapolate_s"] = t_x
    egs = [cold["E_G"], prev["E_G"], extr["E_G"]]
    out = {"metric": "chain of related problems: time to tol of the third "
                     "(mixed precision)",
           "value": extr["seconds"] + t_x, "unit": "s", "n_gpus": 1,
           "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": f"{n}^3 grid, 13-point, V0 + t V1 with "
                                  f"{wells} + {wells} Gaussian wells (seeds "
                                  f"31, 32), t = 0, {dt}, {2 * dt}, m={m}, "
                                  "diagonal preconditioner",
                      "N": N, "m": m, "tol_rms": args.tol},
           "cold": cold, "previous_block": prev, "extrapolated": extr,
           "E_G_spread": max(egs) - min(egs)}
    print(json.dumps(out))


def run_extras(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_4509_gb300 as trm
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream()
    if args.generalized > 0:
        run_generalized(args, torch, trm, stream)
    if args.chain > 0:
        run_chain(args, torch, trm, stream)
    if args.accuracy:
        run_accuracy(args, torch, trm, stream)
    if args.table:
        run_table(args, torch, trm, stream)
    return 0


TABLE_REF = os.path.join(ROOT, "tests", "golden", "table_restbl_reference.json")
TABLE_PRINTED = os.path.join(ROOT, "tests", "golden", "table_restbl.json")
TABLE_CASES = ["laplace2d_96_m220", "laplace2d_192_m220", "laplace2d_192_m534"]


def run_table(args, torch, trm, stream):
    """The paper's workload (Sec. 3, Table RESTBL): the 2-D Dirichlet
    Laplacian of Eq. LAPLACE, no preconditioner, random C0, solved in the
    mixed ladder and in FP64 to the RMS residual tolerance; E_G against the
    closed form (stored by tests/golden/make_table_reference.py), time and
    iterations per solve and per iteration. The paper's own per-iteration
    seconds (one core of an Opteron 6176 SE, full DP and MP2) are quoted as
    context. The rows with m = 1064 and 1519 exceed this library's m <= 1024."""
    import trm_inputs as ti
    ref = {(r["n"], r["m"]): r for r in load_json(TABLE_REF)["rows"]}
    printed = {(r["n"], r["m"]): r for r in load_json(TABLE_PRINTED)["rows"]}
    sptr = stream.cuda_stream
    rows = []
    for name in TABLE_CASES:
        w = ti.workload(name)
        n = w.shape[0]
        E_ref = ref[(n, w.m)]["E_G"]
        row = {"workload": name, "N": w.N, "m": w.m,
               "E_G_closed_form": E_ref,
               "paper_N_iter_full_dp": printed[(n, w.m)].get("N_iter")}
        for mode, prec in (("mixed", trm.TRM_MIXED), ("fp64", trm.TRM_FP64)):
            opt = trm.trm_default_options(precision=prec, precond=0,
                                          stream=sptr, seed=w.seed + 100)
            h = trm.trm_create_stencil(*w.shape, w.order, w.h, None, w.m,
                                       args.tol, opt)
            try:
                for _ in range(args.warmup if mode == "mixed" else 0):
                    _timed_solve(torch, trm, h, w.N, w.m, stream)
                lam, eg, st, status, t = _timed_solve(torch, trm, h, w.N,
                                                      w.m, stream)
            finally:
                trm.trm_destroy(h)
            row[mode] = {"seconds": t, "iterations": st.iterations,
                         "iterations_phase": list(st.iterations_phase),
                         "seconds_per_iteration": t / max(1, st.iterations),
                         "status": status,
                         "rel_err_E_G": abs(eg - E_ref) / abs(E_ref)}
        row["fp64_over_mixed"] = row["fp64"]["seconds"] / row["mixed"]["seconds"]
        rows.append(row)
    out = {"metric": "Table RESTBL cases: time to tol (mixed and FP64)",
           "value": sum(r["mixed"]["seconds"] for r in rows), "unit": "s",
           "n_gpus": 1, "higher_is_better": False, "dtype": "f32+f64",
           "data": "synthetic (the paper's own matrix, Eq. LAPLACE)",
           "config": {"tol_rms": args.tol, "preconditioner": "none",
                      "C0": "random (counter-based, seeded)"},
           "rows": rows,
           "paper_context": ("Table RESTBL, seconds per iteration on one core "
                             "of an AMD Opteron 6176 SE: 96^2/m=220 DP 0.631, "
                             "MP2 0.491; 192^2/m=220 DP 2.520, MP2 1.968; "
                             "192^2/m=534 DP 12.04, MP2 8.772")}
    print(json.dumps(out))


def run_accuracy(args, torch, trm, stream):
    """Accuracy of each precision mode of Sec. 2.2 against the oracle's
    references (Sec. 4's claims: full SP is not accurate enough, MP2 keeps
    near-DP accuracy): for m = 16, 128, 512 (the 16^3, 48^3 and 96^3
    workloads), each mode's E_G relative error, max |lambda_j - ref_j| and
    Davis-Kahan bound on the largest principal angle, ||H C - C diag(lambda)||_2
    / (lambda_ref_{m+1} - lambda_m), with the residual formed on the host by
    the oracle's H; and the solve time. The all-FP64 solve of the 96^3 case
    (about half an hour) is left out."""
    import numpy as np
    import trm_inputs as ti
    from oracle import operator as op
    gold = load_json(GOLDEN, {})
    modes = {"FP64": trm.TRM_FP64, "MP2": trm.TRM_MP2,
             "FULL_SP": trm.TRM_FULL_SP, "MIXED": trm.TRM_MIXED}
    rows = []
    for name in ("grid16_o2_w8_m16", "grid48_o4_w64_m128",
                 "grid96_o4_w512_m512"):
        g = gold.get(name)
        if not g:
            continue
        w = ti.workload(name, seed=g["seed"])
        V = w.potential()
        H = op.grid_hamiltonian(w.shape, w.order, w.h, V)
        ref = np.array(g["lambdas"])
        lam_m1 = g.get("lambda_m1")
        for mode, code in modes.items():
            if mode == "FP64" and w.m > 128:
                continue
            with trm.Solver.stencil(w.shape, w.order, w.h, V, w.m, 1e-10,
                                    precision=code, precond=1,
                                    seed=w.seed + 100,
                                    stream=stream.cuda_stream) as s:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lam, eg, C, st, status = s.solve()
                t = time.perf_counter() - t0
            R = op.apply_h(H, C) - C * lam[None, :]
            RtR = R.T @ R
            r2 = float(np.sqrt(max(np.linalg.eigvalsh(0.5 * (RtR + RtR.T))[-1], 0)))
            del R
            rows.append({"workload": name, "m": w.m, "mode": mode,
                         "status": status, "iterations": st["iterations"],
                         "seconds": t,
                         "rel_err_E_G": abs(eg - g["E_G"]) / abs(g["E_G"]),
                         "max_abs_err_lambda": float(np.max(np.abs(lam - ref))),
                         "sin_angle_bound": (r2 / (lam_m1 - lam[-1])
                                             if lam_m1 else None),
                         "max_residual": st["max_residual"]})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"accuracy": rows}))


LARGE = "grid96_o4_w512_m512"


def run_large(args, torch, trm, sptr, peaks, src):
    """The 96^3 grid, 13-point stencil + 512 wells, m = 512 (N = 884,736):
    one timed mixed-precision solve (iteration graphs, no per-launch events)
    after a short warm-up solve; a short profiled solve for the per-class
    roofline; and the all-FP64 path's time per iteration (a few iterations
    timed, times the mixed solve's iteration count: an extrapolation, since
    a whole FP64 solve here takes about half an hour)."""
    import trm_inputs as ti
    g = load_json(GOLDEN, {}).get(LARGE, {})
    w = ti.workload(LARGE, seed=int(g.get("seed", 0)))
    V = w.potential()
    nx, ny, nz = w.shape
    E_ref = g.get("E_G")

    def handle(**o):
        opt = trm.trm_default_options(precision=trm.TRM_MIXED, precond=1,
                                      stream=sptr, seed=w.seed + 100, **o)
        return trm.trm_create_stencil(nx, ny, nz, w.order, w.h, V, w.m,
                                      args.tol, opt)

    stream = torch.cuda.current_stream()
    hw = handle(max_iter=30)             # warm-up (stencil choice, first launches)
    trm.trm_solve(hw, w.N, w.m)
    trm.trm_destroy(hw)
    h = handle()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lam, eg, st, status = trm.trm_solve(h, w.N, w.m)
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    # FP64 path: time per iteration from an orthonormal random block
    C = torch.empty(w.N * w.m, dtype=torch.float64, device="cuda")
    trm.trm_random_block(w.N, w.m, 7, C.data_ptr(), sptr)
    trm.trm_orthonormalize(w.N, w.m, C.data_ptr(), sptr)
    trm.trm_set_block(h, C.data_ptr())
    del C
    trm.trm_iterate(h, trm.TRM_FP64, restart=True)   # first step untimed
    it64 = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        trm.trm_iterate(h, trm.TRM_FP64, restart=False)
        it64.append(time.perf_counter() - t0)
    trm.trm_destroy(h)
    # per-class roofline from a profiled capped solve (events around launches)
    hp = handle(max_iter=60)
    trm.trm_profile(hp, True)
    trm.trm_solve(hp, w.N, w.m)
    prof = trm.trm_profile_read(hp)
    trm.trm_destroy(hp)
    roof, per_class = roofline(prof, peaks, src)
    per64 = statistics.mean(it64)
    return {"workload": (f"{w.name}: {w.shape[0]}^3 grid, 13-point 4th-order "
                         f"-1/2 nabla^2 + {w.nwells} Gaussian wells (seed "
                         f"{w.seed}), m={w.m}, diagonal preconditioner"),
            "N": w.N, "m": w.m, "tol_rms": args.tol, "seconds": t,
            "iterations": st.iterations,
            "iterations_phase": list(st.iterations_phase), "status": status,
            "rms_residual": st.rms_residual, "E_G": eg, "E_G_ref": E_ref,
            "E_G_ref_source": g.get("method"),
            "rel_err_E_G": abs(eg - E_ref) / abs(E_ref) if E_ref else None,
            "launch_mode": "each kind of iteration replayed as a CUDA graph",
            "fp64_path": {"seconds_per_iteration": per64,
                          "seconds_extrapolated": per64 * st.iterations,
                          "mixed_speedup_extrapolated": per64 * st.iterations / t,
                          "how": ("2 FP64 iterations (trm_iterate) timed on the "
                                  "host after one untimed, times the mixed "
                                  "solve's iteration count")},
            "roofline": roof, "classes": per_class,
            "profiled": "first 60 iterations of the same solve, events around each launch"}


XLARGE = "grid100_o4_w1000_m1024"


def run_xlarge(args, torch, trm, sptr):
    """The 100^3 grid, 13-point stencil + 1000 wells, m = 1024 (N = 10^6):
    one timed cold mixed-precision solve of the stencil (iteration graphs,
    after a 20-iteration warm-up solve), then the same operator as an
    explicit CSR matrix (FP32 values, int32 columns) solved from the
    stencil's converged block (a related request's warm start). E_G against
    the oracle's filtered-subspace reference; the CSR values are the FP32
    roundings, so its E_G differs from the reference by up to m 2^-24 10."""
    import numpy as np
    import trm_inputs as ti
    g = load_json(GOLDEN, {}).get(XLARGE, {})
    w = ti.workload(XLARGE, seed=int(g.get("seed", 0)))
    V = w.potential()
    E_ref = g.get("E_G")
    opts = dict(precision=trm.TRM_MIXED, precond=1, seed=w.seed + 100,
                stream=sptr)
    stream = torch.cuda.current_stream()

    def timed(solver, C0=None):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam, eg, C, st, status = solver.solve(C0=C0)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, eg, C, st, status

    with trm.Solver.stencil(w.shape, w.order, w.h, V, w.m, args.tol,
                            max_iter=20, **opts) as s:
        s.solve(want_C=False)
    with trm.Solver.stencil(w.shape, w.order, w.h, V, w.m, args.tol,
                            **opts) as s:
        t, eg, C, st, status = timed(s)
    rp, ci, va = ti.grid_csr(w.shape, w.order, w.h, V, np.float32)
    with trm.Solver.csr(w.N, rp, ci, va, w.m, args.tol, **opts) as s:
        tc, egc, _, stc, statusc = timed(s, C0=C)
    rel = (lambda e: abs(e - E_ref) / abs(E_ref)) if E_ref else (lambda e: None)
    return {"workload": (f"{w.name}: {w.shape[0]}^3 grid, 13-point 4th-order "
                         f"-1/2 nabla^2 + {w.nwells} Gaussian wells (seed "
                         f"{w.seed}), m={w.m}, diagonal preconditioner"),
            "N": w.N, "m": w.m, "tol_rms": args.tol, "E_G_ref": E_ref,
            "E_G_ref_source": g.get("method"),
            "stencil": {"seconds": t, "iterations": st["iterations"],
                        "iterations_phase": st["iterations_phase"],
                        "status": status, "E_G": eg, "rel_err_E_G": rel(eg)},
            "csr_warm_start": {"seconds": tc, "iterations": stc["iterations"],
                               "status": statusc, "E_G": egc,
                               "rel_err_E_G": rel(egc),
                               "nnz": int(rp[-1])},
            "launch_mode": "each kind of iteration replayed as a CUDA graph"}


def main():
    args = parse()
    if args.serving > 0:
        return run_serving(args)
    if args.generalized > 0 or args.chain > 0 or args.accuracy or args.table:
        return run_extras(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_1108_4509_gb300 as trm

    w, g = workload()
    V = w.potential()
    E_ref = g.get("E_G")
    # a side stream: the library captures iterations as CUDA graphs only on
    # a non-default stream
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    nx, ny, nz = w.shape
    opt = trm.trm_default_options(precision=trm.TRM_MIXED, precond=1,
                                  stream=sptr, seed=w.seed + 100)
    h = trm.trm_create_stencil(nx, ny, nz, w.order, w.h, V, w.m, args.tol, opt)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def solve_once():
        lam, eg, st, status = trm.trm_solve(h, w.N, w.m)
        return lam, eg, st, status

    def timed(n):
        out = []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam, eg, st, status = solve_once()
            e1.record(stream)
            e1.synchronize()
            out.append((e0.elapsed_time(e1) / 1e3, eg, st, status))
        return out

    for _ in range(args.warmup):
        solve_once()
    torch.cuda.synchronize()
    # headline: iterations replayed as CUDA graphs, no per-launch events
    sampler = ClockSampler(torch.cuda.current_device())
    if args.clocks:
        sampler.start()
    launches0 = trm.trm_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    runs = timed(args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = trm.trm_launch_count() - launches0
    clocks = sampler.stop()
    times = [r[0] for r in runs]
    errs = [abs(r[1] - E_ref) / abs(E_ref) if E_ref else None for r in runs]
    iters = [r[2].iterations for r in runs]
    statuses = [r[3] for r in runs]
    t_step = job_seconds(statistics.mean(times), dist, "cuda")

    # profiled pass (its own timed region): the same solves with CUDA events
    # around every launch, graphs off; gives the per-class roofline
    nprof = max(1, min(args.profile_steps, args.steps))
    trm.trm_profile(h, True)
    pruns = timed(nprof)
    prof = trm.trm_profile_read(h)
    trm.trm_profile(h, False)
    t_prof = statistics.mean(r[0] for r in pruns)

    peaks_file = load_json(PEAKS)
    peaks = peaks_file if peaks_file else FALLBACK
    src = "measured" if peaks_file else "fallback"
    roof, per_class = roofline(prof, peaks, src)

    # all-FP64 path, one solve (not part of the timed region)
    fp64 = None
    if args.fp64 and rank == 0:
        opt64 = trm.trm_default_options(precision=trm.TRM_FP64, precond=1,
                                        stream=sptr, seed=w.seed + 100)
        h64 = trm.trm_create_stencil(nx, ny, nz, w.order, w.h, V, w.m,
                                     args.tol, opt64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam64, eg64, st64, status64 = trm.trm_solve(h64, w.N, w.m)
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        trm.trm_destroy(h64)
        fp64 = {"seconds": t64, "iterations": st64.iterations,
                "status": status64,
                "rel_err_E_G": abs(eg64 - E_ref) / abs(E_ref) if E_ref else None,
                "mixed_speedup": t64 / t_step}

    # end to end through the C ABI from host buffers: create (V host->device)
    # + solve + C and lambda device->host, per step
    e2e_times = []
    C_host = np.zeros((w.N, w.m), order="F")
    n_e2e = max(1, min(2, args.steps))
    for _ in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = trm.trm_create_stencil(nx, ny, nz, w.order, w.h, V, w.m,
                                    args.tol, opt)
        lam2, eg2, st2, status2 = trm.trm_solve(h2, w.N, w.m, C_out=C_host)
        trm.trm_destroy(h2)
        e2e_times.append(time.perf_counter() - t0)
    e2e = {"value": statistics.mean(e2e_times), "unit": "s",
           "h2d_bytes_per_step": 8 * w.N,
           "d2h_bytes_per_step": 8 * w.N * w.m + 8 * w.m + 8}
    trm.trm_destroy(h)

    large = None
    if args.large and rank == 0:
        try:
            large = run_large(args, torch, trm, sptr, peaks, src)
        except Exception as exc:  # reported, not fatal
            large = {"error": str(exc)[:300]}

    xlarge = None
    if args.xlarge and rank == 0:
        try:
            xlarge = run_xlarge(args, torch, trm, sptr)
        except Exception as exc:  # reported, not fatal
            xlarge = {"error": str(exc)[:300]}

    serving = None
    if args.serving_leg > 0 and rank == 0:
        try:
            serving = serving_run(trm, torch, args.serving_leg, 50.0,
                                  args.max_live, args.tol, 0,
                                  clocks=args.clocks, sample_alone=8)
        except Exception as exc:  # reported, not fatal
            serving = {"error": str(exc)[:300]}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        try:
            cpu = cpu_baseline(w, g, args.cpu_seconds,
                               iterations_to_solve(g, statistics.mean(iters)))
        except Exception as exc:  # reported, not fatal
            cpu = {"error": str(exc)[:300]}

    if rank == 0:
        out = {"metric": METRIC, "value": t_step, "unit": "s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": t_step * 1e3, "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
               "data": "synthetic", "config": describe(w, g, args.tol),
               "solves_per_s": world / t_step,
               "iterations": iters, "status": statuses,
               "rel_err_E_G": errs,
               "E_G_ok": all(e is not None and e <= 1e-10 for e in errs),
               "roofline": roof, "classes": per_class,
               "profile_ms_per_solve": {
                   k: round(v["ms"] / nprof, 3) for k, v in prof.items()
                   if v["launches"]},
               "profiled_pass": {"steps": nprof, "seconds_per_solve": t_prof,
                                 "over_headline": t_prof / t_step},
               "fp64_path": fp64,
               "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
               "launch_mode": {
                   "timed": "each kind of iteration replayed as a CUDA graph",
                   "profiled_pass": "plain launches, CUDA events around each",
                   "e2e": "each kind of iteration replayed as a CUDA graph"},
               "tensor_core_split": {
                   "gram_f32, grad_f32, rotate_f32, rotate_df":
                       "tcgen05 kind::tf32, FP32 value = TF32 hi + TF32 lo, "
                       "three products hi.hi + hi.lo + lo.hi, FP32 accumulation "
                       "in tensor memory"},
               "large": large,
               **({"xlarge": xlarge} if xlarge is not None else {}),
               "serving": serving,
               "cpu_baseline": cpu}
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
