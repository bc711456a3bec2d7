#!/usr/bin/env python3
"""Throughput of TPMG-preconditioned CG on one GB300 (or N independent replicas).

A step is one full solve, from a zero initial guess to a 1e-5 reduction of the
residual 2-norm, of the pressure-correction system -omega^2 div grad u + u = f
on the thin spherical shell, with the inputs resident in HBM.  The metric is
unknowns per second (unknowns x steps / device time).

Default workload: icosahedral refinement 6 (81,920 triangles) x 64 vertical
levels graded 1.05 over a 10 km shell (5,242,880 unknowns), omega^2/h^2 = 80,
manufactured solution u* = sum of 8 seeded low-order spherical harmonics x
vertical cosines, f = A u*; 6 multigrid levels, 2/2 line-SOR sweeps, 1 coarse
sweep; FP64 throughout.

Other workloads (--workload): batch48 (48 uneven mixed-precision solves in one
graph launch), 1280x16 (the small parity case), 81920x64-mixed
(the same solve with the V-cycle in FP32 on a BF16 stencil and flexible CG in
FP64), 327680x128-mixed (refinement 7 x 128 levels, 41.9M unknowns, mixed
precision), 327680x128 (the same grid in FP64) and 327680x128-learned (the
learned form).  Two studies print the paper's measurements instead of a
throughput: nr-sweep (time per iteration against n_r, Sec. 5.1) and
balanced-flow (TPMG^fac / TPMG^partial / TPMG^full against the buoyancy
frequency, Sec. 5).

Flags: --gpus N --steps K --warmup W [--impl tpmg|reference] [--workload NAME]
Under torchrun (N > 1) every rank solves its own replica (no data exchange:
the path shards only through independent problems on this pool).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns/sec to 1e-5 residual reduction (TPMG-PCG) at 1 GB300; HBM GB/s vs peak"

MIXED = dict(precision=1, coeff_storage=1)   # TPMG_PREC_MIXED, TPMG_COEFF_FULL

WORKLOADS = {
    "81920x64": dict(
        params=dict(refinement=6, n_levels=6, n_r=64, grading=1.05, courant_c=80.0, nu_pre=2, nu_post=2, nu_coarse=1),
        rhs="manufactured", seed=2981002,
        text="icosahedral refinement 6 (81920 triangles) x 64 levels graded 1.05 over 10 km, omega^2/h^2=80, "
             "manufactured spherical-harmonic x cosine solution, f = A u*, 6 MG levels, nu 2/2/1, rtol 1e-5"),
    "1280x16": dict(
        params=dict(refinement=3, n_levels=4, n_r=16, grading=1.0, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1),
        rhs="uniform", seed=2981001,
        text="icosahedral refinement 3 (1280 triangles) x 16 uniform levels over 10 km, omega^2/h^2=8, "
             "RHS uniform[-1,1], 4 MG levels, nu 1/1/1, rtol 1e-5"),
    "81920x64-mixed": dict(
        params=dict(refinement=6, n_levels=6, n_r=64, grading=1.05, courant_c=80.0, nu_pre=2, nu_post=2, nu_coarse=1,
                    **MIXED),
        rhs="manufactured", seed=2981002,
        text="as 81920x64, V-cycle in FP32 on a BF16 stencil, outer flexible CG in FP64"),
    "327680x128-mixed": dict(
        params=dict(refinement=7, n_levels=6, n_r=128, grading=1.05, courant_c=8.0, nu_pre=2, nu_post=2, nu_coarse=1,
                    **MIXED),
        rhs="uniform", seed=2981003,
        text="icosahedral refinement 7 (327680 triangles) x 128 levels graded 1.05 over 10 km, omega^2/h^2=8, "
             "RHS uniform[-1,1], 6 MG levels, nu 2/2/1, V-cycle in FP32 on a BF16 stencil, outer flexible CG "
             "in FP64, rtol 1e-5"),
    "327680x128": dict(
        params=dict(refinement=7, n_levels=6, n_r=128, grading=1.05, courant_c=8.0, nu_pre=2, nu_post=2, nu_coarse=1),
        rhs="uniform", seed=2981003,
        text="as 327680x128-mixed, everything in FP64 (plain TPMG-PCG on the same grid)"),
    "327680x128-learned": dict(
        params=dict(refinement=7, n_levels=6, n_r=128, grading=1.05, courant_c=8.0, nu_pre=2, nu_post=2, nu_coarse=1,
                    **MIXED),
        learned=dict(pairs=2000, cells_per_pair=512, coarse_per_pair=4, hidden=64, l_max=16, train_steps=4000,
                     batch=4096, lr=2e-3),
        rhs="smooth", seed=2981005,
        text="learned form on the 327680x128-mixed grid: a 4-layer per-column network (2 n_r -> 64 -> 64 -> 64 -> "
             "n_r, BF16 weights, FP32 accumulate) as coarsest-level solve and as warm start (+ one line "
             "relaxation), trained by the library's kernels on 2000 seeded (f, u) pairs from plain TPMG-PCG "
             "(smooth f: spherical harmonics up to degree 16 x vertical cosines); flexible CG, "
             "||r|| <= 1e-5 ||f|| on held-out smooth right-hand sides"),
    "nr-sweep": dict(
        study="nr_sweep", refinement=6, n_r=(16, 32, 64, 128, 256), iters=8, seed=2981010,
        text="time per PCG iteration against the number of vertical levels (Sec. 5.1, eq. nzDependency: "
             "t_iter = C + q n_r): icosahedral refinement 6 (81920 columns) x n_r in {16, 32, 64, 128, 256} "
             "graded 1.05 over 10 km, omega^2/h^2=80, RHS uniform[-1,1], 6 MG levels, nu 2/2/1, 8 iterations per "
             "solve (rtol 0); V-cycle TPMG^fac in FP64, TPMG^full in FP64, TPMG^full in mixed precision"),
    "balanced-flow": dict(
        study="balanced_flow", refinement=5, n_r=128, seed=2981011, advection=True,
        n_freq=(None, 0.022, 0.025, 0.028),   # None: N* = g / sqrt(cp T0), where the profiles factorise
        text="balanced zonal flow (Sec. 5, after Davies 2005) at the paper's size: icosahedral refinement 5 "
             "(20480 columns) x 128 levels graded 1.05 over 10 km (2.6M unknowns), omega^2/h^2=8, RHS "
             "uniform[-1,1], 6 MG levels, nu 2/2/1, rtol 1e-5; buoyancy frequency N in {N*, 0.022, 0.025, "
             "0.028} 1/s; the full operator with vertical advection preconditioned by TPMG^fac, TPMG^partial, "
             "TPMG^full (FP64) and TPMG^full (mixed precision) with Richardson and BiCGStab"),
    "balanced-flow-symmetric": dict(
        study="balanced_flow", refinement=5, n_r=128, seed=2981011, advection=False,
        n_freq=(None, 0.022, 0.025, 0.028),
        text="the balanced-flow study without vertical advection (a symmetric operator, so CG applies too): "
             "icosahedral refinement 5 x 128 levels graded 1.05 over 10 km (2.6M unknowns), omega^2/h^2=8, RHS "
             "uniform[-1,1], 6 MG levels, nu 2/2/1, rtol 1e-5; TPMG^fac, TPMG^partial, TPMG^full (FP64) and "
             "TPMG^full (mixed precision) with Richardson, CG and BiCGStab"),
    "prolongation": dict(
        study="prolongation", seed=2981006,
        params=dict(refinement=6, n_levels=6, n_r=64, grading=1.05, courant_c=80.0, nu_pre=2, nu_post=2, nu_coarse=1),
        text="piecewise-constant (P = R^T) against linear prolongation (Sec. 5) on the 81920x64 grid: RHS "
             "uniform[-1,1] (rough, so that the transfer matters), rtol 1e-5, FP64 and mixed-precision V-cycles, "
             "Richardson and BiCGStab"),
    "batch48": dict(
        batch=48, seed=2981004,
        text="48 independent solves in one graph launch: refinement drawn from {4,5,6}, vertical levels from "
             "{32,64,128} graded 1.05, omega^2/h^2 log-uniform in [4,200], all seeded; RHS uniform[-1,1]; "
             "V-cycle in FP32 on a BF16 stencil, outer flexible CG in FP64; 5-6 MG levels, nu 2/2/1, rtol 1e-5"),
}


def batch_problems(seed: int, n: int) -> list:
    """The seeded parameter sets of the batched workload."""
    from paper_1408_2981_gb300 import inputs

    refs = inputs.randint(seed, n, 4, 6)
    nrs = np.array([32, 64, 128])[inputs.randint(seed, n, 0, 2, offset=n)]
    cs = np.exp(np.log(4.0) + (np.log(200.0) - np.log(4.0)) * inputs.uniform01(seed, n, offset=2 * n))
    return [dict(refinement=int(r), n_levels=int(min(r, 5) + 1 if r < 6 else 6), n_r=int(k), grading=1.05,
                 courant_c=float(c), nu_pre=2, nu_post=2, nu_coarse=1, **MIXED) for r, k, c in zip(refs, nrs, cs)]

# Kernel classes of the outer Krylov iteration: FP64 in every form (the V-cycle's
# classes -- relax, restrict, prolong -- run in FP32 in the mixed form).
OUTER_FP64 = ("apply", "residual", "axpy", "dot", "xpby", "finish")
FP32_FMA_PER_CLK_PER_SM = 128   # nominal FP32 lanes per SM (only used to name the binding ceiling)
ORACLE_FULL_SOLVE_MAX_UNKNOWNS = 6_000_000   # larger workloads: the CPU baseline times one iteration


def source_sha256(name: str) -> str:
    import hashlib

    with open(os.path.join(ROOT, "paper_1408_2981_gb300", "csrc", name), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def traffic_records() -> list:
    """Machine-readable lines of the ncu summaries in profiles/ of the form
    ``traffic: class=<kernel class> workload=<name> <source file>=<sha256 prefix> bytes_per_launch=<B>``:
    DRAM bytes (read + write) per launch of a kernel class on a workload, measured
    while the named kernel source had that hash."""
    import glob
    import re

    pat = re.compile(r"traffic: class=(\w+) workload=(\S+) (\S+)=([0-9a-f]{16}) bytes_per_launch=([0-9.eE+]+)"
                     r"(?: algorithmic_per_launch=([0-9.eE+]+))?(?: scope=(\S+))?")
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for m in pat.finditer(fh.read()):
                out.append(dict(kernel=m.group(1), workload=m.group(2), file=m.group(3), sha256=m.group(4),
                                bytes_per_launch=float(m.group(5)),
                                algorithmic_per_launch=float(m.group(6)) if m.group(6) else None,
                                scope=(m.group(7) or "").replace("-", " ") or None,
                                source=os.path.relpath(path, ROOT)))
    return out


def traffic_of(kernel: str, workload: str):
    """ncu DRAM bytes per launch of the class, or None when no capture matches the
    current kernel source."""
    for t in traffic_records():
        if t["kernel"] == kernel and t["workload"] == workload and t["sha256"] == source_sha256(t["file"]):
            return t
    return None


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d.get("hbm_gbs", 6800.0)), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def fp32_nominal_tflops(sm_count: int, mhz: float) -> float:
    return sm_count * FP32_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12


def roofline_of(prof: dict, before: dict, dominant: str, mixed: bool, steps: int, step_ms: float,
                fp64_tflops: float, sm_count: int, workload: str, kernel_note: str = "") -> dict:
    """Roofline of a kernel class from its timed launches: the algorithmic bytes and
    flops the library counted for the launches inside the class's event pairs, over
    their summed device time.  Both ceilings are printed; the binding one is the
    one whose time bound (work / peak) is longer, and `frac` is taken against it."""
    peaks = load_peaks()
    d = prof[dominant]
    b = before.get(dominant, {"launches": 0}) if before else {"launches": 0}
    if not (d["ms"] > 0 and d["timed"] > 0):
        return None
    secs = d["ms"] / 1e3
    tb, tf = d["timed_bytes"], d["timed_flops"]
    fp32 = mixed and dominant not in OUTER_FP64
    alu_peak = fp32_nominal_tflops(sm_count, peaks["sm_max_mhz"]) if fp32 else fp64_tflops
    alu_src = (f"nominal FP32: {sm_count} SMs x {FP32_FMA_PER_CLK_PER_SM} FMA/clk x 2 x {peaks['sm_max_mhz']:.0f} MHz"
               if fp32 else "measured FP64 FMA throughput of this GPU (tpmg_fp64_peak, best of 3 launches)")
    bw, fl = tb / secs / 1e9, tf / secs / 1e12
    ceilings = {
        "hbm": {"achieved": bw, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": bw / peaks["hbm_gbs"],
                "peak_source": f"{peaks['source']} HBM copy bandwidth (MEASURED_PEAKS.json)",
                "time_bound_us": 1e6 * tb / (peaks["hbm_gbs"] * 1e9)},
        "fp32" if fp32 else "fp64": {"achieved": fl, "peak": alu_peak, "unit": "TFLOP/s", "frac": fl / alu_peak,
                                     "peak_source": alu_src, "time_bound_us": 1e6 * tf / (alu_peak * 1e12)},
    }
    alu_key = "fp32" if fp32 else "fp64"
    hbm_bound = ceilings["hbm"]["time_bound_us"] >= ceilings[alu_key]["time_bound_us"]
    c = ceilings["hbm" if hbm_bound else alu_key]
    launches_step = (d["launches"] - b["launches"]) / max(1, steps)
    tr = traffic_of(dominant, workload)
    roof = {"bound": "hbm" if hbm_bound else "alu", "achieved": c["achieved"], "peak": c["peak"], "unit": c["unit"],
            "frac": c["frac"], "peak_source": c["peak_source"],
            "traffic": tr["bytes_per_launch"] if tr else None,
            "traffic_unit": "DRAM bytes (read + write) per launch, ncu, of the launches in traffic_scope",
            "traffic_scope": (tr["scope"] or "every launch of the class") if tr else None,
            "traffic_algorithmic_bytes": tr["algorithmic_per_launch"] if tr else None,
            "traffic_source": tr["source"] if tr else None,
            "algorithmic_bytes_per_launch": tb / d["timed"], "algorithmic_flops_per_launch": tf / d["timed"],
            "kernel": f"{dominant} ({'FP32/BF16' if fp32 else 'FP64'}){kernel_note}",
            "launches_per_step": launches_step, "avg_launch_us": 1e3 * d["ms"] / d["timed"],
            "timed_launches": d["timed"], "ceilings": ceilings,
            "hbm_frac_of_measured": ceilings["hbm"]["frac"],
            "share_of_step": (d["ms"] / d["timed"]) * launches_step / step_ms if step_ms else None}
    if tr:
        alg = tr["algorithmic_per_launch"] or roof["algorithmic_bytes_per_launch"]
        roof["traffic_over_algorithmic"] = tr["bytes_per_launch"] / alg
    return roof


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank number over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate_value(units_per_step: float, steps: int, world: int, local_ms: float) -> tuple[float, float]:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    t_ms = max_over_ranks(local_ms, world)
    return units_per_step * steps * world / (t_ms / 1e3), t_ms


# ----------------------------------------------------------------------------- oracle timing
def oracle_inputs(wl: dict, lib_path: str | None = None):
    import oracle
    from paper_1408_2981_gb300 import inputs

    o = oracle.Oracle(**{k: v for k, v in wl["params"].items() if k not in ("precision", "coeff_storage")},
                      lib_path=lib_path)
    if wl["rhs"] == "manufactured":
        g, v = o.grid(o.refinement), o.vertical()
        ustar = inputs.manufactured_solution(g["centre"], v["r"], wl["seed"])
        f = o.apply(ustar)
    else:
        f = inputs.uniform_pm1(wl["seed"], o.size())
    return o, f


def cpu_model() -> str:
    """The host CPU's name from /proc/cpuinfo (x86: model name; Arm: implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")), "?")
    part = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")), "?")
    return f"Arm implementer {impl} part {part}"


def time_oracle_threads(wl: dict, rtol: float, iters_hint: int | None):
    """The oracle built with OpenMP on all cores of this process's affinity mask (the
    same results bit for bit): a bounded sample like time_oracle's, about 5 s."""
    import oracle

    lib = oracle.build_openmp()
    if lib is None:
        return {"unavailable": "no OpenMP compiler"}
    cores = len(os.sched_getaffinity(0))
    oracle.threads(cores, lib_path=lib)
    v, sample, _ = time_oracle(wl, min_seconds=5.0, max_solves=3, rtol=rtol, iters_hint=iters_hint, lib_path=lib)
    return {"value": v, "unit": "unknowns/s", "cores": cores, "kind": "oracle (OpenMP over columns)",
            "cpu": cpu_model(), "sample": sample.replace("single thread", f"{cores} threads")}


def time_oracle(wl: dict, min_seconds: float, max_solves: int, rtol: float, iters_hint: int | None = None,
                lib_path: str | None = None):
    """Oracle solves of the workload on the host cores (setup excluded).

    Returns (unknowns per second of a full solve, sample text, oracle iterations).
    Up to ORACLE_FULL_SOLVE_MAX_UNKNOWNS the oracle runs whole solves (at least
    one, until min_seconds).  Beyond that a bounded sample: the oracle runs one
    PCG iteration (initial residual, V-cycle, operator, update), and a full
    solve is taken as that time x the iteration count of the GPU solve."""
    o, f = oracle_inputs(wl, lib_path)
    N = o.size()
    flexible = wl["params"].get("precision", 0) == 1
    if flexible:
        o.set_vcycle_bf16(True)
    if N <= ORACLE_FULL_SOLVE_MAX_UNKNOWNS:
        times, iters = [], None
        while len(times) < max_solves and (sum(times) < min_seconds or not times):
            t0 = time.perf_counter()
            res = o.pcg(f, rtol=rtol, max_iter=200, flexible=flexible)
            times.append(time.perf_counter() - t0)
            iters = res["iters"]
        return N * len(times) / sum(times), (f"{len(times)} full oracle solve(s) of the same workload, setup "
                                             f"excluded, {iters} iterations, single thread"), iters
    t0 = time.perf_counter()
    o.pcg(f, rtol=0.0, max_iter=1, flexible=flexible)
    t1 = time.perf_counter() - t0
    k = max(1, iters_hint or 1)
    return N / (t1 * k), (f"bounded sample: 1 oracle PCG iteration of the same workload ({t1:.1f} s, "
                          f"single thread), scaled to the GPU's {k} iterations"), None


# ----------------------------------------------------------------------------- arms
def run_reference(args, wl):
    """The oracle as the reference arm, on the machine's host cores (rank 0 only).
    Each step is one full oracle solve, or for workloads beyond
    ORACLE_FULL_SOLVE_MAX_UNKNOWNS the bounded one-iteration sample of time_oracle."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    values, sample, iters = [], "", None
    for _ in range(args.steps):
        v, sample, iters = time_oracle(wl, min_seconds=0.0, max_solves=1, rtol=args.rtol, iters_hint=args.iters_hint)
        values.append(v)
    N = WORKLOADS_N(wl)
    value = len(values) / sum(1.0 / v for v in values)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
            "steps": len(values), "warmup": 0, "ms_per_step": 1e3 * N / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": wl["text"], "n_unknowns": N},
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters": iters}
    print(json.dumps(line), flush=True)
    return 0


def WORKLOADS_N(wl: dict) -> int:
    p = wl["params"]
    return 20 * 4 ** p["refinement"] * p["n_r"]


def run_tpmg(args, wl):
    import numpy as np
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, inputs

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    s = binding.Solver(stream=stream, **wl["params"])
    N = s.N
    mixed = wl["params"].get("precision", 0) == 1
    m = s.export_mesh()
    if wl["rhs"] == "manufactured":
        ustar = torch.from_numpy(inputs.manufactured_solution(m["centres"], m["r_faces"], wl["seed"])).cuda()
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        s.apply_operator(ustar, f)
    else:
        f = torch.from_numpy(inputs.uniform_pm1(wl["seed"], N)).cuda()
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    fp64_tflops = binding.fp64_peak_tflops(stream)   # the FP64-pipe ceiling, measured here

    # warm-up; the last warm-up solve times every kernel class to find the dominant one
    for w in range(args.warmup):
        if w == args.warmup - 1:
            s.profile(classes=tuple(c for c in binding.KERNEL_CLASSES if c != "copy"))
        u.zero_()
        st, it, rel, _ = s.solve(f, u, rtol=args.rtol, max_iter=200)
    prof_all = s.profile_read()
    # device time per solve of each class: average timed launch x launches of the solve
    shares = {k: v["ms"] / v["timed"] * v["launches"] for k, v in prof_all.items() if v["timed"] > 0}
    dominant = max(shares, key=shares.get) if shares else "relax"

    # re-arm the tracer for the dominant class only; the untimed solve below
    # captures the V-cycle graph with an event pair around each launch of that class
    s.profile(classes=(dominant,))
    u.zero_()
    s.solve(f, u, rtol=args.rtol, max_iter=200)
    before = s.profile_read()

    # timed region: K solves, L2 flushed between steps
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    torch.cuda.nvtx.range_push("timed")   # for ncu --nvtx-include timed/
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        u.zero_()
        st, it, rel, _ = s.solve(f, u, rtol=args.rtol, max_iter=200)
        evs[k][1].record(stream)
        iters.append(it)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    local_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, t_ms = aggregate_value(N, args.steps, world, local_ms)
    prof = s.profile_read()
    gpu_launches = int(sum(prof[c]["launches"] - before[c]["launches"] for c in prof if c != "copy"))

    # end to end through the C ABI with host buffers: the steps' right-hand sides in
    # pinned host memory, their solutions read back into pinned host memory, every copy
    # inside the timed call (tpmg_solve_host_many overlaps step j's solve with the copies
    # of steps j - 1 and j + 1; the guess is zero, so only f is copied in)
    # every timed step, each with its own pinned solution array, up to 2 GB of them
    e2e_steps = max(1, min(args.steps, (2 << 30) // (8 * N)))
    f_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    f_host.copy_(f)
    u_hosts = [torch.zeros(N, dtype=torch.float64, pin_memory=True) for _ in range(e2e_steps)]
    fh, uhs = f_host.numpy(), [t.numpy() for t in u_hosts]
    # untimed kernels from here on, and one untimed call that captures the solve graphs
    # of the host-buffer path, as the warm-up solves did for the device path
    s.profile(classes=())
    s.solve_host_many([fh] * 2, uhs[:2] if e2e_steps >= 2 else [uhs[0], np.zeros(N)], rtol=args.rtol,
                      max_iter=200)
    barrier(world)
    t0 = time.perf_counter()
    _, e2e_iters, _, _ = s.solve_host_many([fh] * e2e_steps, uhs, rtol=args.rtol, max_iter=200)
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), world)
    e2e_value = N * e2e_steps * world / (e2e_ms / 1e3)
    # the same through one tpmg_solve_host call per step (copies of f, the zero guess and
    # u, none overlapped)
    uh = uhs[0]
    s.solve_host(fh, uh, rtol=args.rtol, max_iter=200)
    barrier(world)
    pc_s = 0.0
    for _ in range(e2e_steps):
        uh[:] = 0.0
        t0 = time.perf_counter()
        s.solve_host(fh, uh, rtol=args.rtol, max_iter=200)
        pc_s += time.perf_counter() - t0
    pc_ms = max_over_ranks(1e3 * pc_s, world)
    pc_value = N * e2e_steps * world / (pc_ms / 1e3)

    # roofline of the dominant kernel class: its launches in the timed region
    # carry event pairs (event-record nodes in the replayed graph hold the last
    # replay, i.e. the last timed step); the library counts each launch's
    # algorithmic bytes and flops
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    roof = roofline_of(prof, before, dominant, mixed, args.steps, local_ms / args.steps, fp64_tflops, sm_count,
                       args.workload)
    # aggregate algorithmic HBM rate of the whole solve (every class's bytes)
    peaks = load_peaks()
    tot_bytes = sum(v["bytes"] - before[c]["bytes"] for c, v in prof.items())
    hbm = {"achieved_gbs": tot_bytes / (local_ms / 1e3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
           "frac": tot_bytes / (local_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "source": peaks["source"],
           "algorithmic_bytes_per_step": tot_bytes / args.steps}

    cpu, cpu_threads = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v_o, sample, _ = time_oracle(wl, min_seconds=10.0, max_solves=3, rtol=args.rtol, iters_hint=iters[-1])
        cpu = {"value": v_o, "unit": "unknowns/s", "cores": 1, "kind": "oracle", "sample": sample, "cpu": cpu_model()}
        cpu_threads = time_oracle_threads(wl, args.rtol, iters[-1])
    extra = None
    tuning = [["warp", "cta64", "cta128", "cta256", "warp-deep"][v] if v >= 0 else "heuristic" for v, _ in s.tuning()]
    if rank == 0 and world == 1 and not args.no_extra_configs and args.workload == "81920x64":
        s.close()
        extra = run_extra_configs(args, stream, flush)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
                "config": {"workload": wl["text"], "n_unknowns": N, "parallelism": f"replicas{world}",
                           "l2": "flushed between steps (write of 2x L2 outside the timed events)",
                           "relax_kernel_per_level": tuning},
                "e2e": {"value": e2e_value, "unit": "unknowns/s", "h2d_bytes_per_step": 8 * N,
                        "d2h_bytes_per_step": 8 * N, "steps": e2e_steps, "ms": e2e_ms,
                        "iters": [int(i) for i in e2e_iters],
                        "call": "tpmg_solve_host_many (pinned host f in, u out; copies of neighbouring steps "
                                "overlap each solve)",
                        "note": "host clock around one call; its solves run without the roofline's CUDA-event "
                                "brackets and without an L2 flush between steps, which the device-timed value "
                                "carries, so it can exceed value",
                        "per_call": {"value": pc_value, "unit": "unknowns/s", "h2d_bytes_per_step": 2 * 8 * N,
                                     "d2h_bytes_per_step": 8 * N, "ms": pc_ms,
                                     "call": "tpmg_solve_host once per step (f and the guess in, u out)"}},
                "gpu_launches": gpu_launches, "roofline": roof, "hbm": hbm, "cpu_baseline": cpu,
                "cpu_baseline_threads": cpu_threads,
                "clocks": clk, "iters": iters[-1], "rel_resid": rel, "gpus_active": world,
                "fp64_peak_tflops_measured": fp64_tflops,
                "kernel_ms_per_step": {c: round(v, 4) for c, v in shares.items()},
                "other_configs": extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def solve_config(name: str, stream, flush, steps: int, warmup: int, rtol: float, rhs=None, keep_u=False):
    """Solves of one named workload from a zero guess (untimed set-up, `warmup`
    untimed solves, `steps` solves timed with CUDA events, L2 flushed between
    them): median ms, iterations, unknowns/s, the true relative residual."""
    import torch

    from paper_1408_2981_gb300 import binding, inputs

    wl = WORKLOADS[name]
    t0 = time.perf_counter()
    s = binding.Solver(stream=stream, **wl["params"])
    setup_s = time.perf_counter() - t0
    N = s.N
    if rhs is None:
        if wl["rhs"] == "manufactured":
            m = s.export_mesh()
            ustar = torch.from_numpy(inputs.manufactured_solution(m["centres"], m["r_faces"], wl["seed"])).cuda()
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            s.apply_operator(ustar, f)
        else:
            f = torch.from_numpy(inputs.uniform_pm1(wl["seed"], N)).cuda()
    else:
        f = rhs
    s.profile(classes=())
    res = time_solves(s, f, steps, warmup, rtol, 200, flush, stream)
    launches = launches_of(s)
    ms = statistics.median(r[0] for r in res)
    it, st = res[-1][1], res[-1][2]
    u = torch.zeros_like(f)
    s.solve(f, u, rtol=rtol, max_iter=200, raise_on_fail=False)
    au = torch.empty_like(u)
    s.apply_operator(u, au)
    true_rel = float(torch.linalg.norm(f - au) / torch.linalg.norm(f))
    out = {"workload": wl["text"], "n_unknowns": N, "status": binding.status_name(st), "iters": it,
           "ms_per_solve": ms, "unknowns_per_s": N / (ms / 1e3), "solves": len(res),
           "true_rel_resid": true_rel, "setup_s": setup_s, "gpu_launches": launches,
           "dtype": "f32+f64" if wl["params"].get("precision", 0) == 1 else "f64"}
    s.close()
    return out, f, (u if keep_u else None)


def run_extra_configs(args, stream, flush) -> dict:
    """The other configurations of the benchmark, each solved a few times in the same
    run (a few seconds each): the small case, the headline grid with a rough
    right-hand side (several iterations), refinement 7 x 128 in FP64 and in mixed
    precision (with the mixed solution's distance from the FP64 one), and the
    48-problem batch."""
    import torch

    out = {}
    out["1280x16"], _, _ = solve_config("1280x16", stream, flush, 20, 3, args.rtol)
    wl = dict(WORKLOADS["81920x64"], rhs="uniform", seed=2981010)
    WORKLOADS["_81920x64-uniform"] = dict(wl, text=WORKLOADS["81920x64"]["text"].replace(
        "manufactured spherical-harmonic x cosine solution, f = A u*", "RHS uniform[-1,1] (seed 2981010)"))
    out["81920x64-uniform"], _, _ = solve_config("_81920x64-uniform", stream, flush, 10, 3, args.rtol)
    del WORKLOADS["_81920x64-uniform"]
    out["327680x128"], f, u64 = solve_config("327680x128", stream, flush, 5, 3, args.rtol, keep_u=True)
    out["327680x128-mixed"], _, umx = solve_config("327680x128-mixed", stream, flush, 5, 3, args.rtol, rhs=f,
                                                   keep_u=True)
    mx = out["327680x128-mixed"]
    mx["speedup_vs_fp64"] = out["327680x128"]["ms_per_solve"] / mx["ms_per_solve"]
    mx["rel_diff_vs_fp64_solution"] = float(torch.linalg.norm(umx - u64) / torch.linalg.norm(u64))
    del f, u64, umx
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    b, wlist = batch_both(WORKLOADS["batch48"], stream, flush, steps=5, warmup=2, rtol=args.rtol)
    out["batch48"] = {k: b[k] for k in ("workload", "n_unknowns", "problems", "ms_per_step", "unknowns_per_s",
                                        "iters", "gpu_launches", "form")}
    out["batch48"]["other_form"] = wlist
    del b
    torch.cuda.empty_cache()
    return out


def batch_stats(wl, stream, flush, steps: int, warmup: int, rtol: float, form: str = "auto", groups: int = 0,
                problems=None) -> dict:
    """Set-up and timed runs of a batched workload (one tpmg_batch run per step).
    problems: (solvers, fs, us) to reuse, else created from the workload."""
    import torch

    from paper_1408_2981_gb300 import binding, inputs

    if problems is None:
        probs = batch_problems(wl["seed"], wl["batch"])
        solvers = [binding.Solver(stream=stream, **kw) for kw in probs]
        fs = [torch.from_numpy(inputs.uniform_pm1(wl["seed"] + 100 + j, s.N)).cuda() for j, s in enumerate(solvers)]
        us = [torch.zeros_like(f) for f in fs]
    else:
        solvers, fs, us = problems
    N = sum(s.N for s in solvers)
    batch = binding.Batch(solvers, fs, us, rtol=rtol, max_iter=200, form=form, groups=groups)

    def step():
        for u in us:
            u.zero_()
        return batch.run(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches, iters = 0, None
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        st, iters, rel, sts, nl = step()
        evs[k][1].record(stream)
        launches += nl
        if st != binding.TPMG_OK:
            raise RuntimeError(f"batch did not converge: statuses {sts.tolist()}")
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    out = {"workload": wl["text"], "n_unknowns": N, "problems": len(solvers), "ms_per_step": ms / steps,
           "unknowns_per_s": N * steps / (ms / 1e3), "iters": [int(i) for i in iters], "gpu_launches": launches,
           "local_ms": ms, "form": batch.form, "groups": groups, "batch": batch, "solvers": solvers, "fs": fs,
           "us": us, "step": step}
    return out


BATCH_WORKLIST_GROUPS = 16   # the work-list form's root branches in the batch lines (measured best of 1..48)


def batch_both(wl, stream, flush, steps: int, warmup: int, rtol: float) -> tuple:
    """The batch in its automatic form, then in the work-list form on the same problems."""
    import torch

    a = batch_stats(wl, stream, flush, steps, warmup, rtol)   # stays open for the caller (end-to-end runs)
    torch.cuda.synchronize()
    w = batch_stats(wl, stream, flush, steps, warmup, rtol, form="worklist", groups=BATCH_WORKLIST_GROUPS,
                    problems=(a["solvers"], a["fs"], a["us"]))
    w["batch"].close()
    torch.cuda.synchronize()
    other = {k: w[k] for k in ("form", "groups", "ms_per_step", "unknowns_per_s", "gpu_launches")}
    return a, other


def run_batch(args, wl):
    """The batched form: one step = one tpmg_batch run of all problems (device-side
    loops, one graph launch).  value = unknowns of all problems / device time."""
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, inputs

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    b, wlist = batch_both(wl, stream, flush, args.steps, args.warmup, args.rtol)
    clk = clocks.stop()
    fs, us, step, N, solvers, launches, iters = b["fs"], b["us"], b["step"], b["n_unknowns"], b["solvers"], \
        b["gpu_launches"], b["iters"]
    value, t_ms = aggregate_value(N, args.steps, world, b["local_ms"])

    # end to end: right-hand sides from pinned host memory and solutions back, inside the timed region
    f_host = [torch.empty(f.numel(), dtype=torch.float64, pin_memory=True).copy_(f) for f in fs]
    u_host = [torch.empty(f.numel(), dtype=torch.float64, pin_memory=True) for f in fs]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        for f, fh in zip(fs, f_host):
            f.copy_(fh, non_blocking=True)
        step()
        for u, uh in zip(us, u_host):
            uh.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), world)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": wl["text"], "n_unknowns": N, "problems": len(solvers),
                           "parallelism": f"replicas{world}",
                           "l2": "flushed between steps (write of 2x L2 outside the timed events)"},
                "e2e": {"value": N * e2e_steps * world / (e2e_ms / 1e3), "unit": "unknowns/s",
                        "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
                "gpu_launches": launches, "roofline": None, "cpu_baseline": None, "clocks": clk,
                "iters": [int(i) for i in iters], "form": b["form"], "other_form": wlist, "gpus_active": world,
                "note": "the loops run on the device, so kernels carry no event pairs: no per-kernel roofline here"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_learned(args, wl):
    """The learned form: training data from plain solves, training of both
    networks (outside the timed region, reported), then K timed learned solves
    of held-out right-hand sides beside K plain mixed-precision solves of the
    same right-hand sides (same context, same stop test ||r|| <= rtol ||f||)."""
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, learned

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    cfg = dict(wl["learned"])
    if args.pairs:
        cfg["pairs"] = args.pairs
    if args.levels:   # a shallower hierarchy: the coarsest level is then horizontally coupled
        wl = dict(wl, params=dict(wl["params"], n_levels=args.levels),
                  text=wl["text"] + f"; {args.levels} multigrid levels")
    seed = wl["seed"] + 7919 * rank
    t_setup = time.perf_counter()
    data_solver = binding.Solver(stream=stream, graphs=0, **wl["params"])
    fields = learned.SmoothFields(data_solver, l_max=cfg["l_max"])
    data = learned.generate(data_solver, fields, n_pairs=cfg["pairs"], seed=seed + 1000,
                            cells_per_pair=cfg["cells_per_pair"], coarse_per_pair=cfg["coarse_per_pair"])
    data_solver.close()
    nets, train_out = {}, {}
    for name, role, x, t in (("warm", binding.TPMG_NET_WARM, data["xw"], data["tw"]),
                             ("coarse", binding.TPMG_NET_COARSE, data["xc"], data["tc"])):
        net = binding.Net(wl["params"]["n_r"], cfg["hidden"], stream=stream)
        net.set_params(learned.init_params(net.sizes, seed + 11 * role + 3))
        out = learned.train(net, x, t, steps=cfg["train_steps"], seed=seed + 13 * role + 5, batch=cfg["batch"],
                            lr=cfg["lr"])
        nets[name] = net
        train_out[name] = {"rows": int(x.shape[0]), "loss_first": out["history"][0][1], "loss_final": out["final"],
                           "target_mean_square": float(t.double().pow(2).mean()), "seconds": out["seconds"]}
    del data
    torch.cuda.empty_cache()
    s = binding.Solver(stream=stream, **wl["params"])
    N = s.N
    s.attach_net(binding.TPMG_NET_WARM, nets["warm"])
    s.attach_net(binding.TPMG_NET_COARSE, nets["coarse"])
    setup_s = time.perf_counter() - t_setup
    fs = [fields.field(seed + 10_000_000 + k) for k in range(args.steps)]   # held out
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    # one right-hand-side buffer: the solve graphs are captured for fixed vectors
    f_buf = torch.empty(N, dtype=torch.float64, device="cuda")
    for w in range(args.warmup):
        f_buf.copy_(fs[w % len(fs)])
        u.zero_()
        s.solve_learned(f_buf, u, rtol=args.rtol, max_iter=200)
        u.zero_()
        s.solve(f_buf, u, rtol=args.rtol, max_iter=200)
    torch.cuda.synchronize()

    def timed(learned_arm: bool):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in fs]
        its, rels, infos, fbs, launches = [], [], [], [], 0
        barrier(world)
        torch.cuda.synchronize()
        for k, f in enumerate(fs):
            f_buf.copy_(f)
            flush.fill_(float(k))
            evs[k][0].record(stream)
            u.zero_()
            if learned_arm:
                st, it, rel, info, fb, nl = s.solve_learned(f_buf, u, rtol=args.rtol, max_iter=200)
                infos.append(info)
                fbs.append(fb)
                launches += nl
            else:
                st, it, rel, _ = s.solve(f_buf, u, rtol=args.rtol, max_iter=200)
            evs[k][1].record(stream)
            its.append(it)
            rels.append(rel)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, its, rels, infos, fbs, launches

    def attach(coarse, warm):
        s.attach_net(binding.TPMG_NET_COARSE, coarse)
        s.attach_net(binding.TPMG_NET_WARM, warm)
        f_buf.copy_(fs[0])
        u.zero_()
        s.solve_learned(f_buf, u, rtol=args.rtol, max_iter=200)   # capture the solve graph, untimed

    # the learned form (both networks) is the headline arm; each network alone and
    # plain TPMG-PCG are timed on the same right-hand sides
    arms = {}
    for name, coarse, warm in (("warm", None, nets["warm"]), ("coarse", nets["coarse"], None)):
        attach(coarse, warm)
        ms_a, its_a, _, infos_a, fbs_a, _ = timed(True)
        arms[name] = {"value": aggregate_value(N, len(fs), world, ms_a)[0], "ms_per_step": ms_a / len(fs),
                      "iters": its_a, "info": infos_a, "fallback_iters": fbs_a}
    attach(nets["coarse"], nets["warm"])
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")   # the learned arm's timed region (for ncu --nvtx-include timed/)
    ms_l, its_l, rels_l, infos, fbs, launches = timed(True)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    ms_p, its_p, rels_p, _, _, _ = timed(False)
    value, t_ms = aggregate_value(N, len(fs), world, ms_l)
    plain_value, _ = aggregate_value(N, len(fs), world, ms_p)

    # initial residual of the warm start alone (network + one line relaxation), held-out f
    r0s = []
    s.attach_net(binding.TPMG_NET_COARSE, None)
    for f in fs[:3]:
        f_buf.copy_(f)
        u.zero_()
        s.solve_learned(f_buf, u, rtol=1.0, max_iter=1)
        r = torch.empty_like(f)
        s.apply_operator(u, r)
        r0s.append(float(torch.linalg.norm(f - r) / torch.linalg.norm(f)))
    s.attach_net(binding.TPMG_NET_COARSE, nets["coarse"])

    # the warm-start prediction over every fine column (point values, scale,
    # features, the fused tensor-core network), timed alone
    up = torch.empty_like(u)
    s.net_predict(binding.TPMG_NET_WARM, fs[0], up)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("predict")   # ncu --nvtx-include predict/
    for _ in range(5):
        s.net_predict(binding.TPMG_NET_WARM, fs[0], up)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 5
    sizes = nets["warm"].sizes
    fwd_flops = 2.0 * s.n_cells * sum(i * o for i, o in zip(sizes[:-1], sizes[1:]))

    # end to end with host buffers: f in, learned solve, u out
    f_host = torch.empty(N, dtype=torch.float64, pin_memory=True).copy_(fs[0])
    u_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    f_dev = f_buf
    f_dev.copy_(fs[0])
    u.zero_()
    s.solve_learned(f_dev, u, rtol=args.rtol, max_iter=200)   # re-capture after the re-attachment, untimed
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(len(fs), 5))
    for _ in range(e2e_steps):
        f_dev.copy_(f_host, non_blocking=True)
        u.zero_()
        s.solve_learned(f_dev, u, rtol=args.rtol, max_iter=200)
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), world)

    # kernel classes of the learned solve: with classes timed it runs kernel by
    # kernel from the host (the same kernels in the same order), each launch
    # bracketed by CUDA events; roofline of the dominant class from it
    peaks = load_peaks()
    s.profile(classes=tuple(c for c in binding.KERNEL_CLASSES if c != "copy"))
    f_buf.copy_(fs[0])
    u.zero_()
    torch.cuda.nvtx.range_push("learned_solve_kernels")   # direct launches: ncu --nvtx-include learned_solve_kernels/
    s.solve_learned(f_buf, u, rtol=args.rtol, max_iter=200)
    torch.cuda.nvtx.range_pop()
    prof = s.profile_read()
    s.profile(classes=())
    shares = {k: v["ms"] for k, v in prof.items() if v["timed"] > 0}
    dominant = max(shares, key=shares.get)
    roof = roofline_of(prof, None, dominant, True, 1, None, binding.fp64_peak_tflops(stream),
                       torch.cuda.get_device_properties(local).multi_processor_count, args.workload,
                       ", from one learned solve run kernel by kernel with every class timed")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v_o, sample, _ = time_oracle(dict(wl, rhs="uniform"), min_seconds=10.0, max_solves=1, rtol=args.rtol,
                                     iters_hint=its_p[-1])
        cpu = {"value": v_o, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
               "sample": sample + " (plain oracle PCG; the per-iteration cost does not depend on the RHS values)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": len(fs),
                "warmup": args.warmup, "ms_per_step": t_ms / len(fs), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64+bf16w", "data": "synthetic",
                "config": {"workload": wl["text"], "n_unknowns": N, "parallelism": f"replicas{world}",
                           "pairs": cfg["pairs"], "stop": "||r|| <= rtol ||f||",
                           "l2": "flushed between steps (write of 2x L2 outside the timed events)"},
                "e2e": {"value": N * e2e_steps * world / (e2e_ms / 1e3), "unit": "unknowns/s",
                        "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "learned": {"iters": its_l, "rel_resid": rels_l, "info": infos, "fallback_iters": fbs,
                            "warm_start_rel_resid": r0s},
                "plain": {"value": plain_value, "iters": its_p, "rel_resid": rels_p, "ms_per_step": ms_p / len(fs)},
                "arms": arms,
                "speedup_vs_plain": value / plain_value,
                "training": train_out, "setup_seconds": setup_s,
                "warm_start_prediction": {"rows": s.n_cells, "ms": fwd_ms,
                                          "network_tflops_over_whole_call": fwd_flops / (fwd_ms / 1e3) / 1e12},
                "kernel_ms_per_step": {c: round(v, 4) for c, v in shares.items()},
                "net_launches_per_step": prof["net"]["launches"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def time_solves(s, f, steps: int, warmup: int, rtol: float, max_iter: int, flush, stream):
    """Device time (ms) and iterations of `steps` solves from a zero guess, L2 flushed
    between solves outside the events, after `warmup` untimed solves."""
    import torch

    u = torch.zeros_like(f)
    for _ in range(warmup):
        u.zero_()
        s.solve(f, u, rtol=rtol, max_iter=max_iter, raise_on_fail=False)
    out = []
    for k in range(steps):
        flush.fill_(float(k))
        u.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, it, rel, _ = s.solve(f, u, rtol=rtol, max_iter=max_iter, raise_on_fail=False)
        b.record(stream)
        b.synchronize()
        out.append((a.elapsed_time(b), it, st, rel))
    return out


def launches_of(s) -> int:
    prof = s.profile_read()
    return int(sum(v["launches"] for c, v in prof.items() if c != "copy"))


def study_line(args, wl, metric, value, unit, higher, dtype, extra, clk, launches, world):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": higher, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": wl["text"], "parallelism": f"replicas{world}",
                       "l2": "flushed between solves (write of 2x L2 outside the timed events)"},
            "e2e": None, "gpu_launches": launches, "roofline": None, "cpu_baseline": None, "clocks": clk}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_nr_sweep(args, wl):
    """Sec. 5.1, eq. nzDependency: time per iteration against n_r, fitted by least
    squares to t = C + q n_r; C / t is the share of the per-column work that does
    not grow with n_r (indirect addressing, launches, the coarse levels)."""
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    variants = {"TPMG^fac FP64": dict(),
                "TPMG^full FP64": dict(coeff_storage=binding.TPMG_COEFF_FULL),
                "TPMG^full mixed": dict(MIXED)}
    K = wl["iters"]
    points, launches = [], 0
    clocks = ClockSampler(local)
    clocks.start()
    for n_r in wl["n_r"]:
        for name, extra in variants.items():
            s = binding.Solver(stream=stream, refinement=wl["refinement"], n_levels=6, n_r=n_r, grading=1.05,
                               courant_c=80.0, nu_pre=2, nu_post=2, nu_coarse=1, **extra)
            f = torch.from_numpy(inputs.uniform_pm1(wl["seed"], s.N)).cuda()
            s.profile(classes=())
            res = time_solves(s, f, args.steps, args.warmup, 0.0, K, flush, stream)
            launches += launches_of(s)
            assert all(it == K for _, it, _, _ in res), res
            ms = statistics.median(r[0] for r in res)
            points.append({"n_r": n_r, "variant": name, "t_iter_ms": ms / K, "unknowns": s.N,
                           "ns_per_unknown_iter": 1e6 * ms / K / s.N})
            del s
            torch.cuda.synchronize()
    clk = clocks.stop()
    fits = {}
    for name in variants:
        xs = np.array([p["n_r"] for p in points if p["variant"] == name], dtype=np.float64)
        ys = np.array([p["t_iter_ms"] for p in points if p["variant"] == name])
        q, c = np.polyfit(xs, ys, 1)
        pred = c + q * xs
        r2 = 1.0 - float(((ys - pred) ** 2).sum() / ((ys - ys.mean()) ** 2).sum())
        fits[name] = {"C_ms": c, "q_ms_per_level": q, "r2": r2,
                      "overhead_at_128": c / (c + 128 * q), "overhead_at_256": c / (c + 256 * q)}
    if rank == 0:
        study_line(args, wl, "share of the time per iteration that does not grow with n_r, at n_r = 128 "
                   "(Sec. 5.1: C / (C + 128 q), TPMG^fac FP64)", fits["TPMG^fac FP64"]["overhead_at_128"],
                   "fraction", False, "f64", {"points": points, "fit": fits, "iters_per_solve": K}, clk, launches,
                   world)
    return 0


def run_balanced_flow(args, wl):
    """Sec. 5, Figs. 3-4 and Table 1's preconditioners: iterations, time per iteration
    and total solve time against the buoyancy frequency for TPMG^fac, TPMG^partial and
    TPMG^full (FP64) and TPMG^full in mixed precision, each preconditioning the full
    operator (with vertical advection: Richardson and BiCGStab, the paper's two)."""
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    precs = {"TPMG^fac FP64": dict(),
             "TPMG^partial FP64": dict(coeff_storage=binding.TPMG_COEFF_PARTIAL),
             "TPMG^full FP64": dict(coeff_storage=binding.TPMG_COEFF_FULL),
             "TPMG^full mixed": dict(MIXED)}
    outers = {"Richardson": binding.TPMG_OUTER_RICHARDSON, "BiCGStab": binding.TPMG_OUTER_BICGSTAB}
    if not wl.get("advection"):   # CG needs the symmetric operator
        outers["CG"] = binding.TPMG_OUTER_CG
    kw = dict(refinement=wl["refinement"], n_levels=6, n_r=wl["n_r"], grading=1.05, courant_c=8.0,
              nu_pre=2, nu_post=2, nu_coarse=1)
    probe = binding.Solver(stream=stream, **kw)
    mesh = probe.export_mesh()
    N = probe.N
    del probe
    f = torch.from_numpy(inputs.uniform_pm1(wl["seed"], N)).cuda()
    rows, launches = [], 0
    steps = max(1, min(args.steps, 5))
    clocks = ClockSampler(local)
    clocks.start()
    for n_freq in wl["n_freq"]:
        n_freq = 9.81 / math.sqrt(1005.0 * 273.0) if n_freq is None else n_freq
        outer_prof, fac_prof, eps = inputs.balanced_flow(mesh["centres"], mesh["r_faces"], n_freq,
                                                         advection=wl.get("advection", False))
        for pname, pextra in precs.items():
            for oname, outer in outers.items():
                s = binding.Solver(stream=stream, profiles=fac_prof, outer=outer, **kw, **pextra)
                s.set_outer_profiles(**outer_prof)
                s.profile(classes=())
                res = time_solves(s, f, steps, args.warmup, 1e-5, 300, flush, stream)
                launches += launches_of(s)
                ms = statistics.median(r[0] for r in res)
                it, st, rel = res[-1][1], res[-1][2], res[-1][3]
                rows.append({"N": n_freq, "eps": round(eps, 3), "preconditioner": pname, "outer": oname,
                             "status": st, "iters": it, "rel_resid": rel, "t_solve_ms": ms,
                             "t_iter_ms": ms / max(it, 1)})
                del s
                torch.cuda.synchronize()
    clk = clocks.stop()
    ok = [r for r in rows if r["status"] == 0]

    def t_iter(prec, outer, eps_i=0):
        e = sorted({r["eps"] for r in rows})[eps_i]
        return next(r["t_iter_ms"] for r in rows if r["preconditioner"] == prec and r["outer"] == outer
                    and r["eps"] == e)

    ratios = {o: {"full/fac": t_iter("TPMG^full FP64", o) / t_iter("TPMG^fac FP64", o),
                  "partial/fac": t_iter("TPMG^partial FP64", o) / t_iter("TPMG^fac FP64", o),
                  "full-mixed/fac": t_iter("TPMG^full mixed", o) / t_iter("TPMG^fac FP64", o)}
              for o in ("Richardson", "BiCGStab")}
    eps_max = max(r["eps"] for r in rows)
    best = min((r for r in ok if r["eps"] == eps_max), key=lambda r: r["t_solve_ms"])
    if rank == 0:
        study_line(args, wl, "time to a 1e-5 residual reduction at the largest eps (Sec. 5, Fig. 4), fastest "
                   "preconditioner and outer iteration", best["t_solve_ms"], "ms", False, "f64 / f32+f64",
                   {"best": best, "t_iter_ratio_eps0": ratios, "table": rows, "unknowns": N}, clk, launches,
                   world)
    return 0


def run_prolongation(args, wl):
    """Sec. 5's linear prolongation against P = R^T: iterations, time per iteration and
    solve time with Richardson and BiCGStab (CG needs the symmetric P = R^T)."""
    import torch

    from paper_1408_2981_gb300 import binding, build as _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    rows, launches, f = [], 0, None
    clocks = ClockSampler(local)
    clocks.start()
    for prec_name, prec in (("FP64", dict()), ("mixed", dict(MIXED))):
        for oname, outer in (("Richardson", binding.TPMG_OUTER_RICHARDSON), ("BiCGStab", binding.TPMG_OUTER_BICGSTAB)):
            for pname, prol in (("constant", binding.TPMG_PROLONG_CONSTANT), ("linear", binding.TPMG_PROLONG_LINEAR)):
                s = binding.Solver(stream=stream, outer=outer, prolongation=prol, **wl["params"], **prec)
                if f is None:
                    f = torch.from_numpy(inputs.uniform_pm1(wl["seed"], s.N)).cuda()
                s.profile(classes=())
                res = time_solves(s, f, max(1, min(args.steps, 10)), args.warmup, 1e-5, 200, flush, stream)
                launches += launches_of(s)
                ms = statistics.median(r[0] for r in res)
                it, st = res[-1][1], res[-1][2]
                rows.append({"precision": prec_name, "outer": oname, "prolongation": pname, "status": st, "iters": it,
                             "t_solve_ms": ms, "t_iter_ms": ms / max(it, 1), "unknowns_per_s": s.N / (ms / 1e3)})
                del s
                torch.cuda.synchronize()
    clk = clocks.stop()
    best = min((r for r in rows if r["status"] == 0), key=lambda r: r["t_solve_ms"])
    if rank == 0:
        study_line(args, wl, "unknowns/sec to 1e-5 with the fastest prolongation / outer iteration / precision "
                   "(Sec. 5 linear prolongation against P = R^T)", best["unknowns_per_s"], "unknowns/s", True,
                   "f64 / f32+f64", {"best": best, "table": rows}, clk, launches, world)
    return 0


def free_port() -> int:
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def replica_command(argv: list, n: int, port: int) -> list:
    """The torchrun command line that starts n ranks of this bench on one node, one
    per GPU, each solving its own replica of the workload."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


def launcher_check() -> int:
    """Each rank reports how it was started (after a gloo barrier); no GPU is used."""
    world, rank, local = dist_env()
    line = json.dumps({"launcher_check": True, "rank": rank, "world": world, "local_rank": local})
    if world <= 1:
        print(line, flush=True)
        return 0
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method="env://")
    for r in range(world):   # one rank at a time, so that the lines do not interleave
        if r == rank:
            print(line, flush=True)
        dist.barrier()
    dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["tpmg", "reference"], default="tpmg")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="81920x64")
    ap.add_argument("--rtol", type=float, default=1e-5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="headline workload: skip the other configurations (small case, refinement 7, batch)")
    ap.add_argument("--pairs", type=int, default=None, help="learned workload: training pairs (default 2000)")
    ap.add_argument("--levels", type=int, default=None,
                    help="learned workload: multigrid levels (default 6; the coarse network replaces the coarsest "
                         "level's solve)")
    ap.add_argument("--iters-hint", type=int, default=None,
                    help="reference arm on workloads sampled by one iteration: iterations of a full solve")
    ap.add_argument("--no-autotune", action="store_true",
                    help="single-problem workloads: the fixed kernel heuristic instead of the autotuner (for "
                         "ncu launch lists, under which the autotuner's timings are distorted)")
    ap.add_argument("--launcher-check", action="store_true",
                    help="start the ranks as --gpus asks, print each rank's view of the launch and exit (no GPU)")
    argv = list(sys.argv[1:] if argv is None else argv)
    args = ap.parse_args(argv)
    if args.warmup < 1 and args.impl == "tpmg":
        ap.error("--warmup must be >= 1")
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    world_env = os.environ.get("WORLD_SIZE")
    if world_env is None and args.gpus > 1:
        # not started by torchrun: start the N replica ranks here (one process per GPU)
        return subprocess.call(replica_command(argv, args.gpus, free_port()))
    if world_env is not None and int(world_env) != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world_env}: start one rank per GPU", file=sys.stderr)
        return 2
    if args.launcher_check:
        return launcher_check()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        if "study" in wl:
            print(json.dumps({"impl": "reference", "unavailable": "a study of the GPU kernels' time per iteration "
                              "(no oracle arm); the oracle arm times the single-problem workloads"}))
            return 0
        if "batch" in wl:
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle arm: its "
                              "problems are each an oracle solve of the single-problem workloads"}))
            return 0
        return run_reference(args, wl)
    if "study" in wl:
        return {"nr_sweep": run_nr_sweep, "balanced_flow": run_balanced_flow,
                "prolongation": run_prolongation}[wl["study"]](args, wl)
    if "batch" in wl:
        return run_batch(args, wl)
    if "learned" in wl:
        return run_learned(args, wl)
    if args.no_autotune:
        wl = dict(wl, params=dict(wl["params"], autotune=0))
    return run_tpmg(args, wl)


if __name__ == "__main__":
    sys.exit(main())
