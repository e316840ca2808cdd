#!/usr/bin/env python3
"""Benchmark: solves/sec of ML(n)BiCGStab (plain FP64) on the 3-D 7-point
log-normal convection-diffusion system, 128^3 unknowns, to relative
residual 1e-10.

One "step" is one complete solve from x0 = 0 (all iterations of the method,
each an SpMV fused with shadow inner products plus the fused recurrence
passes) through the C ABI, with b and x already in device memory.  The
matrix (175 MB) and the solver state (> 300 MB) are larger than the 129 MB
L2 cache, so no flush is needed between steps.

Arms
  default           the CUDA library (one persistent kernel per solve)
  --impl reference  the CPU oracle on the host cores, on a bounded sample
                    of iterations of the same workload, converted to
                    solves/sec with the iteration count of a full solve

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 through
torch.distributed.run, one rank per GPU, each rank solving its own replica
(independent systems: weak scaling, no collective on the data path).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/sec and SpMV+dot HBM GB/s (% of peak) at rel. residual 1e-10"
UNIT = "solves/s"

# Workloads (the benchmark line uses DEFAULT).  `iters` is the iteration
# count of one full solve on the GPU path (measured: 20,752 for the
# headline system, one restart included), used only to convert the
# reference arm's per-iteration sample into solves/sec.
WORKLOADS = {
    "cd3d128_n4_fp64": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, iters=20752,
                            precision=0),
    "cd3d128_n4_refined": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=1),
    # the largest single-GPU workload: measured with its own roofline,
    # CPU-baseline and end-to-end figures
    "helmholtz_n8_c128": dict(kind="helmholtz", n=8, tol=1e-10, maxit=40000, precision=0, full=True),
    "helmholtz_n8_c64_refined": dict(kind="helmholtz", n=8, tol=1e-10, maxit=40000, precision=1),
    # the omega guard of Eq. 5.1 (kappa = 0.7, the value suggested by
    # Sleijpen & van der Vorst) on the same complex system
    "helmholtz_n8_c128_kappa07": dict(kind="helmholtz", n=8, tol=1e-10, maxit=40000, precision=0,
                                      kappa=0.7),
    # Jacobi right preconditioning (Algorithm 7.1, M = diag(A)) on the
    # headline system (not in the default list: on this family it converges
    # about 4x slower than M = I, in the oracle as well)
    "cd3d128_n4_fp64_jacobi": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=0,
                                   precond=1),
    # ILU(0) right preconditioning (Algorithm 7.1 with M = L U, the
    # preconditioner of the paper's experiments, §5) on the headline system
    # and on the batch (one CTA per system, CTA barriers between levels)
    "cd3d128_n4_fp64_ilu0": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=0, precond=2),
    "batch512_n4_fp64_ilu0": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=0, precond=2),
    "reservoir_n8_fp64": dict(kind="reservoir", n=8, tol=1e-10, maxit=20000, precision=0),
    # the same 3x3-block reservoir system with ILU(0): a handful of
    # iterations where M = I needs tens of thousands
    "reservoir_n8_fp64_ilu0": dict(kind="reservoir", n=8, tol=1e-10, maxit=20000, precision=0, precond=2),
    "batch512_n4_fp64": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=0),
    # the autotuner on a mid-size system (default configuration vs tuned)
    "tune_cd2d256": dict(kind="tune", m=256, n=4, tol=1e-10, maxit=40000, precision=0),
    # a sequence of right-hand sides with n chosen by the rule of §5
    # (n0 = 4, step 2, n in [1, 16]) against the same sequence at fixed n = 4
    "sequence8_cd3d64": dict(kind="sequence", m=64, n=16, count=8, n0=4, step=2, n_min=1, n_max=16,
                             tol=1e-10, maxit=40000, precision=0),
    "batch512_n4_refined": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=1),
    # FP32-inner / FP64-refined with the FP32 ILU(0) factors in the inner
    # solve, against the FP64 solve with the same preconditioner
    "cd3d128_n4_refined_ilu0": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=1, precond=2),
    "reservoir_n8_refined_ilu0": dict(kind="reservoir", n=8, tol=1e-10, maxit=20000, precision=1, precond=2),
    "batch512_n4_refined_ilu0": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=1, precond=2),
    # ILU(0) in a multicolour order (precond 3): one level per colour in the
    # triangular solves instead of one per wavefront; a different (weaker)
    # preconditioner than the paper's natural-order ILU(0)
    "cd3d128_n4_fp64_ilu0mc": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=0, precond=3),
    "cd3d128_n4_refined_ilu0mc": dict(kind="cd3d", m=128, n=4, tol=1e-10, maxit=40000, precision=1, precond=3),
    "reservoir_n8_fp64_ilu0mc": dict(kind="reservoir", n=8, tol=1e-10, maxit=20000, precision=0, precond=3),
    "reservoir_n8_refined_ilu0mc": dict(kind="reservoir", n=8, tol=1e-10, maxit=20000, precision=1, precond=3),
    "batch512_n4_fp64_ilu0mc": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=0, precond=3),
    "helmholtz_n8_c128_ilu0mc": dict(kind="helmholtz", n=8, tol=1e-10, maxit=40000, precision=0, precond=3),
    # the fused product y = A x, d = Q^H y alone (mlbicgstab_spmv_qdot) on
    # the headline matrix, for n = 1, 4, 16 shadow vectors
    "spmv_qdot_cd3d128": dict(kind="spmv_qdot", m=128, n=4, ns=(1, 4, 8, 16), calls=50),
    # the batch after mlbicgstab_autotune_batch (tile cap per size class;
    # tuning is setup, not timed), against batch512_n4_fp64 (default caps)
    "batch512_n4_fp64_tuned": dict(kind="batch", n=4, tol=1e-10, maxit=20000, precision=0, tune=True),
}
for _n in (1, 8, 16):
    WORKLOADS[f"cd3d128_n{_n}_fp64"] = dict(kind="cd3d", m=128, n=_n, tol=1e-10, maxit=60000,
                                           precision=0)
DEFAULT = "cd3d128_n4_fp64"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the solve
# kernel on the headline workload, from one ncu capture of a 300-iteration
# launch of the current kernel: 136.46 GB + 30.39 GB.  Traffic grows in
# proportion to the iterations, so a full launch is scaled by its
# iteration count.  Set to None whenever the kernel changes until it is
# captured again.
NCU_DRAM_BYTES_PER_ITER = (136.456225e9 + 30.393382e9) / 300
VARIANTS = ["spmv_qdot_cd3d128", "cd3d128_n1_fp64", "cd3d128_n8_fp64", "cd3d128_n16_fp64",
            "cd3d128_n4_fp64_ilu0", "cd3d128_n4_refined_ilu0", "cd3d128_n4_fp64_ilu0mc", "cd3d128_n4_refined_ilu0mc",
            "reservoir_n8_fp64", "reservoir_n8_fp64_ilu0", "reservoir_n8_refined_ilu0",
            "reservoir_n8_fp64_ilu0mc", "reservoir_n8_refined_ilu0mc",
            "batch512_n4_fp64", "batch512_n4_fp64_tuned", "batch512_n4_fp64_ilu0", "batch512_n4_fp64_ilu0mc",
            "batch512_n4_refined", "batch512_n4_refined_ilu0",
            "helmholtz_n8_c128", "helmholtz_n8_c128_kappa07", "helmholtz_n8_c128_ilu0mc", "helmholtz_n8_c64_refined",
            "sequence8_cd3d64", "tune_cd2d256"]
# (variant, the variant it is compared with): refined against FP64 with the
# same preconditioner, preconditioned against unpreconditioned, the omega
# guard against kappa = 0.  A speedup is reported only when both sides
# converged (every solve flag 0 with true relative residual below tol).
PAIRS = [("batch512_n4_fp64_tuned", "batch512_n4_fp64", "speedup_vs_default"),
         ("cd3d128_n4_refined_ilu0", "cd3d128_n4_fp64_ilu0", "speedup_vs_fp64"),
         ("cd3d128_n4_refined_ilu0mc", "cd3d128_n4_fp64_ilu0mc", "speedup_vs_fp64"),
         ("reservoir_n8_refined_ilu0mc", "reservoir_n8_fp64_ilu0mc", "speedup_vs_fp64"),
         ("reservoir_n8_fp64_ilu0mc", "reservoir_n8_fp64", "speedup_vs_unpreconditioned"),
         ("batch512_n4_fp64_ilu0mc", "batch512_n4_fp64", "speedup_vs_unpreconditioned"),
         ("helmholtz_n8_c128_ilu0mc", "helmholtz_n8_c128", "speedup_vs_unpreconditioned"),
         ("reservoir_n8_refined_ilu0", "reservoir_n8_fp64_ilu0", "speedup_vs_fp64"),
         ("batch512_n4_refined_ilu0", "batch512_n4_fp64_ilu0", "speedup_vs_fp64"),
         ("batch512_n4_refined", "batch512_n4_fp64", "speedup_vs_fp64"),
         ("helmholtz_n8_c64_refined", "helmholtz_n8_c128", "speedup_vs_fp64"),
         ("cd3d128_n4_refined", "cd3d128_n4_fp64", "speedup_vs_fp64"),
         ("reservoir_n8_fp64_ilu0", "reservoir_n8_fp64", "speedup_vs_unpreconditioned"),
         ("batch512_n4_fp64_ilu0", "batch512_n4_fp64", "speedup_vs_unpreconditioned"),
         ("helmholtz_n8_c128_kappa07", "helmholtz_n8_c128", "speedup_vs_kappa0")]


def _load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _make_inputs(wl):
    from paper_1106_3678_gb300 import workloads as W
    A = W.cd3d_lognormal(wl["m"])
    b = W.uniform_rhs(A.n_rows, seed=2)
    return A, b


def _make_variant_inputs(wl):
    """(list of (A, AH or None, b)) for a variant workload."""
    from paper_1106_3678_gb300 import workloads as W
    kind = wl["kind"]
    if kind == "cd3d":
        A, b = _make_inputs(wl)
        return [(A, None, b)]
    if kind == "helmholtz":
        A = W.helmholtz3d_c()
        return [(A, W.conj_transpose(A), W.row_sums(A))]
    if kind == "reservoir":
        # passed in BSR(3) storage (3x3 blocks, one column index per block)
        B = W.reservoir_bsr3()
        return [(B, None, W.row_sums(W.bsr3_to_csr(B)))]
    if kind == "batch":
        return [(A, None, W.row_sums(A)) for A, _ in W.batch_cd(512, seed=5)]
    if kind == "tune":
        A = W.cd2d(wl["m"])
        return [(A, None, W.row_sums(A))]
    if kind == "sequence":
        A = W.cd3d_lognormal(wl["m"])
        return [(A, None, W.uniform_rhs(A.n_rows, seed=10 + k)) for k in range(wl["count"])]
    if kind == "spmv_qdot":
        A = W.cd3d_lognormal(wl["m"])
        return [(A, None, W.uniform_rhs(A.n_rows, seed=3))]
    raise ValueError(kind)


def _variant_desc(name, wl, systems):
    N = sum(A.n_rows for A, _, _ in systems)
    nnz = sum(A.nnz for A, _, _ in systems)
    if wl["kind"] == "spmv_qdot":
        return (f"fused y = A x, d = Q^H y on the 3-D log-normal convection-diffusion {wl['m']}^3 matrix "
                f"(N={N:,}, nnz={nnz:,}), n in {list(wl['ns'])}, x U[-1,1], fp64, {wl['calls']} calls each")
    what = {"cd3d": "3-D log-normal convection-diffusion 128^3",
            "helmholtz": "complex damped shifted Laplacian 256x256x64, A^H as separate CSR",
            "reservoir": "3x3-block reservoir system 64x64x32 cells, BSR(3) input",
            "batch": "512 2-D/3-D convection-diffusion systems, N ~ logU[1e3,1e5], one launch",
            "tune": f"2-D 5-point convection-diffusion {wl.get('m', 0)}^2, default launch configuration vs autotuned",
            "sequence": (f"sequence of {wl.get('count', 0)} right-hand sides U[-1,1] (seeds 10..) on the 3-D "
                         f"log-normal convection-diffusion {wl.get('m', 0)}^3 system, n by the rule of §5 "
                         f"(n0={wl.get('n0')}, step {wl.get('step')}, n in [{wl.get('n_min')}, {wl.get('n_max')}])")}[wl["kind"]]
    extra = ""
    if wl.get("kappa", 0.0) > 0:
        extra += f", omega guard kappa={wl['kappa']:g} (Eq. 5.1)"
    if wl.get("precond", 0) == 1:
        extra += ", Jacobi M=diag(A) (Algorithm 7.1)"
    if wl.get("precond", 0) == 2:
        extra += ", ILU(0) M=LU (Algorithm 7.1; level-scheduled triangular solves)"
    if wl.get("precond", 0) == 3:
        extra += ", multicolour ILU(0) M=P^T LU P (one triangular-solve level per colour)"
    if wl.get("tune"):
        extra += ", team size and per-class tile caps from mlbicgstab_autotune_batch (trials: A x = 1 to tol)"
    return f"{what} (N={N:,}, nnz={nnz:,}), n={wl['n']}, {_prec_name(wl)}{extra}, tol {wl['tol']:g}"


def _prec_name(wl):
    return "fp32-inner/fp64-refined" if wl.get("precision", 0) == 1 else "fp64"


def _config(wl, A, extra=None):
    cfg = {
        "workload": (f"cd3d_lognormal {wl['m']}^3 (N={A.n_rows:,}, nnz={A.nnz:,}), "
                     f"n={wl['n']}, {_prec_name(wl)}, b~U[-1,1] seed 2, x0=0, "
                     f"Q~N(0,1) seed 0, tol {wl['tol']:g}, maxit {wl['maxit']}"),
        "N": A.n_rows, "nnz": A.nnz, "n": wl["n"], "tol": wl["tol"],
        "maxit": wl["maxit"], "precision": _prec_name(wl),
        "l2": "inputs larger than L2 (no flush)",
    }
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    from paper_1106_3678_gb300 import replicas
    return replicas.world()


def cpu_info():
    """Host cores and CPU model of this machine."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return cores, f"{model or 'unknown'} ({platform.machine()})"


def oracle_sample(A, b, n, iters, threads=None):
    """Time `iters` iterations of the CPU oracle on the workload; returns
    (seconds per iteration, iterations done, threads).  threads=None: the
    sequential oracle on one core; else its multi-core build (fixed-block
    reductions) on that many threads."""
    import oracle as O
    lib = None
    used = 1
    if threads is not None:
        lib = O.load_par()
        used = O.par_threads(threads)
    cplx = np.iscomplexobj(b)
    Q = O.q_gauss(0, A.n_rows, n, complex_=cplx)
    t0 = time.perf_counter()
    r = O.mlbicgstabt(A, b, np.zeros_like(b), Q, iters, 0.0, lib=lib)
    dt = time.perf_counter() - t0
    return dt / max(r.iter, 1), r.iter, used


def cpu_baseline(A, b, n, iters_per_solve, it_all, it_one, unit=None):
    """The oracle on all host cores (the reported value) and on one core,
    each on a bounded sample of iterations of the same solve, converted to
    solves/sec with the iteration count of a full solve."""
    cores, model = cpu_info()
    spi_all, done_all, used = oracle_sample(A, b, n, it_all, threads=cores)
    spi_one, done_one, _ = oracle_sample(A, b, n, it_one)
    return {"value": 1.0 / (spi_all * iters_per_solve), "unit": unit or UNIT, "cores": used,
            "kind": "oracle", "cpu_model": model, "nproc": cores,
            "sample": (f"{done_all} iterations of the same solve on {used} host threads (the oracle's "
                       f"multi-core build: OpenMP, fixed-block reductions); solves/sec = 1/(seconds per "
                       f"iteration x {int(iters_per_solve)} iterations per GPU solve)"),
            "seconds_per_iteration": spi_all,
            "single_thread": {"value": 1.0 / (spi_one * iters_per_solve), "cores": 1,
                              "seconds_per_iteration": spi_one,
                              "sample": f"{done_one} iterations, sequential oracle, one core"}}


def fp64_peak(dev):
    """Dense FP64 throughput of this GPU (cuBLAS DGEMM through torch, 4096^3,
    best of 5, CUDA events; changes no GPU setting)."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    bm = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = a @ bm
    best = None
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ bm
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, bm, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def run_reference(args, wl):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    A, b = _make_inputs(wl)
    iters_solve = wl["iters"] or args.iters_per_solve
    sample = args.ref_iters
    cores, model = cpu_info()
    times = []
    used = cores
    for s in range(args.warmup + args.steps):
        spi, done, used = oracle_sample(A, b, wl["n"], sample, threads=cores)
        if s >= args.warmup:
            times.append(spi)
    spi = statistics.median(times)
    value = 1.0 / (spi * iters_solve) if iters_solve else None
    spi1, done1, _ = oracle_sample(A, b, wl["n"], max(10, sample // 10))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": spi * sample * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config(wl, A, {"iters_per_solve": iters_solve}),
        "cpu_baseline": {
            "value": value, "unit": UNIT, "cores": used, "kind": "oracle", "cpu_model": model,
            "nproc": cores,
            "sample": (f"{sample} iterations of the solve per step on {used} host threads (the "
                       f"oracle's multi-core build); solves/sec = 1/(seconds per iteration x "
                       f"{iters_solve} iterations per full solve)"),
            "single_thread": {"value": 1.0 / (spi1 * iters_solve), "cores": 1,
                              "seconds_per_iteration": spi1,
                              "sample": f"{done1} iterations, sequential oracle"}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed_solves(M, h, b_d, x_d, wl, stream, steps, warmup, barrier):
    """Warm-up solves, then `steps` timed solves; returns (total_ms, results)."""
    import torch
    for _ in range(warmup):
        with torch.cuda.stream(stream):
            x_d.zero_()
        M.mlbicgstab_solve(h, b_d, x_d, wl["tol"], wl["maxit"])
    results = []
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        with torch.cuda.stream(stream):
            x_d.zero_()
        res, _ = M.mlbicgstab_solve(h, b_d, x_d, wl["tol"], wl["maxit"])
        results.append(res.as_dict())
    ev1.record(stream)
    barrier()
    return ev0.elapsed_time(ev1), results


def _create(M, A, wl, stream):
    return M.mlbicgstab_create(A, n=wl["n"], q_seed=0, max_outer=10, stream=stream,
                               precision=wl.get("precision", 0),
                               inner_tol=wl.get("inner_tol"))


def _measure_variant(M, name, args, dev, stream, barrier, ws):
    import torch
    vwl = dict(WORKLOADS[name])
    vmax = args.variant_maxit if args.variant_maxit is not None else args.maxit
    if vmax > 0:
        vwl["maxit"] = vmax
    systems = _make_variant_inputs(vwl)
    if vwl["kind"] == "sequence":
        return _measure_sequence(M, name, vwl, systems, dev, stream, barrier, ws)
    if vwl["kind"] == "tune":
        return _measure_tune(M, name, vwl, systems, dev, stream, barrier, ws, args)
    if vwl["kind"] == "spmv_qdot":
        return _measure_spmv_qdot(M, name, vwl, systems, dev, stream, barrier, ws)
    dt = torch.complex128 if np.iscomplexobj(systems[0][2]) else torch.float64
    hs = [M.mlbicgstab_create(A, AH=AH, n=vwl["n"], q_seed=0, max_outer=10, stream=stream,
                              precision=vwl.get("precision", 0), inner_tol=vwl.get("inner_tol"),
                              kappa=vwl.get("kappa", 0.0), precond=vwl.get("precond", 0))
          for A, AH, _ in systems]
    bs = [torch.tensor(b, dtype=dt, device=dev) for _, _, b in systems]
    xs = [torch.zeros_like(b) for b in bs]
    steps = max(1, args.variant_steps)
    out = {"workload": name, "config": _variant_desc(name, vwl, systems),
           "precision": _prec_name(vwl), "n": vwl["n"], "unit": UNIT,
           "kappa": vwl.get("kappa", 0.0), "precond": ["none", "jacobi", "ilu0", "ilu0_mc"][vwl.get("precond", 0)]}
    if vwl["kind"] == "batch":
        if vwl.get("tune"):
            t0 = time.perf_counter()
            tr = M.mlbicgstab_autotune_batch(hs, tol=vwl["tol"], maxit=vwl["maxit"], use_cache=False)
            caps = [M.mlbicgstab_get_tuning(h)["batch_spt_cap"] for h in hs]
            out["autotune"] = dict(tr, seconds=time.perf_counter() - t0,
                                   caps={str(c): caps.count(c) for c in sorted(set(caps))})

        def once():
            for x in xs:
                x.zero_()
            return M.mlbicgstab_solve_batch(hs, bs, xs, [vwl["tol"]] * len(hs),
                                            [vwl["maxit"]] * len(hs))
        once()   # warm-up
        barrier()
        t0 = time.perf_counter()
        runs = [once() for _ in range(steps)]
        barrier()
        secs = (time.perf_counter() - t0) / steps
        res = runs[-1]
        out.update({
            "value": ws * len(hs) / secs, "ms_per_step": secs * 1e3,
            "systems_per_launch": len(hs),
            "kernel_ms": res[0].kernel_ms,
            "flags": sorted({r.flag for r in res}),
            "not_converged": sum(1 for r in res if r.flag != 0 or not r.true_relres < vwl["tol"]),
            "iters_total": sum(r.iter for r in res), "iters_max": max(r.iter for r in res),
            "true_relres_max": max(r.true_relres for r in res),
            "systems_by_ctas": {str(c): sum(1 for r in res if r.ctas == c) for c in sorted({r.ctas for r in res})},
        })
        # the batch kernel's algorithmic bytes (every system's passes, as
        # counted by the kernel) over the launch's device time
        kb = sum(r.bytes for r in res)
        kms = res[0].kernel_ms
        peak, peak_kind = _load_peaks()
        if kms > 0:
            out["roofline"] = {"bound": "hbm", "achieved": kb / (kms * 1e-3) / 1e9, "peak": peak,
                               "unit": "GB/s", "frac": kb / (kms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
                               "algorithmic_bytes_per_launch": kb, "kernel_ms_per_launch": kms,
                               "note": "systems smaller than L2 are served partly from L2"}
        # the same systems solved one by one with the plain FP64 path
        if vwl.get("precision", 0) == 0:
            for x in xs:
                x.zero_()
            barrier()
            t0 = time.perf_counter()
            for h, b, x in zip(hs, bs, xs):
                M.mlbicgstab_solve(h, b, x, vwl["tol"], vwl["maxit"])
            barrier()
            one = time.perf_counter() - t0
            out["one_by_one_fp64"] = {"value": ws * len(hs) / one, "seconds": one}
            out["speedup_vs_one_by_one_fp64"] = out["value"] / out["one_by_one_fp64"]["value"]
    else:
        h, b, x = hs[0], bs[0], xs[0]
        vms, vres = _timed_solves(M, h, b, x, vwl, stream, steps, 0, barrier)
        kb = sum(r["bytes"] for r in vres)
        kf = sum(r["flops"] for r in vres)
        kms = sum(r["kernel_ms"] for r in vres)
        gbs = kb / (kms * 1e-3) / 1e9 if kms > 0 else None
        peak, peak_kind = _load_peaks()
        out.update({
            "value": ws * len(vres) / (vms * 1e-3), "ms_per_step": vms / len(vres),
            "iters_per_solve": [r["iter"] for r in vres], "outer": [r["outer"] for r in vres],
            "flags": [r["flag"] for r in vres], "true_relres": [r["true_relres"] for r in vres],
            "achieved_gbs": gbs,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak if gbs else None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": kb / len(vres),
                         "kernel_ms_per_launch": kms / len(vres)},
            "flop_rate_tflops": kf / (kms * 1e-3) / 1e12 if kms > 0 else None,
        })
        if vwl.get("full"):
            # the largest single-GPU workload: end to end through the C ABI
            # with pinned host buffers, and the oracle on the host cores
            import torch
            A0, _, bh = systems[0]
            bp = torch.tensor(bh).pin_memory()
            xp = torch.zeros_like(bp).pin_memory()
            bn_, xn_ = bp.numpy(), xp.numpy()
            barrier()
            t0 = time.perf_counter()
            for _ in range(steps):
                xn_[:] = 0
                M.mlbicgstab_solve(h, bn_, xn_, vwl["tol"], vwl["maxit"])
            barrier()
            e2e_s = time.perf_counter() - t0
            es = bh.itemsize
            out["e2e"] = {"value": ws * steps / e2e_s, "unit": UNIT,
                          "h2d_bytes_per_step": 2 * A0.n_rows * es, "d2h_bytes_per_step": A0.n_rows * es + 168}
            if getattr(args, "no_cpu_baseline", False) is False:
                it = statistics.median(out["iters_per_solve"])
                out["cpu_baseline"] = cpu_baseline(A0, bh, vwl["n"], it, 100, 20)
    out["converged"] = _converged(out, vwl["tol"])
    for hh in hs:
        hh.destroy()
    return out


def _converged(v, tol):
    """Every solve of a variant flag 0 with true relative residual < tol."""
    flags = v.get("flags")
    if flags is None:
        return None
    rel = v.get("true_relres", v.get("true_relres_max"))
    rel = rel if isinstance(rel, list) else [rel]
    return all(f == 0 for f in flags) and all(r is not None and r < tol for r in rel)


def _measure_spmv_qdot(M, name, vwl, systems, dev, stream, barrier, ws):
    """The fused product y = A x, d = Q^H y alone, for n in vwl["ns"]:
      * FP64 through the synchronous call (mlbicgstab_spmv_qdot: launch,
        copy of d to the host, synchronisation), its device time from CUDA
        events around the launch inside the library, and the whole call;
      * FP64 and FP32 (the copies a refined handle keeps) through the
        asynchronous call, `calls` launches back to back on the stream
        between two CUDA events: the device time per product that a
        pipelined caller sees.
    The inputs (about 165-500 MB) exceed L2, so no flush between calls.
    Algorithmic bytes: A's SELL values and columns and slice offsets once,
    x once, y written once, the n columns of Q once."""
    import torch
    A, _, b = systems[0]
    N = A.n_rows
    peak, peak_kind = _load_peaks()
    x = torch.tensor(b, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    out = {"workload": name, "config": _variant_desc(name, vwl, systems), "precision": "fp64 and fp32",
           "n": vwl["n"], "unit": "products/s", "by_n": {}}

    def back_to_back(h, xx, yy, n):
        dd = torch.zeros(n + 1, dtype=torch.float64, device=dev)
        for _ in range(3):
            M.mlbicgstab_spmv_qdot_async(h, xx, yy, dd)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(vwl["calls"]):
            M.mlbicgstab_spmv_qdot_async(h, xx, yy, dd)
        e1.record(stream)
        e1.synchronize()
        ok = float(dd[-1].item()) == 0.0
        return e0.elapsed_time(e1) * 1e-3 / vwl["calls"], ok

    for n in vwl["ns"]:
        h = M.mlbicgstab_create(A, n=n, q_seed=0, stream=stream)
        info = M.mlbicgstab_info(h)
        byts = info["nnz_padded"] * 12 + 8 * (N // 32 + 2) + 8 * N * (2 + n)
        byts32 = info["nnz_padded"] * 8 + 8 * (N // 32 + 2) + 4 * N * (2 + n)
        for _ in range(3):
            M.mlbicgstab_spmv_qdot(h, x, y)
        barrier()
        kms = []
        t0 = time.perf_counter()
        for _ in range(vwl["calls"]):
            M.mlbicgstab_spmv_qdot(h, x, y)
            kms.append(M.mlbicgstab_info(h)["qd_kernel_ms"])
        call = (time.perf_counter() - t0) / vwl["calls"]
        barrier()
        k = float(np.mean(kms)) * 1e-3
        t64, ok64 = back_to_back(h, x, y, n)
        # the autotuner's choice of fused columns (and tile cap), then the
        # same back-to-back timing with it
        tune64 = M.mlbicgstab_autotune(h, iters=10, use_cache=False)
        t64t, ok64t = back_to_back(h, x, y, n)
        h.destroy()
        h32 = M.mlbicgstab_create(A, n=n, q_seed=0, stream=stream, precision=1)
        t32, ok32 = back_to_back(h32, x32, y32, n)
        tune32 = M.mlbicgstab_autotune(h32, iters=10, use_cache=False)
        t32t, ok32t = back_to_back(h32, x32, y32, n)
        h32.destroy()
        out["by_n"][str(n)] = {
            "fp64": {"kernel_us_sync_call": k * 1e6, "kernel_us_min_sync_call": min(kms) * 1e3,
                     "call_us": call * 1e6, "us_per_product_back_to_back": t64 * 1e6,
                     "algorithmic_bytes": byts, "achieved_gbs": byts / t64 / 1e9,
                     "frac_of_" + peak_kind + "_hbm": byts / t64 / 1e9 / peak,
                     "achieved_gbs_sync_call": byts / k / 1e9, "status_ok": ok64,
                     "fused_columns_default": _qd_rule(n, False),
                     "tuned": {"fused_columns": tune64["qd_fused"], "spt_cap": tune64["spt_cap"],
                               "tuner_us": tune64["qd_us"], "tuner_default_us": tune64["qd_default_us"],
                               "us_per_product_back_to_back": t64t * 1e6,
                               "frac_of_" + peak_kind + "_hbm": byts / t64t / 1e9 / peak,
                               "status_ok": ok64t}},
            "fp32": {"us_per_product_back_to_back": t32 * 1e6, "algorithmic_bytes": byts32,
                     "achieved_gbs": byts32 / t32 / 1e9,
                     "frac_of_" + peak_kind + "_hbm": byts32 / t32 / 1e9 / peak, "status_ok": ok32,
                     "fused_columns_default": _qd_rule(n, False, True),
                     "tuned": {"fused_columns": tune32["qd_fused"], "spt_cap": tune32["spt_cap"],
                               "tuner_us": tune32["qd_us"], "tuner_default_us": tune32["qd_default_us"],
                               "us_per_product_back_to_back": t32t * 1e6,
                               "frac_of_" + peak_kind + "_hbm": byts32 / t32t / 1e9 / peak,
                               "status_ok": ok32t}}}
    main = out["by_n"][str(vwl["n"])]
    out["value"] = ws * 1e6 / main["fp64"]["us_per_product_back_to_back"]
    out["ms_per_step"] = main["fp64"]["us_per_product_back_to_back"] * 1e-3
    out["roofline"] = {"bound": "hbm", "achieved": main["fp64"]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                       "frac": main["fp64"]["achieved_gbs"] / peak, "peak_kind": peak_kind,
                       "timing": "back-to-back asynchronous launches between CUDA events"}
    out["roofline_fp32"] = {"bound": "hbm", "achieved": main["fp32"]["achieved_gbs"], "peak": peak,
                            "unit": "GB/s", "frac": main["fp32"]["achieved_gbs"] / peak, "peak_kind": peak_kind}
    return out


def _qd_rule(n, cplx, narrow=False):
    """The library's built-in count of Q columns fused into the product."""
    if n == 4 and not cplx:
        return 4
    if n > 4 and not cplx and not narrow:
        return 1
    return 2 if n >= 2 else 1


def _measure_tune(M, name, vwl, systems, dev, stream, barrier, ws, args):
    """The same solve with the default launch configuration, then after
    mlbicgstab_autotune (tuning itself is setup and not timed)."""
    import torch
    A, _, b = systems[0]
    h = M.mlbicgstab_create(A, n=vwl["n"], q_seed=0, max_outer=10, stream=stream)
    bd = torch.tensor(b, dtype=torch.float64, device=dev)
    xd = torch.zeros_like(bd)
    steps = max(1, args.variant_steps)
    out = {"workload": name, "config": _variant_desc(name, vwl, systems), "precision": "fp64",
           "n": vwl["n"], "unit": UNIT}
    ms0, r0 = _timed_solves(M, h, bd, xd, vwl, stream, steps, 1, barrier)
    grid0 = M.mlbicgstab_info(h)["grid"]
    tune = M.mlbicgstab_autotune(h, iters=30, use_cache=False)
    ms1, r1 = _timed_solves(M, h, bd, xd, vwl, stream, steps, 1, barrier)
    out["default"] = {"value": ws * steps / (ms0 * 1e-3), "grid": grid0, "spt_cap": 15,
                      "iters": [r["iter"] for r in r0]}
    out["tuned"] = {"value": ws * steps / (ms1 * 1e-3), "grid": tune["grid"], "spt_cap": tune["spt_cap"],
                    "iters": [r["iter"] for r in r1], "trials": tune["trials"]}
    out["value"] = out["tuned"]["value"]
    out["ms_per_step"] = ms1 / steps
    out["flags"] = sorted({r["flag"] for r in r0 + r1})
    out["speedup_vs_default"] = out["tuned"]["value"] / out["default"]["value"]
    h.destroy()
    return out


def _measure_sequence(M, name, vwl, systems, dev, stream, barrier, ws):
    """One handle (built for n_max) solves the right-hand sides in order,
    first with n chosen by mlbicgstab_solve_sequence, then at fixed n0."""
    import torch
    A = systems[0][0]
    h = M.mlbicgstab_create(A, n=vwl["n"], q_seed=0, max_outer=10, stream=stream)
    bs = [torch.tensor(b, dtype=torch.float64, device=dev) for _, _, b in systems]
    count = len(bs)
    out = {"workload": name, "config": _variant_desc(name, vwl, systems), "precision": "fp64",
           "n": vwl["n0"], "unit": UNIT}
    for label, step in (("adaptive", vwl["step"]), ("fixed_n0", 0)):
        xs = [torch.zeros_like(b) for b in bs]
        barrier()
        t0 = time.perf_counter()
        res, used = M.mlbicgstab_solve_sequence([h] * count, bs, xs, [vwl["tol"]] * count, [vwl["maxit"]] * count,
                                                n0=vwl["n0"], step=step, n_min=vwl["n_min"], n_max=vwl["n_max"])
        barrier()
        secs = time.perf_counter() - t0
        out[label] = {"value": ws * count / secs, "seconds": secs, "n_used": used,
                      "iters": [r.iter for r in res], "flags": sorted({r.flag for r in res}),
                      "true_relres_max": max(r.true_relres for r in res)}
    out["value"] = out["adaptive"]["value"]
    out["ms_per_step"] = 1e3 * out["adaptive"]["seconds"] / count
    out["speedup_vs_fixed_n0"] = out["adaptive"]["value"] / out["fixed_n0"]["value"]
    h.destroy()
    return out


def run_ours(args, wl):
    import torch

    from paper_1106_3678_gb300 import mlbicgstab as M

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    A, b = _make_inputs(wl)
    N = A.n_rows
    stream = torch.cuda.Stream()
    h = _create(M, A, wl, stream)
    # setup, like create: not timed (--no-autotune: the default launch
    # configuration, e.g. so that a profiler's first solve launch is the
    # timed one)
    tune = None if args.no_autotune else M.mlbicgstab_autotune(h, iters=20, use_cache=False)
    info = M.mlbicgstab_info(h)
    b_d = torch.tensor(b, dtype=torch.float64, device=dev)
    x_d = torch.zeros(N, dtype=torch.float64, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    total_ms, results = _timed_solves(M, h, b_d, x_d, wl, stream, args.steps, args.warmup, barrier)
    clk = clocks.stop()

    from paper_1106_3678_gb300 import replicas
    total_ms = replicas.max_over_ranks(total_ms, dev)

    # variants: other workloads, precisions and the batched form
    variants = []
    for name in ([] if args.no_variants else (args.variant or VARIANTS)):
        variants.append(_measure_variant(M, name, args, dev, stream, barrier, ws))
    head_value = ws * args.steps / (total_ms * 1e-3)
    head_ok = all(r["flag"] == 0 and r["true_relres"] < wl["tol"] for r in results)
    by_name = {v["workload"]: v for v in variants}
    by_name.setdefault(args.workload, {"workload": args.workload, "value": head_value, "converged": head_ok})
    for v in variants:
        if v["workload"] in ("cd3d128_n4_fp64_jacobi", "cd3d128_n4_fp64_ilu0", "cd3d128_n4_fp64_ilu0mc"):
            ok = bool(v.get("converged")) and head_ok
            v["pairs"] = {"speedup_vs_unpreconditioned": {
                "against": args.workload, "speedup": v["value"] / head_value if ok else None,
                "both_converged": ok, "iters": v.get("iters_per_solve"),
                "iters_against": [r["iter"] for r in results]}}
    for name, base, key in PAIRS:
        v, bv = by_name.get(name), by_name.get(base)
        if v is None or bv is None or "value" not in v:
            continue
        ok = bool(v.get("converged")) and bool(bv.get("converged"))
        v.setdefault("pairs", {})[key] = {
            "against": base, "speedup": v["value"] / bv["value"] if ok else None,
            "both_converged": ok,
            "iters": v.get("iters_per_solve", v.get("iters_total")),
            "iters_against": bv.get("iters_per_solve", bv.get("iters_total"))}

    # end to end through the C ABI with pinned host buffers
    b_h = torch.tensor(b, dtype=torch.float64).pin_memory()
    x_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    bn, xn = b_h.numpy(), x_h.numpy()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = 0 if args.no_e2e else max(1, args.steps)
    for _ in range(e2e_steps):
        xn[:] = 0.0
        M.mlbicgstab_solve(h, bn, xn, wl["tol"], wl["maxit"])
    barrier()
    e2e_s = replicas.max_over_ranks(max(time.perf_counter() - t0, 1e-9), dev)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = _load_peaks()
    kern_ms = sum(r["kernel_ms"] for r in results)
    kern_bytes = sum(r["bytes"] for r in results)
    achieved = kern_bytes / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None
    iters = [r["iter"] for r in results]
    value = ws * args.steps / (total_ms * 1e-3)

    cpu = None
    if not args.no_cpu_baseline and ws >= 1:
        cpu = cpu_baseline(A, b, wl["n"], statistics.median(iters), 300, 100)
    kern_flops = sum(r["flops"] for r in results)
    fp64 = None
    if not args.no_fp64_peak:
        pk = fp64_peak(dev)
        fl = kern_flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
        fp64 = {"achieved_tflops": fl, "peak_tflops": pk, "frac": fl / pk if fl else None,
                "peak_source": "cuBLAS DGEMM 4096^3 through torch, best of 5, CUDA events, this run",
                "flops_per_launch": kern_flops / len(results),
                "flops_model": "Table 4.3 operations: 2 per stored entry per product, 2 per element "
                               "per inner product, AXPY or norm, 1 per scaling"}
    nconv = sum(1 for r in results if r["flag"] == 0 and r["true_relres"] < wl["tol"])

    # ML(n)BiCGStab against BiCGStab (n = 1) on the headline system: the
    # comparison the paper reports (its figures: Matlab, Pentium 4, ILU(0))
    vs_bicg = None
    n1 = next((v for v in variants if v["workload"] == "cd3d128_n1_fp64"), None)
    if args.workload == DEFAULT and n1 is not None and n1.get("converged") and nconv == len(results):
        vs_bicg = {"against": "cd3d128_n1_fp64", f"n{wl['n']}": value / n1["value"]}
        for v in variants:
            if v["workload"] in ("cd3d128_n8_fp64", "cd3d128_n16_fp64") and v.get("converged"):
                vs_bicg[f"n{v['n']}"] = v["value"] / n1["value"]
        vs_bicg["iters_n1"] = n1.get("iters_per_solve")
        vs_bicg["context"] = ("the paper reports ML(n)BiCGStab time reductions over BiCGStab only for "
                              "ILU(0)-preconditioned Matlab runs on a Pentium 4 (figures, no values in "
                              "the text) and >70% / ~60% on SPE9 sequences")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config(wl, A, {"grid": info["grid"], "block": info["block"],
                                  "nnz_sell32": info["nnz_padded"],
                                  "check": (f"{nconv} of {len(results)} timed solves converged (flag 0, "
                                            f"true relative residual < {wl['tol']:g}); max true relres "
                                            f"{max(r['true_relres'] for r in results):.3g}"),
                                  "autotune": None if tune is None else
                                  {k: tune[k] for k in ("grid", "spt_cap", "us_per_iter",
                                                        "default_us_per_iter", "trials")}}),
        "iters_per_solve": iters, "flags": [r["flag"] for r in results],
        "true_relres": [r["true_relres"] for r in results],
        "restarts": [r["outer"] for r in results],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": (NCU_DRAM_BYTES_PER_ITER * statistics.median(iters)
                                 if NCU_DRAM_BYTES_PER_ITER and args.workload == DEFAULT else None),
                     "traffic_source": "ncu dram bytes of a 300-iteration launch, scaled by iterations",
                     "peak_kind": peak_kind,
                     "kernel": "solve_kernel<double> (persistent, one launch per solve)",
                     "algorithmic_bytes_per_launch": kern_bytes / len(results),
                     "kernel_ms_per_launch": kern_ms / len(results),
                     "fp64": fp64},
        "e2e": {"value": (ws * e2e_steps / e2e_s) if e2e_steps else None, "unit": UNIT,
                "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8 + 168},
        "gpu_launches": args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "speedup_vs_bicgstab": vs_bicg,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    h.destroy()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--ref-iters", type=int, default=200,
                    help="oracle iterations per CPU sample")
    ap.add_argument("--iters-per-solve", type=int, default=0,
                    help="reference arm: iterations of a full solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-peak", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch configuration of the headline handle")
    ap.add_argument("--variant", action="append", choices=sorted(WORKLOADS),
                    help="extra workloads measured on the same matrix (repeatable)")
    ap.add_argument("--variant-steps", type=int, default=1)
    ap.add_argument("--maxit", type=int, default=0,
                    help="override the iteration cap (short runs for profiling)")
    ap.add_argument("--variant-maxit", type=int, default=None,
                    help="iteration cap of the variants (default: --maxit; 0: each workload's own)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.maxit > 0:
        wl["maxit"] = args.maxit
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
