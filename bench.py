"""Benchmark: p-BiCGStab time to a 1e-10 true relative residual on GB300, mixed vs FP64.

Headline workload (one "step" = one complete solve): 2D upwind convection-diffusion,
1024 x 1024 grid (N = 1,048,576), cell Peclet 0.5, matrix stored as 5 FP64 diagonals,
Jacobi preconditioner, x* ~ U[0,1] (seed 2), b = A x*, x0 = 0, tol 1e-10 on
||b - A x|| / ||b|| (verified in FP64).  The headline variant is set by --precision:
mixed (FP32 recurrences restarted from the FP64 residual every 50 iterations, the
default) or fp64; the FP64 variants (the same restart policy, the paper's periodic
replacement, and classic BiCGStab, Algorithm 1) are measured alongside.  The 3D
256^3 CSR system with the degree-2 Neumann preconditioner (N = 16,777,216) is measured
in the same run ("convdiff3d" block; --no-3d skips it).

Prints ONE JSON line on rank 0.  --impl reference times the oracle instead: the same
headline solve, run to completion by the C oracle on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p-BiCGStab time to true rel. residual 1e-10 & HBM GB/s, mixed vs FP64"
GRID = 1024


# ----------------------------------------------------------------------------- byte model
MASK_BYTES = 2   # stencil storage: one 16-bit presence mask per row and SpMV


def bytes_per_row_iteration(precision: str, fmt: str = "dia", ndiag: int = 5, nnz_row: float = 5.0,
                            storage: str = "stencil") -> float:
    """Algorithmic bytes per row and iteration of the fused two-pass iteration
    (Jacobi folded into the operator A D^{-1}, m and n formed on the fly, q, u, y
    recomputed, neighbour gathers counted once):
      pass A reads w k g l s z v r + D^{-1}, writes g s l z t;
      pass B reads z x g k l r s w t r0 + D^{-1}, writes v x r k w;
    28 vector streams (x read+written in FP64) plus two reads of the operator.
    DIA: the folded operator stores ndiag-1 diagonals and D^{-1} replaces the unit
    main diagonal, so operator + D^{-1} = ndiag values per row per pass.  Stencil
    storage: the operator is the per-row mask and D^{-1} one constant."""
    es = 8 if precision == "fp64" else 4
    vec = 26 * es + 2 * 8            # x is FP64 in both modes
    if storage == "stencil":
        mat = 2 * MASK_BYTES
    elif fmt == "dia":
        mat = 2 * ndiag * es
    else:
        mat = 2 * (nnz_row * (es + 4) + 4 + es)   # values + col + row_ptr + D^{-1}
    return float(vec + mat)


def bytes_per_row_iteration_neumann(precision: str, degree: int = 2, nnz_row: float = 7.0,
                                    storage: str = "stencil") -> float:
    """Algorithmic bytes per row and iteration with a degree-d Neumann preconditioner on a
    CSR matrix: m and n must be stored, each M^{-1} application adds d Jacobi sweeps, so
    the iteration streams 30 + 8d vectors (x in FP64) and reads the matrix 2 + 2d times
    (values + int32 columns + row pointer; stencil storage: the mask).  Degree 2:
    46 streams + 6 matrix reads."""
    es = 8 if precision == "fp64" else 4
    streams = 30 + 8 * degree
    vec = (streams - 2) * es + 2 * 8
    per_read = MASK_BYTES if storage == "stencil" else nnz_row * (es + 4) + 4
    mat = (2 + 2 * degree) * per_read
    return float(vec + mat)


def bytes_per_row_replacement(precision: str, ndiag: int = 5, storage: str = "stencil") -> float:
    """Eq. (rr) pass pair: R1 reads b, x, g, z + 2 FP64 operator reads, writes r k s l n;
    R2 reads r, s, r0 + 2 folded operator reads, writes w z."""
    es = 8 if precision == "fp64" else 4
    op64 = MASK_BYTES if storage == "stencil" else ndiag * 8
    opT = MASK_BYTES if storage == "stencil" else ndiag * es
    r1 = 2 * 8 + es * 2 + 2 * op64 + 5 * es
    r2 = 3 * es + 2 * opT + 2 * es
    return float(r1 + r2)


def fp64_flops_per_row_iteration(ndiag: int = 5) -> float:
    """Algorithmic FP64 flops per row and iteration of Algorithm 2 with Jacobi folded into
    A D^{-1} (DIA, unit main diagonal): two SPMVs of ndiag-1 FMAs, two D^{-1} scalings,
    the 18 AXPY-equivalents of Algorithm 2 and 7 dot products (6 + the stopping norm),
    an FMA counting 2 flops."""
    return 2 * 2 * (ndiag - 1) + 2 + 2 * 18 + 2 * 7


def fp64_flops_per_row_iteration_neumann(nnz_row: int = 7, degree: int = 2) -> float:
    """The same count with a degree-d Neumann preconditioner on a CSR operator (diagonal
    stored): t = A m and v = A n (nnz_row FMAs each); each M^{-1} application runs d Jacobi
    sweeps of one SpMV plus 3 flops (subtract, FMA) -- the first also scales by D^{-1} --
    for m and for n; the AXPYs (18) and 7 dot products as above."""
    spmv = 2 * nnz_row
    sweeps = 2 * (degree * (spmv + 3) + 1)
    return 2 * spmv + sweeps + 2 * 18 + 2 * 7


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("common.cuh", "solver.cuh", "capi.cu", "capi_internal.h", "stencil.cu", "kernels_f64.cu",
              "kernels_f32.cu", "kernels_vec.cu"):
        h.update(open(os.path.join(ROOT, "paper_1809_01948_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(variant: str, workload: str):
    """Per-iteration DRAM bytes from profiles/dram_per_iteration.txt, if the kernel is unchanged."""
    try:
        hsh = kernel_source_hash()
        for line in open(os.path.join(ROOT, "profiles", "dram_per_iteration.txt")):
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[0] == variant and f[1] == workload and f[2] == hsh:
                return float(f[3])
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock, power and throttle reasons during a timed region;
    the raw CSV goes to ``path`` (``--clocks-csv``), else to a temporary file."""

    def __init__(self, path=None):
        import tempfile
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), "pbcg_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                s = float(f[1])
                mx = float(f[2])
            except ValueError:
                continue
            sm.append(s)
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        busy = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm
def bytes_per_row_restart(precision: str, ndiag: int = 5, storage: str = "stencil") -> float:
    """A (re)start of Algorithm 2 (reading R20): the initialisation pass reads b, x and the FP64
    operator, writes r, r0, k and zeros g, s, l, z, v; the next pass reads k and the operator
    and writes w."""
    es = 8 if precision == "fp64" else 4
    op64 = MASK_BYTES if storage == "stencil" else ndiag * 8
    opT = MASK_BYTES if storage == "stencil" else ndiag * es
    return float(2 * 8 + op64 + 8 * es + es + opT + es)


def measured_fp64_tflops(dev) -> float:
    """FP64 arithmetic rate of this GPU, measured here: a cuBLAS DGEMM (4096^3, best of 5,
    CUDA events) -- the denominator of the FP64-pipe roofline."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b_ = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b_)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b_)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b_
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def workload_setup(kind: str, grid: int, dev, degree: int = 2):
    """The synthetic system of a workload, its solver inputs, and the byte / flop models
    (degree: the Neumann degree of the 3D system)."""
    import torch
    import testproblems as tp
    if kind == "convdiff2d":
        prob = tp.problem_convdiff2d(grid)
        off, data = tp.csr_to_dia(prob.A)
        mat = dict(offsets=off.tolist(), dia=torch.from_numpy(data).to(dev), precond="jacobi")
        name = "convdiff2d_%dx%d_dia5_jacobi_tol1e-10" % (grid, grid)
        fmt = "DIA 5 diagonals FP64"
        variants = {
            # FP32 recurrences restarted from the FP64 residual every 50 iterations (reading R20)
            "mixed": dict(precision="mixed", restart_period=50, stag_window=4000),
            # FP64 with the same restart policy (every 100 iterations)
            "fp64": dict(precision="fp64", restart_period=100, stag_window=4000),
            # the paper's periodic residual replacement (Section 3.6, every 100 iterations)
            "fp64_rr100": dict(precision="fp64", rr_period=100),
            # Algorithm 1, the paper's reference method
            "classic": dict(precision="fp64", method="classic"),
        }
        model = dict(bpr=lambda prec, st: bytes_per_row_iteration(prec, storage=st),
                     flops=fp64_flops_per_row_iteration())
    else:
        prob = tp.problem_convdiff3d(grid)
        mat = dict(row_ptr=torch.from_numpy(prob.A.row_ptr).to(dev), col=torch.from_numpy(prob.A.col).to(dev),
                   val=torch.from_numpy(prob.A.val).to(dev), precond="neumann", degree=degree)
        name = "convdiff3d_%d^3_csr7_neumann%d_tol1e-10" % (grid, degree)
        fmt = "CSR int32, 7 nnz/row, FP64 values"
        variants = {
            # FP32 recurrences restarted every 75 iterations (reading R20)
            "mixed": dict(precision="mixed", restart_period=75, stag_window=4000),
            # the paper's periodic replacement (every 100 iterations)
            "fp64": dict(precision="fp64", rr_period=100),
        }
        model = dict(bpr=lambda prec, st: bytes_per_row_iteration_neumann(prec, degree=degree, storage=st),
                     flops=fp64_flops_per_row_iteration_neumann(degree=degree))
    return prob, mat, name, fmt, variants, model


def roofline_of(kind, model, prec, res, n, hbm_peak, hbm_src, fp64_peak, storage, workload):
    """Roofline of the persistent solver kernel (one launch per solve) from its CUDA-event
    time: achieved algorithmic bytes (the section 8(d) model: matrix values as stored by the
    general formats) and the same with the stencil storage's actual operand set, DRAM traffic
    from the ncu table, and for FP64 the FP64-pipe rate against the measured DGEMM peak."""
    its, nrep, nrst = res["iterations"], res["n_replacements"], res["n_restarts"]
    kernel_s = res["kernel_ms"] * 1e-3

    def gbs(st):
        b = n * (model["bpr"](prec, st) * its + bytes_per_row_replacement(prec, storage=st) * nrep
                 + bytes_per_row_restart(prec, storage=st) * nrst)
        return b / kernel_s / 1e9

    per_it = measured_traffic(prec, workload)
    hbm = {"achieved": round(gbs("general"), 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(gbs("general") / hbm_peak, 4), "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)",
           "model": "section 8(d) algorithmic bytes: %.0f B per row and iteration" % model["bpr"](prec, "general"),
           "traffic": per_it * its if per_it is not None else None,
           "stencil_storage_model": {"bytes_per_row_iteration": model["bpr"](prec, "stencil"),
                                     "achieved": round(gbs("stencil"), 1),
                                     "frac": round(gbs("stencil") / hbm_peak, 4)} if storage == "stencil" else None}
    if prec == "fp64":
        ach = model["flops"] * n * its / kernel_s / 1e12
        return {"bound": "alu", "achieved": round(ach, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                "frac": round(ach / fp64_peak, 4), "traffic": hbm["traffic"],
                "peak_source": "measured in this run (cuBLAS DGEMM 4096^3, FP64 pipe)",
                "flops_per_row_iteration": model["flops"], "hbm": hbm}
    out = {"bound": "hbm"}
    out.update(hbm)
    return out


def run_gpu(args):
    import numpy as np
    import torch
    import paper_1809_01948_gb300 as pb
    from paper_1809_01948_gb300.sharding import max_over_ranks
    pb.build()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    hbm_peak, hbm_src = _hbm_peak()
    fp64_peak = measured_fp64_tflops(dev)
    sampler = ClockSampler(args.clocks_csv)
    sampler_on = False

    def measure(kind, grid, headline):
        nonlocal sampler_on
        prob, mat, name, fmt, variants, model = workload_setup(kind, grid, dev, args.degree)
        b = torch.from_numpy(prob.b).to(dev)
        n = prob.A.n
        if args.only:
            variants = {headline: variants[headline]}
        solvers = {k: pb.Solver(n, tol=1e-10, max_it=args.max_it, **mat, **v) for k, v in variants.items()}
        storage = solvers[headline].storage

        def one(vname):
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, res = solvers[vname].solve(b, x)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), res

        results = {}
        for vname in [headline] + [k for k in variants if k != headline]:
            for _ in range(args.warmup):
                one(vname)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            if not sampler_on:
                sampler.start()
                sampler_on = True
            times, ktimes, last = [], [], None
            for _ in range(args.steps):
                ms, res = one(vname)
                times.append(ms)
                ktimes.append(res.time_ms)
                last = res
            torch.cuda.synchronize()
            total = max_over_ranks(sum(times), device=dev)   # replicas: the slowest rank's time
            r = dict(ms_per_solve=round(total / args.steps, 4), kernel_ms=round(statistics.mean(ktimes), 4),
                     iterations=last.iterations, n_replacements=last.n_replacements, n_restarts=last.n_restarts,
                     rel_res_true=last.rel_res_true, status=pb.STATUS_NAMES[last.status],
                     policy=variants[vname])
            prec = variants[vname]["precision"]
            r["roofline"] = roofline_of(kind, model, prec, r, n, hbm_peak, hbm_src, fp64_peak,
                                        solvers[vname].storage, name)
            results[vname] = r
        return dict(prob=prob, n=n, name=name, fmt=fmt, storage=storage, results=results, solvers=solvers,
                    variants=variants)

    headline = args.precision
    third = None
    if args.workload == "convdiff3d":          # the 3D system alone, as the headline
        main = measure("convdiff3d", args.grid3 or 256, headline)
    else:
        main = measure("convdiff2d", args.grid or GRID, headline)
        if not args.no_3d:
            third = measure("convdiff3d", args.grid3 or 256, headline)
            for s_ in third["solvers"].values():
                s_.close()
    clocks = sampler.stop() if sampler_on else None
    head = main["results"][headline]
    n = main["n"]

    # end-to-end through the public API with host buffers (pinned)
    b_pin = torch.from_numpy(main["prob"].b).pin_memory()
    x_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for k in range(0 if args.no_e2e else max(1, args.steps)):
        x_pin.zero_()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, res = main["solvers"][headline].solve_host(b_pin.numpy(), x_pin.numpy())
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": round(statistics.mean(e2e_times), 4) if e2e_times else None, "unit": "ms",
           "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n + 64}
    for s_ in main["solvers"].values():
        s_.close()

    def block(m):
        res = m["results"]
        out = {"config": {"workload": m["name"], "n": m["n"], "format": m["fmt"],
                          "operator_storage": m["storage"]},
               "variants": {k: {kk: vv for kk, vv in v.items() if kk != "roofline"} for k, v in res.items()},
               "rooflines": {k: v["roofline"] for k, v in res.items()}}
        if "mixed" in res and "fp64" in res:
            out["mixed_vs_fp64"] = round(res["fp64"]["ms_per_solve"] / res["mixed"]["ms_per_solve"], 3)
        return out

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        prec = main["variants"][headline]["precision"]
        line = {
            "metric": METRIC, "value": head["ms_per_solve"], "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_solve"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": main["name"], "n": n, "format": main["fmt"],
                       "operator_storage": main["storage"] + (
                           " (constant coefficients detected at create: one value per offset + 16-bit row mask)"
                           if main["storage"] == "stencil" else ""),
                       "precision": prec + (" (FP32 vectors, values, SpMV and recurrences; FP64 x, dot products, "
                                            "scalars, restart residual; true residual verified in FP64)"
                                            if prec == "mixed" else ""),
                       "policy": main["variants"][headline], "global_batch": 1 * world,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between steps (256 MB write)"},
            "iterations": head["iterations"], "n_restarts": head["n_restarts"],
            "n_replacements": head["n_replacements"], "rel_res_true": head["rel_res_true"],
            "status": head["status"],
            "iters_per_s": round(head["iterations"] / (head["kernel_ms"] * 1e-3), 1),
            "kernel_ms": head["kernel_ms"],
            "mixed_vs_fp64": block(main).get("mixed_vs_fp64"),
            "variants": block(main)["variants"],
            "variant_rooflines": block(main)["rooflines"],
            "roofline": head["roofline"],
            "convdiff3d": block(third) if third else None,
            "e2e": e2e, "clocks": clocks,
            "gpu_launches": 3 * args.steps,
            "fp64_peak_tflops": round(fp64_peak, 4),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle arm
# The oracle timed on the host cores: the C oracle (oracle/c_oracle.c, OpenMP over every
# core), which restates the numpy oracle step for step, runs the headline solve of the 2D
# 1024^2 system to completion with the headline variant's policy.
HEADLINE_POLICY = {
    "mixed": dict(mixed=True, restart_period=50, stag_window=4000),
    "fp64": dict(mixed=False, restart_period=100, stag_window=4000),
}


def _c_oracle_solve(prec: str, grid: int = GRID):
    import numpy as np
    import testproblems as tp
    from oracle import c_oracle
    prob = tp.problem_convdiff2d(grid)
    A = prob.A.to_scipy()
    t0 = time.perf_counter()
    x, r = c_oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-10, maxit=20000, **HEADLINE_POLICY[prec])
    dt = time.perf_counter() - t0
    true = float(np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b))
    return dict(seconds=dt, iterations=r["iterations"], status=r["status"], rel_res_true=true,
                n_restarts=r["n_restarts"], n=prob.A.n)


def cpu_baseline(args):
    """The headline solve by the C oracle on all host cores, run to completion."""
    from oracle import c_oracle
    s = _c_oracle_solve(args.precision, args.grid or GRID)
    bpr = bytes_per_row_iteration("fp64" if args.precision == "fp64" else "mixed", storage="general")
    return {"value": round(s["seconds"] * 1e3, 1), "unit": "ms", "cores": c_oracle.threads(), "kind": "oracle",
            "sample": "one complete solve of the 2D %d^2 system to a 1e-10 true residual with the headline "
                      "policy (%s) by the C oracle (OpenMP, all host cores): %d iterations, %s, true residual %.2e"
                      % (args.grid or GRID, args.precision, s["iterations"], s["status"], s["rel_res_true"]),
            "ms_per_iteration": round(s["seconds"] * 1e3 / max(1, s["iterations"]), 3),
            "algorithmic_gbs": round(bpr * s["n"] * s["iterations"] / s["seconds"] / 1e9, 1),
            "host_copy_gbs": round(c_oracle.host_copy_gbs(), 1), "host": _host()}


def _host():
    """The machine the CPU baseline ran on."""
    import platform
    return {"arch": platform.machine(), "logical_cpus": os.cpu_count()}


# ----------------------------------------------------------------------------- batched and autograd
def _timed_steps(args, one, sampler_on=True):
    """W warm-up steps, then K timed steps bracketed by synchronisation; returns (ms list, clocks)."""
    import torch
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    sampler = ClockSampler(args.clocks_csv) if sampler_on else None
    if sampler:
        sampler.start()
    out = []
    for _ in range(args.steps):
        out.append(one())
    torch.cuda.synchronize()
    return out, (sampler.stop() if sampler else None)


def _hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return peaks.get("hbm_gbs", 6800.0), "measured" if "hbm_gbs" in peaks else "fallback"
    except Exception:
        return 6800.0, "fallback"


def run_batched(args):
    """Batched workload: 512 independent random banded systems (N_k ~ U[2048, 65536], 7-15
    non-zeros per row, FP32 values), mixed precision, Jacobi, tol 1e-8, one persistent
    launch replayed from a CUDA graph.  A step is one batch solve of all systems."""
    import numpy as np
    import torch
    import testproblems as tp
    import paper_1809_01948_gb300 as pb
    from paper_1809_01948_gb300.sharding import max_over_ranks, shard_systems
    pb.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bp = tp.problem_batched_banded()
    if world > 1:   # independent systems: each rank solves its share, no collective on the data path
        import torch.distributed as dist
        dist.init_process_group("nccl")
        mine = shard_systems([s_.A.n for s_ in bp.systems], world)[rank]
        bp = tp.BatchProblem(bp.name, [bp.systems[k] for k in mine], tol=bp.tol, maxit=bp.maxit)
    c = bp.concat()
    row_off, nnz_off = c["row_off"], c["nnz_off"]
    rp = torch.from_numpy(c["row_ptr"]).to(dev)
    col = torch.from_numpy(c["col"]).to(dev)
    val = torch.from_numpy(c["val"]).to(dev)
    b = torch.from_numpy(c["b"]).to(dev)
    s = pb.BatchSolver(row_off, nnz_off, rp, col, val, precond="jacobi", precision="mixed", tol=1e-8,
                       max_it=1000, rr_theta=1e-3)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    last = {}

    def one():
        flush.fill_(1.0)
        x = torch.zeros_like(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, info = s.solve(b, x)
        e1.record()
        torch.cuda.synchronize()
        last.update(info)
        return e0.elapsed_time(e1)

    times, clocks = _timed_steps(args, one)
    ms = max_over_ranks(statistics.mean(times), device=dev)   # the job ends with its slowest rank
    sizes = np.diff(row_off)
    nnz_row = float(nnz_off[-1]) / float(row_off[-1])
    row_its = float(np.sum(sizes * last["iterations"]))
    # per row and iteration: 26 FP32 vector streams + FP64 x twice + two CSR reads (FP32 values,
    # int32 columns, row pointer, D^-1)
    bpr = 26 * 4 + 2 * 8 + 2 * (nnz_row * 8 + 4 + 4)
    peak, src = _hbm_peak()
    ach = bpr * row_its / (last["time_ms"] * 1e-3) / 1e9
    line = {"metric": "batched p-BiCGStab time to solve all systems to 1e-8", "value": round(ms, 4), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batched_512_random_banded_fp32_jacobi_tol1e-8", "n_sys": len(row_off) - 1,
                       "total_rows": int(row_off[-1]), "nnz_per_row": round(nnz_row, 2),
                       "launch": "%d x %d, %d block(s) per system, %d thread(s) per row, %s build (autotuned), "
                                 "CUDA graph" % (last["grid_blocks"], last["block_threads"], last["cluster_blocks"],
                                                 last["lanes_per_row"], last["build"]),
                       "l2": "flushed between steps (256 MB write)"},
            "n_ok": int(last["n_ok"]), "iterations_mean": float(np.mean(last["iterations"])),
            "iterations_max": int(np.max(last["iterations"])), "kernel_ms": round(last["time_ms"], 4),
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "traffic": None, "peak_source": src,
                         "bytes_per_row_iteration": round(bpr, 1), "row_iterations": row_its},
            "e2e": {"value": None, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "clocks": clocks, "gpu_launches": args.steps, "cpu_baseline": None}
    if world > 1:
        line["config"]["parallelism"] = "systems split across %d ranks (largest first, balanced rows)" % world
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_autograd(args):
    """Differentiable workload: loss = sum ||X - X_t||^2 with X = A^{-1} B through the differentiable
    solve (16 right-hand sides on the 512^2 convection-diffusion CSR system, FP64); a step is
    the forward multi-RHS solve plus the backward pass (transposed-matrix adjoint solve and
    the value gradient)."""
    import torch
    import testproblems as tp
    import paper_1809_01948_gb300 as pb
    pb.build()
    dev = torch.device("cuda", 0)
    mp = tp.problem_convdiff2d_multi()
    rp = torch.from_numpy(mp.A.row_ptr).to(dev)
    col = torch.from_numpy(mp.A.col).to(dev)
    vals0 = torch.from_numpy(mp.A.val).to(dev)
    B0 = torch.from_numpy(mp.B).to(dev)
    Xt = torch.from_numpy(mp.X_target).to(dev)
    # replacement every 200 iterations plus the relative trigger: with period 100 a few adjoint
    # columns of this system run 5000+ iterations (every replacement restarts the recurrences);
    # with this policy every forward and adjoint column converges in <= 1100
    opts = dict(precond="jacobi", tol=1e-10, max_it=30000, rr_period=200, rr_theta=1e-3, max_restarts=3)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one():
        flush.fill_(1.0)
        vals = vals0.clone().requires_grad_(True)
        B = B0.clone().requires_grad_(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        X = pb.sparse_solve(vals, B, rp, col, **opts)
        loss = ((X - Xt) ** 2).sum()
        loss.backward()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    times, clocks = _timed_steps(args, one)
    ms = statistics.mean(times)
    line = {"metric": "differentiable p-BiCGStab: forward + adjoint gradient time", "value": round(ms, 4),
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "convdiff2d_512x512_csr_16rhs_autograd_tol1e-10", "n": mp.A.n, "nrhs": mp.B.shape[1],
                       "replacement": {"rr_period": 200, "rr_theta": 1e-3},
                       "l2": "flushed between steps (256 MB write)"},
            "roofline": None, "e2e": {"value": None, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "clocks": clocks, "gpu_launches": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The reference arm: the oracle (there is no reference implementation; the reference is
    the paper) on the headline workload and policy, each step one complete solve by the C
    oracle on all host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import c_oracle
    c_oracle.build()
    grid = args.grid or GRID
    for _ in range(args.warmup):
        _c_oracle_solve(args.precision, grid)
    per = []
    last = None
    for _ in range(args.steps):
        last = _c_oracle_solve(args.precision, grid)
        per.append(last["seconds"] * 1e3)
    value = statistics.mean(per)
    pol = HEADLINE_POLICY[args.precision]
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(value, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "convdiff2d_%dx%d_dia5_jacobi_tol1e-10" % (grid, grid), "precision": args.precision,
                       "policy": {k: v for k, v in pol.items() if k != "mixed"}},
            "iterations": last["iterations"], "status": last["status"], "rel_res_true": last["rel_res_true"],
            "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": c_oracle.threads(), "kind": "oracle",
                             "sample": "%d complete solves by the C oracle (OpenMP, all host cores), %d iterations "
                                       "each" % (args.steps, last["iterations"]), "host": _host()},
            "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="headline variant: mixed (FP32 recurrences with FP64 restarts) or fp64")
    ap.add_argument("--max-it", type=int, default=20000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", action="store_true", help="measure the headline variant only")
    ap.add_argument("--grid", type=int, default=0, help="2D grid size per dimension (profiling of smaller cases)")
    ap.add_argument("--grid3", type=int, default=0, help="3D grid size per dimension (profiling of smaller cases)")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D 256^3 workload")
    ap.add_argument("--degree", type=int, default=2,
                    help="Neumann degree of the 3D system (profiling of sweep-dominated launches)")
    ap.add_argument("--workload", default="convdiff2d", choices=["convdiff2d", "convdiff3d", "batched", "autograd"],
                    help="convdiff2d (default): 2D convection-diffusion 1024^2 DIA headline, with the 3D 256^3 CSR "
                         "Neumann-2 system measured alongside; convdiff3d: the 3D system alone; batched: 512 banded "
                         "systems; autograd: differentiable solve, 16 RHS, forward + backward")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="keep the raw nvidia-smi clock samples in this file")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "autograd":
        run_autograd(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
