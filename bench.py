"""Benchmark: p-BiCGStab time to a 1e-10 true relative residual on GB300.

Workload (one "step" = one complete solve): 2D upwind convection-diffusion,
1024 x 1024 grid (N = 1,048,576), cell Peclet 0.5, matrix stored as 5 FP64
diagonals, Jacobi preconditioner, x* ~ U[0,1] (seed 2), b = A x*, x0 = 0,
tol 1e-10 on ||b - A x|| / ||b||.  The headline variant is set by --precision
(fp64 with periodic replacement every 100 iterations by default); the other
variants (mixed precision, and on the 2D workload classic BiCGStab, Algorithm 1)
are measured alongside.

Prints ONE JSON line on rank 0.  --impl reference times the CPU oracle instead
(a bounded sample of iterations, extrapolated with the oracle's iteration count
stored in tests/golden/oracle_iterations_convdiff2d_1024.json).
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
GOLDEN_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_iterations_convdiff2d_1024.json")


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
    for f in ("common.cuh", "solver.cuh", "capi.cu", "capi_internal.h", "stencil.cu"):
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
def run_gpu(args):
    import numpy as np
    import torch
    import testproblems as tp
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

    if args.workload == "convdiff2d":
        prob = tp.problem_convdiff2d(args.grid or GRID)
        off, data = tp.csr_to_dia(prob.A)
        mat = dict(offsets=off.tolist(), dia=torch.from_numpy(data).to(dev), precond="jacobi")
        workload = "convdiff2d_%dx%d_dia5_jacobi_tol1e-10" % ((args.grid or GRID), (args.grid or GRID))
    else:
        prob = tp.problem_convdiff3d(args.grid or 256)
        mat = dict(row_ptr=torch.from_numpy(prob.A.row_ptr).to(dev), col=torch.from_numpy(prob.A.col).to(dev),
                   val=torch.from_numpy(prob.A.val).to(dev), precond="neumann", degree=2)
        workload = "convdiff3d_%d^3_csr7_neumann2_tol1e-10" % (args.grid or 256)
    b = torch.from_numpy(prob.b).to(dev)
    n = prob.A.n
    variants = {
        "fp64": dict(precision="fp64", rr_period=100, rr_theta=0.0),
        "mixed": dict(precision="mixed", rr_period=args.mixed_period, rr_theta=args.theta),
    }
    if args.workload == "convdiff2d":
        # Algorithm 1, the paper's reference method, on the same system (three reduction
        # phases per iteration instead of two)
        variants["classic"] = dict(precision="fp64", method="classic", rr_period=0, rr_theta=0.0)
        # the relative replacement trigger instead of the period (fewer replacements)
        variants["fp64_theta"] = dict(precision="fp64", rr_period=0, rr_theta=1e-3)
    # the headline variant with the matrix values kept as given (CSR / DIA) instead of the
    # constant-coefficient stencil storage the library selects for these operators
    variants[args.precision + "_general"] = dict(variants[args.precision], operator_storage="general")
    solvers = {k: pb.Solver(n, tol=1e-10, max_it=args.max_it, **mat, **v) for k, v in variants.items()}
    storage = solvers[args.precision].storage
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def one(name):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, res = solvers[name].solve(b, x)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res, x

    results = {}
    clocks = None
    order = (args.precision,) + (() if args.only else tuple(k for k in variants if k != args.precision))
    for name in order:
        for _ in range(args.warmup):
            one(name)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(args.clocks_csv) if name == args.precision else None
        if sampler:
            sampler.start()
        times, ktimes, its, nrep, trues, stat = [], [], [], [], [], []
        for _ in range(args.steps):
            ms, res, x = one(name)
            times.append(ms)
            ktimes.append(res.time_ms)
            its.append(res.iterations)
            nrep.append(res.n_replacements)
            trues.append(res.rel_res_true)
            stat.append(res.status)
        torch.cuda.synchronize()
        if sampler:
            clocks = sampler.stop()
        total = max_over_ranks(sum(times), device=dev)   # replicas: the slowest rank's time
        results[name] = dict(ms_per_solve=total / args.steps, kernel_ms=statistics.mean(ktimes),
                             iterations=its[-1], n_replacements=nrep[-1], rel_res_true=max(trues),
                             status=[pb.STATUS_NAMES[s] for s in stat][-1])

    # end-to-end through the public API with host buffers (pinned)
    head = results[args.precision]
    b_pin = torch.from_numpy(prob.b).pin_memory()
    x_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for k in range(0 if args.no_e2e else max(1, args.steps)):
        x_pin.zero_()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, res = solvers[args.precision].solve_host(b_pin.numpy(), x_pin.numpy())
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": statistics.mean(e2e_times) if e2e_times else None, "unit": "ms", "h2d_bytes_per_step": 2 * 8 * n,
           "d2h_bytes_per_step": 8 * n + 64}

    # roofline of the dominant kernel (the persistent solver), per launch
    prec = args.precision
    bpr = (bytes_per_row_iteration(prec, storage=storage) if args.workload == "convdiff2d"
           else bytes_per_row_iteration_neumann(prec, storage=storage))
    alg_bytes = n * (bpr * head["iterations"] + bytes_per_row_replacement(prec, storage=storage) * head["n_replacements"])
    kernel_s = head["kernel_ms"] * 1e-3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    per_it = measured_traffic(prec, workload)
    traffic = per_it * head["iterations"] if per_it is not None else None
    hbm = {"achieved": round(alg_bytes / kernel_s / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(alg_bytes / kernel_s / 1e9 / hbm_peak, 4),
           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
           "bytes_per_row_iteration": bpr}
    # the same time against the byte model of the general (CSR / DIA values) storage, which
    # the stencil storage undercuts: the effective bandwidth of the solve
    gen = (bytes_per_row_iteration(prec, storage="general") if args.workload == "convdiff2d"
           else bytes_per_row_iteration_neumann(prec, storage="general"))
    gen_bytes = n * (gen * head["iterations"] + bytes_per_row_replacement(prec, storage="general") * head["n_replacements"])
    hbm["general_storage_model"] = {"bytes_per_row_iteration": gen,
                                    "effective_gbs": round(gen_bytes / kernel_s / 1e9, 1),
                                    "frac": round(gen_bytes / kernel_s / 1e9 / hbm_peak, 4)}
    if prec == "fp64":
        # FP64 pipe bound: GB300 runs FP64 at 1/58 of FP32; nominal 1.25 TFLOP/s (measured DFMA 1.197)
        fpr = fp64_flops_per_row_iteration() if args.workload == "convdiff2d" else fp64_flops_per_row_iteration_neumann()
        ach = fpr * n * head["iterations"] / kernel_s / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": 1.25, "unit": "TFLOP/s",
                "frac": round(ach / 1.25, 4), "traffic": traffic,
                "peak_source": "nominal FP64 rate of the profiling recipe (measured DFMA: 1.197)",
                "flops_per_row_iteration": fpr, "hbm": hbm}
    else:
        roof = {"bound": "hbm", "achieved": hbm["achieved"], "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm["frac"], "traffic": traffic, "peak_source": hbm["peak_source"],
                "bytes_per_row_iteration": bpr, "general_storage_model": hbm["general_storage_model"],
                }
        if args.workload == "convdiff2d":
            roof["note"] = "working set is L2-resident across iterations (DRAM traffic ~3 B/row/it)"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == "convdiff2d":
        cpu = cpu_baseline(args, head["iterations"], sample_iters=args.cpu_iters)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(head["ms_per_solve"], 4), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head["ms_per_solve"], 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": workload, "n": n,
                       "format": "DIA 5 diagonals FP64" if args.workload == "convdiff2d" else "CSR int32, 7 nnz/row, FP64 values",
                       "operator_storage": storage + (" (constant coefficients detected at create: one value per "
                                                      "offset + 16-bit row mask)" if storage == "stencil" else ""),
                       "precision": prec, "replacement": variants[prec], "global_batch": 1 * world,
                       "parallelism": "replicas" if world > 1 else "single", "l2": "flushed between steps (256 MB write)"},
            "iterations": head["iterations"], "n_replacements": head["n_replacements"],
            "rel_res_true": head["rel_res_true"], "status": head["status"],
            "iters_per_s": round(head["iterations"] / (head["kernel_ms"] * 1e-3), 1),
            "kernel_ms": round(head["kernel_ms"], 4),
            "variants": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                         for k, v in results.items()},
            "roofline": roof, "e2e": e2e, "clocks": clocks,
            "gpu_launches": 3 * args.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle arm
_ORACLE_SNIPPET = r"""
import json, sys, time, os
sys.path.insert(0, %(root)r)
import numpy as np
import testproblems as tp
from oracle import krylov
prob = tp.problem_convdiff2d(%(grid)d)
A = prob.A.to_scipy()
t0 = time.perf_counter()
r = krylov.pbicgstab(A, prob.b, precond="jacobi", tol=1e-300, maxit=%(iters)d, rr_period=100)
dt = time.perf_counter() - t0
print(json.dumps({"seconds": dt, "iterations": r.iterations}))
"""


def _oracle_sample(iters: int):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", _ORACLE_SNIPPET % dict(root=ROOT, grid=GRID, iters=iters)],
                         capture_output=True, text=True, env=env, timeout=900)
    if out.returncode:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _golden_iterations(default: int) -> int:
    try:
        return int(json.load(open(GOLDEN_ITERS))["fp64_rr100"]["iterations"])
    except Exception:
        return default


def cpu_baseline(args, gpu_iterations: int, sample_iters: int = 40):
    s = _oracle_sample(sample_iters)
    per_it = s["seconds"] / s["iterations"]
    iters = _golden_iterations(gpu_iterations)
    return {"value": round(per_it * iters * 1e3, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": "%d iterations of the FP64 numpy oracle on the full 1024x1024 system (%.1f s), "
                      "extrapolated to %d iterations" % (s["iterations"], s["seconds"], iters),
            "ms_per_iteration": round(per_it * 1e3, 3), "host": _host()}


def _host():
    """The machine the CPU baseline ran on (the oracle itself uses one thread)."""
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
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    for _ in range(args.warmup):
        _oracle_sample(args.cpu_iters)
    per = []
    for _ in range(args.steps):
        s = _oracle_sample(args.cpu_iters)
        per.append(s["seconds"] / s["iterations"])
    iters = _golden_iterations(2000)
    value = statistics.mean(per) * iters * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(value, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "convdiff2d_1024x1024_dia5_jacobi_tol1e-10", "precision": "fp64",
                       "replacement": {"rr_period": 100}},
            "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": "%d iterations per step of the numpy oracle, extrapolated to %d iterations"
                                       % (args.cpu_iters, iters), "host": _host()},
            "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--theta", type=float, default=3e-3, help="mixed variant: relative replacement trigger")
    ap.add_argument("--mixed-period", type=int, default=0, help="mixed variant: replacement period")
    ap.add_argument("--max-it", type=int, default=20000)
    ap.add_argument("--cpu-iters", type=int, default=40)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", action="store_true", help="measure the headline variant only")
    ap.add_argument("--grid", type=int, default=0, help="grid size per dimension (profiling of smaller cases)")
    ap.add_argument("--workload", default="convdiff2d", choices=["convdiff2d", "convdiff3d", "batched", "autograd"],
                    help="convdiff2d: 2D convection-diffusion 1024^2 DIA (default); convdiff3d: 3D 256^3 CSR "
                         "Neumann-2; batched: 512 banded systems; autograd: differentiable solve, 16 RHS, "
                         "forward + backward")
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
