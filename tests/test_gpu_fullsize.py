"""Parity at the benchmark sizes, in the launch configuration bench.py times (default
options: automatic grid and block shape).

2D: 1024 x 1024 convection-diffusion, 5 FP64 diagonals, Jacobi, tol 1e-10.
3D: 256^3 convection-diffusion, CSR, Jacobi + Neumann degree 2, tol 1e-10.
Batched: the 512 random banded systems, mixed precision, tol 1e-8.

The oracle runs the first iterations at full size (each costs tens of milliseconds in 2D
and a few seconds in 3D), so the first iterates are compared element-wise; for the whole
solve, properties that hold at any size are checked: the status, the FP64 true residual
recomputed by the oracle's SpMV, and the iteration count against the oracle's own count
stored in tests/golden (written by tests/golden/make_oracle_iterations.py)."""
import json
import os

import numpy as np
import pytest

import oracle
import testproblems as tp
from gpu_common import gpu_solve, make_solver, oracle_sensitivity, iterate_tolerance

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def convdiff2d():
    return tp.problem_convdiff2d(1024)


@pytest.fixture(scope="module")
def convdiff3d():
    return tp.problem_convdiff3d(256)


def _true_rel(A, b, x):
    return float(np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b))


def test_convdiff2d_1024_first_iterates(convdiff2d):
    K = 8
    A = convdiff2d.A.to_scipy()
    ref, sens = oracle_sensitivity(A, convdiff2d.b, K, precond="jacobi", rr_period=100)
    tol_i = iterate_tolerance(sens)
    s = make_solver(convdiff2d, fmt="dia", tol=1e-300, max_it=K, rr_period=100)
    _, res, its, hist = gpu_solve(s, convdiff2d.b, K=K, hist_len=K)
    assert res.iterations == K
    for i in range(K):
        d = np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i])
        assert d <= tol_i[i], (i, d, tol_i[i])
    assert np.allclose(hist[:K, 0], ref.alpha[:K], rtol=1e-8, atol=0)
    assert np.allclose(hist[:K, 1], ref.omega[:K], rtol=1e-8, atol=0)


@pytest.mark.parametrize("method", ["pipelined", "classic"])
def test_convdiff2d_1024_full_solve(convdiff2d, method):
    golden = json.load(open(os.path.join(HERE, "golden", "oracle_iterations_convdiff2d_1024.json")))["fp64_rr100"]
    A = convdiff2d.A.to_scipy()
    kw = dict(rr_period=100) if method == "pipelined" else {}
    s = make_solver(convdiff2d, fmt="dia", tol=1e-10, max_it=20000, method=method, **kw)
    x, res, _, _ = gpu_solve(s, convdiff2d.b)
    assert res.status == 0, res.as_dict()
    true = _true_rel(A, convdiff2d.b, x)
    assert true <= 1e-10
    assert abs(true - res.rel_res_true) <= 1e-3 * true
    if method == "pipelined":
        # the count is multi-modal under rounding (see the smaller-grid tests); the oracle
        # needed 3608 on this system
        assert golden["iterations"] // 2 <= res.iterations <= 1.25 * golden["iterations"], res.iterations
        assert res.n_replacements >= 1


def test_convdiff3d_256_first_iterates(convdiff3d):
    """Three iterations of Algorithm 2 with Neumann(2) at 16.7M rows.  On this operator the
    oracle's self-sensitivity is below 1e-14 at iterate 3 (8e-13 at iterate 20 on 24^3), so
    the 1e-10 floor of the iterate tolerance applies."""
    K = 3
    A = convdiff3d.A.to_scipy()
    ref = oracle.pbicgstab(A, convdiff3d.b, precond="neumann", degree=2, tol=1e-300, maxit=K, record=K, rr_period=100)
    s = make_solver(convdiff3d, fmt="csr", tol=1e-300, max_it=K, rr_period=100)
    _, res, its, hist = gpu_solve(s, convdiff3d.b, K=K, hist_len=K)
    assert res.iterations == K
    for i in range(K):
        d = np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i])
        assert d <= 1e-10, (i, d)
    assert np.allclose(hist[:K, 0], ref.alpha[:K], rtol=1e-10, atol=0)
    assert np.allclose(hist[:K, 1], ref.omega[:K], rtol=1e-10, atol=0)


def test_convdiff2d_1024_mixed_restarts_reach_1e10_before_fp64(convdiff2d):
    """The benchmark's headline comparison at full size, with its options: mixed precision
    restarted every 50 iterations (reading R20) reaches a 1e-10 true residual, in less
    kernel time than FP64 restarted every 100; the C oracle's mixed emulation with the same
    policy converges in a comparable number of iterations."""
    from oracle import c_oracle
    A = convdiff2d.A.to_scipy()
    out = {}
    for precision, P in (("mixed", 50), ("fp64", 100)):
        s = make_solver(convdiff2d, fmt="dia", precision=precision, tol=1e-10, max_it=20000, restart_period=P,
                        stag_window=4000)
        x, res, _, _ = gpu_solve(s, convdiff2d.b)
        assert res.status == 0, (precision, res.as_dict())
        true = _true_rel(A, convdiff2d.b, x)
        assert true <= 1e-10 and abs(true - res.rel_res_true) <= 1e-3 * true
        out[precision] = res
    print("mixed %d it. %.1f ms, fp64 %d it. %.1f ms" % (out["mixed"].iterations, out["mixed"].time_ms,
                                                        out["fp64"].iterations, out["fp64"].time_ms))
    assert out["mixed"].time_ms < out["fp64"].time_ms
    _, r = c_oracle.pbicgstab(A, convdiff2d.b, precond="jacobi", mixed=True, tol=1e-10, maxit=20000,
                              restart_period=50, stag_window=4000)
    assert r["status"] == "OK"
    assert out["mixed"].iterations <= 2 * r["iterations"] + 200 and r["iterations"] <= 2 * out["mixed"].iterations + 200


@pytest.mark.parametrize("precision,kw", [("fp64", dict(rr_period=100)), ("mixed", dict(rr_theta=3e-3)),
                                          ("mixed", dict(restart_period=75, stag_window=4000))])
def test_convdiff3d_256_full_solve(convdiff3d, precision, kw):
    A = convdiff3d.A.to_scipy()
    s = make_solver(convdiff3d, fmt="csr", precision=precision, tol=1e-10, max_it=2000, **kw)
    x, res, _, _ = gpu_solve(s, convdiff3d.b)
    assert res.status == 0, res.as_dict()
    true = _true_rel(A, convdiff3d.b, x)
    assert true <= 1e-10
    assert abs(true - res.rel_res_true) <= 1e-3 * true
    assert 150 <= res.iterations <= 600, res.iterations


def test_convdiff2d_1024_automated_replacement_schedule(convdiff2d):
    """Eq. (criterion) at full size: over the first 150 iterations the GPU replaces in the
    same iterations as the oracle (both compute the bound f^r of Eq. DDr_bound from the same
    norms and constants).  On this system the criterion fires every 6-15 iterations from the
    start and the solve eventually diverges, in the oracle as on the GPU (the design notes
    record it); only the schedule is compared here."""
    K = 150
    A = convdiff2d.A.to_scipy()
    ref = oracle.pbicgstab(A, convdiff2d.b, precond="jacobi", tol=1e-300, maxit=K, rr_auto=True)
    s = make_solver(convdiff2d, fmt="dia", tol=1e-300, max_it=K, rr_auto=True)
    _, res, _, hist = gpu_solve(s, convdiff2d.b, hist_len=K)
    rep_gpu = [i for i in range(res.iterations) if hist[i, 4] == 1.0]
    rep_ref = [i for i, f in enumerate(ref.replaced) if f]
    assert len(rep_ref) >= 8
    assert rep_gpu[:8] == rep_ref[:8], (rep_gpu, rep_ref)


def test_batched_512_systems_full_size():
    """The batched workload at full size (512 random banded systems, 17.7M rows), with the
    benchmark's options and autotuned launch: every system converges with its FP64 true
    residual (recomputed here by the oracle's SpMV) below 1e-8, and on the largest, the
    median and the smallest system the solution matches the oracle's mixed-precision
    solve and the generating x* to 1e-6 (both solves stop at a 1e-8 true residual; these
    diagonally dominant systems have condition numbers of order ten)."""
    import torch
    import paper_1809_01948_gb300 as pb
    bp = tp.problem_batched_banded()
    c = bp.concat()
    dev = torch.device("cuda:0")
    s = pb.BatchSolver(c["row_off"], c["nnz_off"], torch.from_numpy(c["row_ptr"]).to(dev),
                       torch.from_numpy(c["col"]).to(dev), torch.from_numpy(c["val"]).to(dev), precond="jacobi",
                       precision="mixed", tol=1e-8, max_it=1000, rr_theta=1e-3)
    x, info = s.solve(torch.from_numpy(c["b"]).to(dev))
    x = x.cpu().numpy()
    s.close()
    assert info["n_ok"] == 512 and np.all(info["status"] == 0)
    assert np.max(info["rel_res_true"]) <= 1e-8 * (1 + 1e-12)   # OK means ||b - A x|| <= tol ||b||
    sizes = np.diff(c["row_off"])
    order = np.argsort(sizes)
    for k, sysk in enumerate(bp.systems):
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        assert _true_rel(sysk.A.to_scipy(np.float64), sysk.b, xk) <= 1.01e-8, k
    for k in (order[-1], order[len(order) // 2], order[0]):
        sysk = bp.systems[k]
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        ref = oracle.pbicgstab(sysk.A.to_scipy(np.float64), sysk.b, precond="jacobi", tol=1e-8, maxit=1000,
                               rr_theta=1e-3, mixed=True)
        assert ref.status == oracle.Status.OK
        assert np.linalg.norm(xk - ref.x) <= 1e-6 * np.linalg.norm(ref.x), k
        assert np.linalg.norm(xk - sysk.x_star) <= 1e-6 * np.linalg.norm(sysk.x_star), k
