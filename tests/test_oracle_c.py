"""The C oracle (oracle/c_oracle.c, all host cores) against the numpy oracle it restates.

Both evaluate Algorithm 2 with the same readings and brackets; they differ only in the
summation order of the dot products (OpenMP thread blocks vs BLAS), so iterates agree to
the numpy oracle's own sensitivity to that order, and statuses, replacement / restart
counts and final residuals agree as on the GPU.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import c_oracle, krylov
import testproblems as tp
from gpu_common import oracle_sensitivity, iterate_tolerance

CASES = {
    "poisson_100_none": (lambda: tp.problem_poisson2d(), {}),
    "convdiff2d_64_jacobi_rr25": (lambda: tp.problem_convdiff2d(64), dict(rr_period=25)),
    "convdiff3d_12_neumann2_rr100": (lambda: tp.problem_convdiff3d(12), dict(rr_period=100)),
    "convdiff2d_64_restart7": (lambda: tp.problem_convdiff2d(64), dict(restart_period=7)),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    c_oracle.build()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("threads", [1, 4])
def test_fp64_iterate_after_20_iterations(name, threads):
    maker, kw = CASES[name]
    prob = maker()
    A = prob.A.to_scipy()
    K = 20
    ref, sens = oracle_sensitivity(A, prob.b, K, precond=prob.precond, degree=prob.degree, **kw)
    x, r = c_oracle.pbicgstab(A, prob.b, precond=prob.precond, degree=prob.degree, tol=1e-300, maxit=K,
                              threads=threads, **kw)
    assert r["iterations"] == K and r["n_replacements"] == ref.n_replacements and r["n_restarts"] == ref.n_restarts
    d = np.linalg.norm(x - ref.xs[K - 1]) / np.linalg.norm(ref.xs[K - 1])
    assert d <= iterate_tolerance(sens)[K - 1], (d, sens[K - 1])


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_solve_agrees(name):
    maker, kw = CASES[name]
    prob = maker()
    A = prob.A.to_scipy()
    ref = oracle.pbicgstab(A, prob.b, precond=prob.precond, degree=prob.degree, tol=prob.tol, maxit=5000, **kw)
    x, r = c_oracle.pbicgstab(A, prob.b, precond=prob.precond, degree=prob.degree, tol=prob.tol, maxit=5000,
                              threads=4, **kw)
    assert r["status"] == ref.status.name
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert abs(true - r["rel_res_true"]) <= 1e-6 * true
    assert true <= 10 * max(ref.rel_res_true, 1e-16)
    assert abs(r["iterations"] - ref.iterations) <= max(5, 0.25 * ref.iterations)


def test_mixed_twenty_iterates_track_the_numpy_emulation():
    """Mixed emulation: the two oracles order the FP64 dot sums differently; the FP32
    iterates then differ by about the emulation's sensitivity to single roundings."""
    prob = tp.problem_poisson2d(100)
    A = prob.A.to_scipy()
    K = 20
    ref = oracle.pbicgstab(A, prob.b, tol=1e-300, maxit=K, record=K, mixed=True)
    alt = oracle.pbicgstab(A, prob.b, tol=1e-300, maxit=K, record=K, mixed=True, contract=True)
    sens = np.linalg.norm(ref.xs[K - 1] - alt.xs[K - 1]) / np.linalg.norm(ref.xs[K - 1])
    x, r = c_oracle.pbicgstab(A, prob.b, mixed=True, tol=1e-300, maxit=K, threads=4)
    d = np.linalg.norm(x - ref.xs[K - 1]) / np.linalg.norm(ref.xs[K - 1])
    assert d <= max(1e-6, 20 * sens), (d, sens)


@pytest.mark.parametrize("grid", [64, 128])
def test_mixed_restart_solve_agrees(grid):
    prob = tp.problem_convdiff2d(grid)
    A = prob.A.to_scipy()
    kw = dict(restart_period=75, stag_window=4000)
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-10, maxit=8000, mixed=True, **kw)
    x, r = c_oracle.pbicgstab(A, prob.b, precond="jacobi", mixed=True, tol=1e-10, maxit=8000, threads=4, **kw)
    assert r["status"] == ref.status.name == "OK"
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert true <= 1e-10
    assert r["iterations"] <= 2 * ref.iterations + 100 and ref.iterations <= 2 * r["iterations"] + 100


def test_stagnation_window_agrees():
    prob = tp.problem_convdiff2d(64)
    A = prob.A.to_scipy()
    kw = dict(restart_period=50, stag_window=300)
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-17, maxit=5000, **kw)
    x, r = c_oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-17, maxit=5000, threads=4, **kw)
    assert r["status"] == ref.status.name == "STAGNATED"
    assert r["rel_res_true"] <= 10 * max(ref.rel_res_true, 1e-16)


def test_zero_rhs_and_host_bandwidth():
    prob = tp.problem_convdiff2d(16)
    x, r = c_oracle.pbicgstab(prob.A.to_scipy(), np.zeros(prob.A.n), x0=np.ones(prob.A.n), precond="jacobi")
    assert r["status"] == "OK" and r["iterations"] == 0 and np.all(x == 0)
    assert c_oracle.host_copy_gbs(1 << 22, 2) > 0.0 and c_oracle.threads() >= 1
