"""GPU parity tests: the CUDA p-BiCGStab (through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import testproblems as tp
from gpu_common import gpu_solve, make_solver, oracle_sensitivity, iterate_tolerance, torch_cuda, oracle_iteration_spread

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("which", ["poisson_csr", "upwind_dia", "upwind3d_csr", "random_f32_csr"])
def test_spmv_matches_oracle(which):
    torch = torch_cuda()
    if which == "poisson_csr":
        prob, fmt = tp.problem_poisson2d(37), "csr"
    elif which == "upwind_dia":
        prob, fmt = tp.problem_convdiff2d(45), "dia"
    elif which == "upwind3d_csr":
        prob, fmt = tp.problem_convdiff3d(13), "csr"
    else:
        rng = np.random.Generator(np.random.PCG64(9))
        A = tp.random_banded_system(5000, rng)
        prob = tp.Problem("rb", A, np.zeros(A.n), np.zeros(A.n), None, precond="jacobi", fmt="csr")
        fmt = "csr"
    s = make_solver(prob, fmt=fmt)
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.standard_normal(prob.A.n)
    y = s.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.spmv(prob.A.to_scipy(np.float64), x)
    assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)


# ------------------------------------------------------------------ FP64 iterates
CASES = {
    "poisson_100x100": (lambda: tp.problem_poisson2d(), "csr", {}),
    "convdiff2d_128_dia": (lambda: tp.problem_convdiff2d(128), "dia", dict(rr_period=100)),
    "convdiff2d_97_csr_ragged": (lambda: tp.problem_convdiff2d(97), "csr", dict(rr_period=100)),
    "convdiff3d_24_neumann2": (lambda: tp.problem_convdiff3d(24), "csr", dict(rr_period=100)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_iterates_match_oracle(name):
    maker, fmt, kw = CASES[name]
    prob = maker()
    K = 20
    A = prob.A.to_scipy()
    ref, sens = oracle_sensitivity(A, prob.b, K, precond=prob.precond, degree=prob.degree, **kw)
    tol_i = iterate_tolerance(sens)
    s = make_solver(prob, fmt=fmt, tol=1e-300, max_it=K, **kw)
    x, res, its, hist = gpu_solve(s, prob.b, K=K, hist_len=K)
    assert res.iterations == K
    d = np.array([np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i]) for i in range(K)])
    print("%s: applied tolerance per iterate %s; largest d/tol %.3f"
          % (name, np.array2string(tol_i, precision=1), float(np.max(d / tol_i))))
    for i in range(K):
        assert d[i] <= tol_i[i], (i, d[i], tol_i[i])
    # scalars alpha_i, omega_i agree as well (first 10 iterations)
    assert np.allclose(hist[:10, 0], ref.alpha[:10], rtol=1e-8, atol=0)
    assert np.allclose(hist[:10, 1], ref.omega[:10], rtol=1e-8, atol=0)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_final_true_residual(name):
    maker, fmt, kw = CASES[name]
    prob = maker()
    A = prob.A.to_scipy()
    refs = oracle_iteration_spread(A, prob.b, precond=prob.precond, degree=prob.degree, tol=prob.tol,
                                   maxit=5000, **kw)
    ref = refs[0]
    s = make_solver(prob, fmt=fmt, tol=prob.tol, max_it=5000, **kw)
    x, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == int(ref.status), (res.as_dict(), ref.status)
    # the reported true residual is the FP64 ||b - A x|| / ||b|| of the returned x
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert abs(true - res.rel_res_true) <= 1e-3 * true + 1e-18
    assert true <= 10 * max(max(r.rel_res_true for r in refs), 1e-16)
    if ref.status == oracle.Status.OK:
        assert true <= prob.tol
    # iteration counts: on the 2D convection-diffusion grids the count is multi-modal
    # under rounding (the oracle alone gives 192..360 on 97x97 depending on its dot
    # summation order), so only a sanity band around the oracle's spread is checked.
    lo = min(r.iterations for r in refs)
    hi = max(r.iterations for r in refs)
    assert lo // 2 <= res.iterations <= 1.25 * hi + 5, (res.iterations, lo, hi)


def test_replacement_schedule_matches_oracle():
    prob = tp.problem_convdiff2d(64)
    A = prob.A.to_scipy()
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-12, maxit=400, rr_period=25)
    s = make_solver(prob, fmt="dia", tol=1e-12, max_it=400, rr_period=25)
    _, res, _, hist = gpu_solve(s, prob.b, hist_len=400)
    n_it = res.iterations
    rep_gpu = [i for i in range(n_it) if hist[i, 4] == 1.0]
    rep_ref = [i for i, f in enumerate(ref.replaced) if f]
    assert rep_gpu == rep_ref
    assert res.n_replacements == ref.n_replacements


# ------------------------------------------------------------------ mixed precision
def test_mixed_first_iterates_track_oracle_emulation():
    prob = tp.problem_convdiff2d(64)
    A = prob.A.to_scipy()
    K = 6
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-300, maxit=K, record=K, mixed=True)
    s = make_solver(prob, precision="mixed", fmt="dia", tol=1e-300, max_it=K)
    _, res, its, _ = gpu_solve(s, prob.b, K=K)
    for i in range(K):
        d = np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i])
        assert d <= 1e-4, (i, d)


def test_mixed_reaches_tolerance_with_replacement():
    prob = tp.problem_convdiff2d(64)
    A = prob.A.to_scipy()
    s = make_solver(prob, precision="mixed", fmt="dia", tol=1e-10, max_it=3000, rr_theta=1e-3)
    x, res, _, _ = gpu_solve(s, prob.b)
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert res.status == 0 and true <= 1e-10, res.as_dict()
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-10, maxit=3000, mixed=True, rr_theta=1e-3)
    assert true <= 10 * max(ref.rel_res_true, 1e-16)


# ------------------------------------------------------------------ edge cases
def test_zero_rhs_gives_zero():
    prob = tp.problem_convdiff2d(20)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=100)
    x, res, _, _ = gpu_solve(s, np.zeros(prob.A.n), x0=np.ones(prob.A.n))
    assert res.status == 0 and res.iterations == 0 and np.all(x == 0)


def test_exact_initial_guess():
    prob = tp.problem_convdiff2d(20)
    xd = np.linalg.solve(prob.A.to_scipy().toarray(), prob.b)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=100)
    x, res, _, _ = gpu_solve(s, prob.b, x0=xd)
    assert res.status == 0 and res.iterations == 0


def test_single_row_and_tiny_systems():
    for n in (1, 2, 3, 33):
        A = tp.stencil_2d(n, 1, dict(centre=4.0, west=-1.0, east=-1.5, south=0.0, north=0.0))
        b = np.arange(1, n + 1, dtype=np.float64)
        prob = tp.Problem("tiny", A, b, np.zeros(n), None, precond="jacobi", fmt="csr")
        s = make_solver(prob, tol=1e-12, max_it=100)
        x, res, _, _ = gpu_solve(s, b)
        xd = np.linalg.solve(A.to_scipy().toarray(), b)
        assert res.status == 0 and np.allclose(x, xd, rtol=1e-10, atol=1e-12), (n, res.as_dict())


def test_max_it_zero_and_not_converged():
    prob = tp.problem_convdiff2d(32)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=0)
    _, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == 4 and res.iterations == 0
    _, res, _, _ = gpu_solve(s, prob.b, max_it=5)
    assert res.status == 4 and res.iterations == 5


def test_breakdown_reported():
    import scipy.sparse as sp
    A = tp.CSR(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    prob = tp.Problem("swap", A, np.array([1.0, 0.0]), np.zeros(2), None, precond="none", fmt="csr")
    s = make_solver(prob, tol=1e-10, max_it=10)
    x, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == 5 and np.all(np.isfinite(x))
    assert oracle.pbicgstab(sp.csr_matrix(A.to_scipy()), prob.b).status == oracle.Status.BREAKDOWN


def test_invalid_matrix_rejected():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    dev = torch.device("cuda:0")
    rp = torch.tensor([0, 2, 1, 3], dtype=torch.int32, device=dev)          # not monotone
    col = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    val = torch.ones(3, dtype=torch.float64, device=dev)
    with pytest.raises(pb.PBCGError) as e:
        pb.Solver(3, row_ptr=rp, col=col, val=val, precond="none")
    assert e.value.status == 1
    rp = torch.tensor([0, 1, 2, 3], dtype=torch.int32, device=dev)
    col = torch.tensor([0, 5, 2], dtype=torch.int32, device=dev)            # out of range
    with pytest.raises(pb.PBCGError):
        pb.Solver(3, row_ptr=rp, col=col, val=val, precond="none")
    col = torch.tensor([0, 0, 2], dtype=torch.int32, device=dev)            # zero diagonal in row 1
    with pytest.raises(pb.PBCGError):
        pb.Solver(3, row_ptr=rp, col=col, val=val, precond="jacobi")
    bad = torch.tensor([1.0, float("nan"), 1.0], dtype=torch.float64, device=dev)
    col = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    with pytest.raises(pb.PBCGError):
        pb.Solver(3, row_ptr=rp, col=col, val=bad, precond="none")


def test_deterministic_bitwise():
    prob = tp.problem_convdiff2d(100)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=3000, rr_period=100)
    x1, r1, _, _ = gpu_solve(s, prob.b)
    x2, r2, _, _ = gpu_solve(s, prob.b)
    assert np.array_equal(x1, x2) and r1.iterations == r2.iterations


def test_launch_shapes_agree():
    """Different grid sizes change only the reduction order (rounding level)."""
    prob = tp.problem_convdiff2d(80)
    A = prob.A.to_scipy()
    out = []
    for grid, threads in ((1, 256), (7, 128), (0, 0), (150, 1024)):
        s = make_solver(prob, fmt="dia", tol=1e-10, max_it=3000, rr_period=100, grid_blocks=grid,
                        block_threads=threads)
        x, res, _, _ = gpu_solve(s, prob.b)
        assert res.status == 0
        out.append(np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b))
    assert max(out) <= 1e-10


def test_barrier_timeout_is_reported_not_hung():
    torch_cuda()
    import time
    import paper_1809_01948_gb300 as pb
    t = time.time()
    st = pb.test_barrier_timeout(timeout_ms=200.0, extra_arrivals=1)
    assert st == "TIMEOUT"
    assert time.time() - t < 10.0
    # the context is still usable afterwards
    prob = tp.problem_convdiff2d(16)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=500)
    _, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == 0


def test_host_buffers_end_to_end():
    prob = tp.problem_convdiff2d(40)
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=2000, rr_period=100)
    x = np.zeros(prob.A.n)
    x, res = s.solve_host(prob.b, x)
    assert res.status == 0
    assert np.linalg.norm(prob.b - prob.A.to_scipy() @ x) / np.linalg.norm(prob.b) <= 1e-10


# ------------------------------------------------------------------ automated replacement
@pytest.mark.parametrize("name,maker,fmt,tol", [("convdiff2d_64_dia", lambda: tp.problem_convdiff2d(64), "dia", 1e-12),
                                                 ("convdiff2d_64_csr", lambda: tp.problem_convdiff2d(64), "csr", 1e-12),
                                                 ("poisson2d_100_csr", lambda: tp.problem_poisson2d(), "csr", 1e-10)])
def test_automated_replacement_schedule_matches_oracle(name, maker, fmt, tol):
    """Eq. (criterion) with the run-time bound f^r of Eq. (DDr_bound): the GPU replaces in the
    same iterations as the oracle (the bound's constants and norms agree to rounding)."""
    prob = maker()
    A = prob.A.to_scipy()
    ref = oracle.pbicgstab(A, prob.b, precond=prob.precond, tol=tol, maxit=3000, rr_auto=True)
    s = make_solver(prob, fmt=fmt, tol=tol, max_it=3000, rr_auto=True)
    x, res, _, hist = gpu_solve(s, prob.b, hist_len=3000)
    rep_gpu = [i for i in range(res.iterations) if hist[i, 4] == 1.0]
    rep_ref = [i for i, f in enumerate(ref.replaced) if f]
    assert res.status == int(ref.status) == 0, (res.as_dict(), ref.status)
    assert len(rep_ref) >= 1
    # the first replacements coincide exactly; later ones may shift by a few iterations
    # where f^r crosses tau ||r|| within the rounding of the threshold (the criterion compares
    # two nearly equal quantities once the residual nears its attainable accuracy; on
    # Poisson 100^2 a launch-shape change moved the third of eight from 57 to 56)
    assert rep_gpu[:2] == rep_ref[:2], (rep_gpu, rep_ref)
    for i in rep_gpu[:4]:
        assert min(abs(i - j) for j in rep_ref) <= 3, (rep_gpu, rep_ref)
    assert len(rep_ref) / 2 <= len(rep_gpu) <= 2 * len(rep_ref), (rep_gpu, rep_ref)
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert true <= tol


def test_automated_replacement_rejected_with_neumann():
    torch_cuda()
    import paper_1809_01948_gb300 as pb
    prob = tp.problem_convdiff3d(8)
    with pytest.raises(pb.PBCGError):
        make_solver(prob, rr_auto=True)
