"""GPU parity tests of classic BiCGStab (Algorithm 1, options.method = PBCG_CLASSIC)
through the C ABI against the oracle's ``bicgstab``."""
import numpy as np
import pytest

import oracle
import testproblems as tp
from gpu_common import gpu_solve, make_solver, oracle_sensitivity, iterate_tolerance, torch_cuda, oracle_iteration_spread

pytestmark = pytest.mark.gpu

CASES = {
    "poisson_100x100_jacobi_csr": (lambda: tp.problem_poisson2d(), "csr", "jacobi"),
    "convdiff_128_jacobi_dia": (lambda: tp.problem_convdiff2d(128), "dia", "jacobi"),
    "convdiff_97_jacobi_csr_ragged": (lambda: tp.problem_convdiff2d(97), "csr", "jacobi"),
    "convdiff_64_none_dia": (lambda: tp.problem_convdiff2d(64), "dia", "none"),
}


def classic_solver(prob, fmt, precond, **kw):
    return make_solver(prob, fmt=fmt, method="classic", precond=precond, degree=0, **kw)


@pytest.mark.parametrize("name", list(CASES))
def test_classic_iterates_match_oracle(name):
    maker, fmt, precond = CASES[name]
    prob = maker()
    K = 20
    A = prob.A.to_scipy()
    ref, sens = oracle_sensitivity(A, prob.b, K, method=oracle.bicgstab, precond=precond)
    tol_i = iterate_tolerance(sens)
    s = classic_solver(prob, fmt, precond, tol=1e-300, max_it=K)
    _, res, its, hist = gpu_solve(s, prob.b, K=K, hist_len=K)
    assert res.iterations == K and res.status == 4
    for i in range(K):
        d = np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i])
        assert d <= tol_i[i], (i, d, tol_i[i])
    assert np.allclose(hist[:10, 0], ref.alpha[:10], rtol=1e-8, atol=0)
    assert np.allclose(hist[:10, 1], ref.omega[:10], rtol=1e-8, atol=0)
    assert np.allclose(hist[:9, 2], ref.beta[:9], rtol=1e-8, atol=0)
    assert np.allclose(hist[:10, 3], np.array(ref.rnorm[:10]) / np.linalg.norm(prob.b), rtol=1e-8, atol=0)
    assert np.all(hist[:K, 4] == 0.0)   # no replacements


@pytest.mark.parametrize("name", list(CASES))
def test_classic_final_true_residual(name):
    maker, fmt, precond = CASES[name]
    prob = maker()
    A = prob.A.to_scipy()
    refs = oracle_iteration_spread(A, prob.b, method=oracle.bicgstab, precond=precond, tol=prob.tol, maxit=5000)
    ref = refs[0]
    s = classic_solver(prob, fmt, precond, tol=prob.tol, max_it=5000)
    x, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == int(ref.status), (res.as_dict(), ref.status)
    assert res.n_replacements == 0 and res.n_restarts == 0
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    assert abs(true - res.rel_res_true) <= 1e-3 * true + 1e-18
    if ref.status == oracle.Status.OK:
        assert true <= prob.tol
    lo = min(r.iterations for r in refs)
    hi = max(r.iterations for r in refs)
    assert lo // 2 <= res.iterations <= 1.25 * hi + 5, (res.iterations, lo, hi)


def test_classic_and_pipelined_reach_the_same_solution():
    """Algorithms 1 and 2 are the same method in exact arithmetic (Section 2): on a
    well-conditioned problem both converge, to the same x up to the tolerance."""
    prob = tp.problem_convdiff2d(100)
    A = prob.A.to_scipy()
    xd = np.linalg.solve(A.toarray(), prob.b)
    sc = classic_solver(prob, "dia", "jacobi", tol=1e-10, max_it=3000)
    sp_ = make_solver(prob, fmt="dia", tol=1e-10, max_it=3000, rr_period=100)
    xc, rc, _, _ = gpu_solve(sc, prob.b)
    xp, rp, _, _ = gpu_solve(sp_, prob.b)
    assert rc.status == 0 and rp.status == 0
    kappa_est = np.linalg.cond(A.toarray())
    for x in (xc, xp):
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10 * kappa_est


def test_classic_edge_cases():
    # b = 0 gives x = 0 without an iteration
    prob = tp.problem_convdiff2d(20)
    s = classic_solver(prob, "dia", "jacobi", tol=1e-10, max_it=100)
    x, res, _, _ = gpu_solve(s, np.zeros(prob.A.n), x0=np.ones(prob.A.n))
    assert res.status == 0 and res.iterations == 0 and np.all(x == 0)
    # exact initial guess
    xd = np.linalg.solve(prob.A.to_scipy().toarray(), prob.b)
    x, res, _, _ = gpu_solve(s, prob.b, x0=xd)
    assert res.status == 0 and res.iterations == 0
    # iteration limits
    _, res, _, _ = gpu_solve(s, prob.b, max_it=0)
    assert res.status == 4 and res.iterations == 0
    _, res, _, _ = gpu_solve(s, prob.b, max_it=5)
    assert res.status == 4 and res.iterations == 5
    # tiny systems, one block with mostly idle threads
    for n in (1, 2, 3, 33):
        A = tp.stencil_2d(n, 1, dict(centre=4.0, west=-1.0, east=-1.5, south=0.0, north=0.0))
        b = np.arange(1, n + 1, dtype=np.float64)
        p = tp.Problem("tiny", A, b, np.zeros(n), None, precond="jacobi", fmt="csr")
        s = classic_solver(p, "csr", "jacobi", tol=1e-12, max_it=100)
        x, res, _, _ = gpu_solve(s, b)
        assert res.status == 0 and np.allclose(x, np.linalg.solve(A.to_scipy().toarray(), b), rtol=1e-10,
                                               atol=1e-12), (n, res.as_dict())


def test_classic_breakdown_matches_oracle():
    # A = [[0,1],[1,0]], b = e1: (r0, s_0) = 0 in the first iteration
    A = tp.CSR(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    prob = tp.Problem("swap", A, np.array([1.0, 0.0]), np.zeros(2), None, precond="none", fmt="csr")
    s = classic_solver(prob, "csr", "none", tol=1e-10, max_it=10)
    x, res, _, _ = gpu_solve(s, prob.b)
    ref = oracle.bicgstab(A.to_scipy(), prob.b, tol=1e-10, maxit=10)
    assert ref.status == oracle.Status.BREAKDOWN
    assert res.status == 5 and res.iterations == ref.iterations and np.all(np.isfinite(x))


def test_classic_deterministic_and_launch_shapes():
    prob = tp.problem_convdiff2d(80)
    A = prob.A.to_scipy()
    s = classic_solver(prob, "dia", "jacobi", tol=1e-10, max_it=3000)
    x1, r1, _, _ = gpu_solve(s, prob.b)
    x2, r2, _, _ = gpu_solve(s, prob.b)
    assert np.array_equal(x1, x2) and r1.iterations == r2.iterations
    for grid, threads in ((1, 256), (7, 128), (150, 1024)):
        s = classic_solver(prob, "dia", "jacobi", tol=1e-10, max_it=3000, grid_blocks=grid, block_threads=threads)
        x, res, _, _ = gpu_solve(s, prob.b)
        assert res.status == 0
        assert np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b) <= 1e-10


def test_classic_option_rejections():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    prob = tp.problem_convdiff2d(16)
    for kw in (dict(precision="mixed"), dict(rr_period=10), dict(rr_theta=1e-3), dict(rr_auto=True),
               dict(max_restarts=1)):
        with pytest.raises(pb.PBCGError) as e:
            classic_solver(prob, "dia", "jacobi", **kw)
        assert e.value.status == 1, kw
    p3 = tp.problem_convdiff3d(8)
    with pytest.raises(pb.PBCGError):
        make_solver(p3, fmt="csr", method="classic")          # Neumann preconditioner
    s = make_solver(p3, fmt="csr")
    with pytest.raises(pb.PBCGError):
        s.set_options(method="classic")
    # a pipelined context may switch to classic and back
    s = make_solver(prob, fmt="csr", tol=1e-10, max_it=500)
    _, res, _, _ = gpu_solve(s, prob.b, method="classic")
    assert res.status == 0
    _, res, _, _ = gpu_solve(s, prob.b, method="pipelined")
    assert res.status == 0
    # the multi-RHS solver runs Algorithm 2 only
    sc = classic_solver(prob, "csr", "jacobi", tol=1e-10, max_it=500)
    B = torch.zeros(prob.A.n, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.PBCGError):
        sc.solve_multi(B)
