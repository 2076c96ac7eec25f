"""GPU parity of the replacement and restart policies (through the C ABI) against the oracle.

* Iterates across actual Eq. (rr) replacements (period 5, 20 iterations): x, alpha, omega,
  beta and ||r|| after each iteration.
* The six vectors Eq. (rr) recomputes, read back right after a replacement: the identities
  r = b - A x, k = M^{-1} r, w = A k, s = A g, l = M^{-1} s, z = A l on the GPU's own state,
  and element-wise agreement with the oracle's replaced vectors.
* Periodic restarts (reading R20) in FP64: iterates across restarts; in mixed precision: the
  2D convection-diffusion solve that the FP32 recurrences alone do not converge on.
* Progress-based stagnation (reading R21) with the best-iterate fallback.
* Mixed precision: 20 iterates against the emulation, with a tolerance derived from the
  emulation's own sensitivity to the rounding of single FP32 operations, and the FP64
  accumulation of FP32 dot products (a plain FP32 accumulation fails it).

Every iterate test prints the tolerance it applied (pytest -s shows it)."""
import numpy as np
import pytest

import oracle
from oracle import krylov
from oracle.precond import make_precond
import testproblems as tp
from gpu_common import gpu_solve, make_solver, oracle_sensitivity, iterate_tolerance, torch_cuda

pytestmark = pytest.mark.gpu

RR_CASES = {
    "poisson_100x100_csr": (lambda: tp.problem_poisson2d(), "csr"),
    "convdiff2d_128_dia_jacobi": (lambda: tp.problem_convdiff2d(128), "dia"),
    "convdiff3d_24_csr_neumann2": (lambda: tp.problem_convdiff3d(24), "csr"),
}


def _report(name, d, tol):
    worst = int(np.argmax(d / tol))
    print("%s: applied tolerance per iterate %s; largest d/tol %.3f at iterate %d"
          % (name, np.array2string(tol, precision=1), d[worst] / tol[worst], worst))


@pytest.mark.parametrize("name", list(RR_CASES))
def test_iterates_across_replacements_match_oracle(name):
    """rr_period = 5: replacements in iterations 5, 10 and 15 of the 20 compared."""
    maker, fmt = RR_CASES[name]
    prob = maker()
    K = 20
    A = prob.A.to_scipy()
    kw = dict(rr_period=5)
    ref, sens = oracle_sensitivity(A, prob.b, K, precond=prob.precond, degree=prob.degree, **kw)
    assert [i for i, f in enumerate(ref.replaced) if f] == [5, 10, 15]
    tol_i = iterate_tolerance(sens)
    s = make_solver(prob, fmt=fmt, tol=1e-300, max_it=K, **kw)
    x, res, its, hist = gpu_solve(s, prob.b, K=K, hist_len=K)
    assert res.iterations == K and res.n_replacements == 3
    d = np.array([np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i]) for i in range(K)])
    _report(name, d, tol_i)
    assert np.all(d <= tol_i), (d, tol_i)
    assert [i for i in range(K) if hist[i, 4] == 1.0] == [5, 10, 15]
    # scalars and recursive residual norms, element-wise, through all three replacements
    bn = np.linalg.norm(prob.b)
    for i in range(K):
        st = max(1e-8, 1e4 * tol_i[i])   # scalar tolerance scaled like the iterate one
        assert abs(hist[i, 0] - ref.alpha[i]) <= st * abs(ref.alpha[i]), ("alpha", i)
        assert abs(hist[i, 1] - ref.omega[i]) <= st * abs(ref.omega[i]), ("omega", i)
        assert abs(hist[i, 3] - ref.rnorm[i] / bn) <= st * ref.rnorm[i] / bn, ("rnorm", i)
        if i < K - 1:
            assert abs(hist[i, 2] - ref.beta[i]) <= st * abs(ref.beta[i]), ("beta", i)


def _apply_M(prob, A, v):
    return make_precond(prob.precond, A, prob.degree, np.float64).apply(v)


@pytest.mark.parametrize("name", list(RR_CASES))
def test_replaced_vectors_right_after_eq_rr(name):
    """max_it = 6 with rr_period = 5: the solve ends right after iteration 5's replacement,
    so the work vectors are the replaced r_6, k_6, w_6, s_5, l_5, z_5 (and g_5)."""
    torch = torch_cuda()
    maker, fmt = RR_CASES[name]
    prob = maker()
    A = prob.A.to_scipy()
    got = {}

    def obs(stage, i, v):
        if stage == "replace" and i == 5:
            got.update({k: np.array(v[k], dtype=np.float64) for k in ("x", "r", "k", "w", "g", "s", "l", "z")})

    krylov.pbicgstab(A, prob.b, precond=prob.precond, degree=prob.degree, tol=1e-300, maxit=6, rr_period=5,
                     observer=obs)
    assert got, "the oracle did not replace in iteration 5"
    s = make_solver(prob, fmt=fmt, tol=1e-300, max_it=6, rr_period=5)
    x, res, _, _ = gpu_solve(s, prob.b)
    assert res.n_replacements == 1 and res.iterations == 6
    vec = {k: s.get_vector(k).cpu().numpy() for k in ("r", "k", "w", "g", "s", "l", "z")}
    torch.cuda.synchronize()
    rel = lambda a, b_: np.linalg.norm(a - b_) / max(np.linalg.norm(b_), 1e-300)
    # Eq. (rr) on the GPU's own state, in FP64 (rounding of one SpMV / preconditioner application)
    assert rel(vec["r"], prob.b - A @ x) <= 1e-13
    assert rel(vec["k"], _apply_M(prob, A, vec["r"])) <= 1e-13
    assert rel(vec["w"], A @ vec["k"]) <= 1e-13
    assert rel(vec["s"], A @ vec["g"]) <= 1e-13
    assert rel(vec["l"], _apply_M(prob, A, vec["s"])) <= 1e-13
    assert rel(vec["z"], A @ vec["l"]) <= 1e-13
    # element-wise against the oracle's replaced vectors (6 iterations of rounding apart)
    _, sens = oracle_sensitivity(A, prob.b, 6, precond=prob.precond, degree=prob.degree, rr_period=5)
    tol = float(iterate_tolerance(sens)[-1])
    print("%s: tolerance of the replaced vectors %.1e" % (name, tol))
    assert rel(x, got["x"]) <= tol
    # the replaced vectors are products of x and g, whose rounding differences they inherit,
    # amplified where a product cancels (r = b - A x is small): a gross slip (say s = A k)
    # makes them differ by O(1), far above this bound
    vtol = max(1e-8, 1e4 * tol)
    for k in ("r", "k", "w", "g", "s", "l", "z"):
        assert rel(vec[k], got[k]) <= vtol, (k, rel(vec[k], got[k]), vtol)


def test_fp64_iterates_across_restarts_match_oracle():
    """restart_period = 7: restarts after iterations 7 and 14 (new shadow vector, beta = 0)."""
    prob = tp.problem_convdiff2d(128)
    A = prob.A.to_scipy()
    K = 20
    kw = dict(restart_period=7)
    ref, sens = oracle_sensitivity(A, prob.b, K, precond="jacobi", **kw)
    assert ref.n_restarts == 2
    tol_i = iterate_tolerance(sens)
    s = make_solver(prob, fmt="dia", tol=1e-300, max_it=K, **kw)
    x, res, its, hist = gpu_solve(s, prob.b, K=K, hist_len=K)
    assert res.iterations == K and res.n_restarts == 2
    d = np.array([np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i]) for i in range(K)])
    _report("convdiff2d_128 restarts", d, tol_i)
    assert np.all(d <= tol_i)
    # the first iteration of each cycle has beta = 0 on both sides (alpha, omega agree)
    for i in (7, 14):
        assert abs(hist[i, 0] - ref.alpha[i]) <= 1e-8 * abs(ref.alpha[i])
        assert abs(hist[i, 1] - ref.omega[i]) <= 1e-8 * abs(ref.omega[i])


@pytest.mark.parametrize("grid", [128, 256])
def test_mixed_with_restarts_reaches_1e10_on_convdiff2d(grid):
    """FP32 recurrences restarted from the FP64 residual every 100 iterations reach 1e-10 on
    the 2D convection-diffusion system (the emulation does too, in a comparable count)."""
    prob = tp.problem_convdiff2d(grid)
    A = prob.A.to_scipy()
    kw = dict(restart_period=100, stag_window=2000)
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-10, maxit=8000, mixed=True, **kw)
    assert ref.status == oracle.Status.OK
    s = make_solver(prob, precision="mixed", fmt="dia", tol=1e-10, max_it=8000, **kw)
    x, res, _, _ = gpu_solve(s, prob.b)
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    print("grid %d: GPU %d iterations (%d restarts), oracle %d (%d)" % (grid, res.iterations, res.n_restarts,
                                                                      ref.iterations, ref.n_restarts))
    assert res.status == 0 and true <= 1e-10, res.as_dict()
    assert abs(true - res.rel_res_true) <= 1e-3 * true
    assert res.iterations <= 2 * ref.iterations + 200


def test_stagnation_window_returns_best_iterate():
    """tol 1e-17 is below the attainable accuracy: with restarts every 50 iterations the true
    residual stops halving, and the solve returns STAGNATED within the window with the best
    (re)start iterate, as the oracle does."""
    prob = tp.problem_convdiff2d(64)
    A = prob.A.to_scipy()
    kw = dict(restart_period=50, stag_window=300)
    ref = oracle.pbicgstab(A, prob.b, precond="jacobi", tol=1e-17, maxit=5000, **kw)
    assert ref.status == oracle.Status.STAGNATED and ref.iterations < 5000
    s = make_solver(prob, fmt="dia", tol=1e-17, max_it=5000, **kw)
    x, res, _, _ = gpu_solve(s, prob.b)
    true = np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)
    print("GPU stagnated after %d iterations at %.2e; oracle after %d at %.2e"
          % (res.iterations, true, ref.iterations, ref.rel_res_true))
    assert res.status == oracle.Status.STAGNATED
    assert res.iterations < 5000
    assert true <= 10 * max(ref.rel_res_true, 1e-16)


def test_mixed_twenty_iterates_track_emulation():
    """Poisson 100^2, no preconditioner, 20 iterations.  Tolerance per iterate: 20 x the
    difference between the emulation and the same emulation with one rounding per FP32
    a + s c and row product (both valid evaluations of the FP32 iteration), floor 1e-6."""
    prob = tp.problem_poisson2d(100)
    A = prob.A.to_scipy()
    K = 20
    ref = oracle.pbicgstab(A, prob.b, precond="none", tol=1e-300, maxit=K, record=K, mixed=True)
    alt = oracle.pbicgstab(A, prob.b, precond="none", tol=1e-300, maxit=K, record=K, mixed=True, contract=True)
    sens = np.array([np.linalg.norm(ref.xs[i] - alt.xs[i]) / np.linalg.norm(ref.xs[i]) for i in range(K)])
    tol_i = iterate_tolerance(sens, floor=1e-6, factor=20.0)
    s = make_solver(prob, precision="mixed", fmt="csr", tol=1e-300, max_it=K)
    _, res, its, _ = gpu_solve(s, prob.b, K=K)
    d = np.array([np.linalg.norm(its[i] - ref.xs[i]) / np.linalg.norm(ref.xs[i]) for i in range(K)])
    _report("poisson_100 mixed", d, tol_i)
    assert np.all(d <= tol_i)


def test_mixed_dot_products_accumulate_beyond_fp32():
    """||r_0|| of an FP32 residual vector, computed by the kernel's mixed-precision dot
    product (exact FP32 products summed in about 48 bits per thread, then FP64), agrees with
    the FP64 norm of the same FP32 vector to 1e-11.  With 128 threads, each accumulates 32
    products: a plain FP32 accumulation would be off by about 1e-7."""
    torch = torch_cuda()
    prob = tp.problem_convdiff2d(64)
    s = make_solver(prob, precision="mixed", fmt="dia", tol=1e-300, max_it=0, grid_blocks=1, block_threads=128)
    _, res, _, _ = gpu_solve(s, prob.b)
    r0 = prob.b.astype(np.float32).astype(np.float64)   # x0 = 0: r_0 = fl32(b)
    want = np.sqrt(np.dot(r0, r0)) / np.linalg.norm(prob.b)
    assert res.status == oracle.Status.NOT_CONVERGED and res.iterations == 0
    assert abs(res.rel_res_recursive - want) <= 1e-11 * want, (res.rel_res_recursive, want)
