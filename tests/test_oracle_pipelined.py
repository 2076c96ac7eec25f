"""Oracle pins for Algorithm 2 (p-BiCGStab): equivalence with Algorithm 1, dense solves,
preconditioner invariants, edge cases."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import testproblems as tp


def _max_rel_iterate_diff(a, b, k):
    return max(np.linalg.norm(a.xs[i] - b.xs[i]) / np.linalg.norm(a.xs[i]) for i in range(k))


def test_pipelined_equals_classic_poisson_100_first_20():
    """Section 1 / Section 3: Algorithm 2 produces the iterates of Algorithm 1 in exact
    arithmetic; in FP64 they agree to <= 1e-10 relative over the first 20 iterations
    (2D Poisson 100x100, N = 10,000, x* = 1/sqrt(N), x0 = 0, no preconditioner)."""
    p = tp.problem_poisson2d()
    A = p.A.to_scipy()
    c = oracle.bicgstab(A, p.b, tol=p.tol, maxit=20, record=20)
    q = oracle.pbicgstab(A, p.b, tol=p.tol, maxit=20, record=20)
    assert _max_rel_iterate_diff(c, q, 20) <= 1e-10
    # the scalars agree too
    assert np.allclose(c.alpha[:20], q.alpha[:20], rtol=1e-9)
    assert np.allclose(c.omega[:20], q.omega[:20], rtol=1e-9)


@pytest.mark.parametrize("prec,deg,maker", [("jacobi", 0, lambda: tp.problem_convdiff2d(48)),
                                            ("neumann", 2, lambda: tp.problem_convdiff3d(10)),
                                            ("neumann", 1, lambda: tp.problem_convdiff2d(32))])
def test_pipelined_equals_classic_preconditioned(prec, deg, maker):
    """Preconditioned equivalence.  On the convection-diffusion operators the FP64 drift
    between the two algorithms reaches 1e-10 around iteration 15 (a near-cancellation in
    one alpha), so these cases use 1e-9 over 15 iterations."""
    p = maker()
    A = p.A.to_scipy()
    c = oracle.bicgstab(A, p.b, precond=prec, degree=deg, tol=1e-30, maxit=15, record=15)
    q = oracle.pbicgstab(A, p.b, precond=prec, degree=deg, tol=1e-30, maxit=15, record=15)
    assert _max_rel_iterate_diff(c, q, 15) <= 1e-9


def test_poisson_100_outcomes():
    """Poisson 100x100, no preconditioner: classic reaches 1e-12; plain p-BiCGStab stops with its recursive residual
    below 1e-12 (and a true residual within 10x of it, reading R5)."""
    p = tp.problem_poisson2d()
    A = p.A.to_scipy()
    c = oracle.bicgstab(A, p.b, tol=1e-12, maxit=1000)
    q = oracle.pbicgstab(A, p.b, tol=1e-12, maxit=1000)
    assert c.status == oracle.Status.OK and c.rel_res_true <= 1e-12
    assert q.rel_res_recursive <= 1e-12
    assert q.rel_res_true <= 1e-11
    assert q.status in (oracle.Status.OK, oracle.Status.STAGNATED)
    # the solution is x* = 1/sqrt(N) to within the condition number times the residual
    assert np.max(np.abs(c.x - p.x_star)) < 1e-8


@pytest.mark.parametrize("prec,deg", [("none", 0), ("jacobi", 0), ("neumann", 2)])
def test_pipelined_converges_to_dense_lu(prec, deg):
    p = tp.problem_convdiff2d(14)
    A = p.A.to_scipy()
    res = oracle.pbicgstab(A, p.b, precond=prec, degree=deg, tol=1e-12, maxit=1000, rr_period=50)
    xd = np.linalg.solve(A.toarray(), p.b)
    assert res.status == oracle.Status.OK
    assert np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert res.rel_res_true <= 1e-12


def test_jacobi_scale_invariance_constant_diagonal():
    """With a constant diagonal, D^{-1} = c I, and the Krylov iterates do not depend on c:
    Jacobi-preconditioned iterates equal the unpreconditioned ones."""
    p = tp.problem_convdiff2d(40)
    A = p.A.to_scipy()
    assert np.all(A.diagonal() == A.diagonal()[0])
    a = oracle.pbicgstab(A, p.b, precond="none", tol=1e-30, maxit=20, record=20)
    j = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-30, maxit=20, record=20)
    assert _max_rel_iterate_diff(a, j, 20) <= 1e-12


def test_neumann_matches_explicit_polynomial():
    """M^{-1} = sum_{j=0..d} (I - D^{-1} A)^j D^{-1} (dense closed form) vs the Horner recursion."""
    p = tp.problem_convdiff2d(6)
    A = p.A.to_scipy()
    Ad = A.toarray()
    Dinv = np.diag(1.0 / np.diag(Ad))
    Nm = np.eye(A.shape[0]) - Dinv @ Ad
    rng = np.random.Generator(np.random.PCG64(3))
    v = rng.standard_normal(A.shape[0])
    for d in range(4):
        M = oracle.make_precond("neumann", A, d)
        expect = sum(np.linalg.matrix_power(Nm, j) for j in range(d + 1)) @ Dinv @ v
        assert np.allclose(M.apply(v), expect, rtol=1e-13, atol=1e-15)
    # degree 0 is Jacobi
    J = oracle.make_precond("jacobi", A)
    assert np.array_equal(oracle.make_precond("neumann", A, 0).apply(v), J.apply(v))


def test_zero_rhs_and_exact_start():
    p = tp.problem_convdiff2d(8)
    A = p.A.to_scipy()
    r = oracle.pbicgstab(A, np.zeros(A.shape[0]), precond="jacobi")
    assert r.status == oracle.Status.OK and r.iterations == 0 and np.all(r.x == 0)
    xd = np.linalg.solve(A.toarray(), p.b)
    r2 = oracle.pbicgstab(A, p.b, x0=xd, precond="jacobi", tol=1e-10)
    assert r2.status == oracle.Status.OK and r2.iterations == 0


def test_breakdown_detected():
    """(r_0, w_0) = 0 makes alpha_0 undefined: A = [[0,1],[1,0]], b = e_1."""
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))
    r = oracle.pbicgstab(A, np.array([1.0, 0.0]))
    assert r.status == oracle.Status.BREAKDOWN
    assert np.all(np.isfinite(r.x))


def test_maxit_not_converged():
    p = tp.problem_convdiff2d(32)
    r = oracle.pbicgstab(p.A.to_scipy(), p.b, precond="jacobi", tol=1e-10, maxit=5)
    assert r.status == oracle.Status.NOT_CONVERGED and r.iterations == 5


def test_record_and_history_lengths():
    p = tp.problem_convdiff2d(16)
    r = oracle.pbicgstab(p.A.to_scipy(), p.b, precond="jacobi", tol=1e-10, maxit=200, record=7)
    assert len(r.xs) == 7 and len(r.alpha) == r.iterations and len(r.rnorm) == r.iterations
    assert np.isclose(r.rnorm[-1] / np.linalg.norm(p.b), r.rel_res_recursive)
