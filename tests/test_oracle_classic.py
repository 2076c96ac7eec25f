"""Oracle pins for Algorithm 1 (classic preconditioned BiCGStab)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import oracle
import testproblems as tp


def _scipy_iterates(A, b, nit, M=None):
    xs = []
    spl.bicgstab(A, b, rtol=1e-30, maxiter=nit, M=M, callback=lambda x: xs.append(x.copy()))
    return xs


@pytest.mark.parametrize("which", ["poisson", "upwind_jacobi"])
def test_classic_matches_scipy_iterates(which):
    """scipy's bicgstab uses the same shadow vector r_0 and right preconditioning."""
    if which == "poisson":
        p = tp.problem_poisson2d(30)
        A = p.A.to_scipy()
        M = None
        prec = "none"
    else:
        p = tp.problem_convdiff2d(24)
        A = p.A.to_scipy()
        dinv = 1.0 / A.diagonal()
        M = spl.LinearOperator(A.shape, matvec=lambda v: dinv * v)
        prec = "jacobi"
    ref = _scipy_iterates(A, p.b, 10, M)
    res = oracle.bicgstab(A, p.b, precond=prec, tol=1e-30, maxit=10, record=10)
    for i in range(10):
        assert np.linalg.norm(res.xs[i] - ref[i]) <= 1e-10 * np.linalg.norm(ref[i])


def test_classic_converges_to_dense_lu():
    p = tp.problem_convdiff2d(15)
    A = p.A.to_scipy()
    res = oracle.bicgstab(A, p.b, precond="jacobi", tol=1e-13, maxit=500)
    xd = np.linalg.solve(A.toarray(), p.b)
    assert res.status == oracle.Status.OK
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(res.x - xd) <= kappa * 1e-13 * np.linalg.norm(xd) * 10


def test_classic_random_unsymmetric_dense_lu():
    rng = np.random.Generator(np.random.PCG64(11))
    A = tp.random_banded_system(300, rng, band=20)
    As = A.to_scipy(np.float64)
    xs = rng.uniform(-1, 1, 300)
    b = As @ xs
    res = oracle.bicgstab(As, b, precond="jacobi", tol=1e-14, maxit=500)
    assert res.status == oracle.Status.OK
    assert np.linalg.norm(res.x - np.linalg.solve(As.toarray(), b)) <= 1e-11 * np.linalg.norm(xs)
