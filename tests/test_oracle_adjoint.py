"""Oracle pins for the adjoint gradients (standard linear algebra, not in the paper)."""
import numpy as np

from oracle import adjoint
import testproblems as tp


def test_dense_adjoint_matches_central_differences():
    m = tp.problem_convdiff2d_multi(n=5, nrhs=3)
    A = m.A
    X, gb, gv = adjoint.dense_adjoint(A, m.B, m.X_target)
    Ad = A.to_scipy().toarray()
    h = 1e-6

    def L_of_b(B):
        return adjoint.loss(np.linalg.solve(Ad, B), m.X_target)

    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(6):
        i, c = rng.integers(0, A.n), rng.integers(0, 3)
        Bp, Bm = m.B.copy(), m.B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (L_of_b(Bp) - L_of_b(Bm)) / (2 * h)
        assert abs(fd - gb[i, c]) <= 1e-6 * max(1.0, abs(gb[i, c]))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    for _ in range(6):
        e = rng.integers(0, A.nnz)
        Ap, Am = Ad.copy(), Ad.copy()
        Ap[rows[e], A.col[e]] += h
        Am[rows[e], A.col[e]] -= h
        fd = (adjoint.loss(np.linalg.solve(Ap, m.B), m.X_target)
              - adjoint.loss(np.linalg.solve(Am, m.B), m.X_target)) / (2 * h)
        assert abs(fd - gv[e]) <= 1e-6 * max(1.0, abs(gv[e]))


def test_sparse_adjoint_matches_dense():
    m = tp.problem_convdiff2d_multi(n=12, nrhs=2)
    Xd, gbd, gvd = adjoint.dense_adjoint(m.A, m.B, m.X_target)
    Xs, gbs, gvs = adjoint.sparse_adjoint(m.A, m.B, m.X_target, tol=1e-13)
    assert np.linalg.norm(Xs - Xd) <= 1e-11 * np.linalg.norm(Xd)
    assert np.linalg.norm(gbs - gbd) <= 1e-9 * np.linalg.norm(gbd)
    assert np.linalg.norm(gvs - gvd) <= 1e-9 * np.linalg.norm(gvd)
