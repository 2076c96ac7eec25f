"""Input generators: stencils, normalisation, random banded systems, determinism."""
import numpy as np
import pytest

import testproblems as tp


def dense(A):
    return A.to_scipy().toarray()


def test_poisson_stencil_and_symmetry():
    A = tp.poisson_2d(5)
    D = dense(A)
    assert np.allclose(D, D.T)
    assert np.all(np.diag(D) == 4.0)
    # interior row has four -1 neighbours, corner row two
    assert np.sum(D[12] == -1.0) == 4 and np.sum(D[0] == -1.0) == 2


def test_upwind_2d_coefficients():
    A = tp.upwind_2d(4, 0.5)
    D = dense(A)
    r = 1 * 4 + 1  # interior node (i=1, j=1)
    assert D[r, r] == 5.0
    assert D[r, r - 1] == -1.5 and D[r, r - 4] == -1.5   # west, south (upwind)
    assert D[r, r + 1] == -1.0 and D[r, r + 4] == -1.0   # east, north


def test_upwind_3d_coefficients():
    A = tp.upwind_3d(3, 0.8)
    D = dense(A)
    r = 13  # centre node of 3x3x3
    assert np.isclose(D[r, r], 7.4)
    assert np.isclose(D[r, r - 1], -1.8) and np.isclose(D[r, r - 3], -1.4) and np.isclose(D[r, r - 9], -1.2)
    assert D[r, r + 1] == -1.0 and D[r, r + 3] == -1.0 and D[r, r + 9] == -1.0


def test_tp2_upper_triangle_perturbed():
    D = dense(tp.tp2(4, 1e-3))
    assert np.isclose(D[5, 6], -1 + 1e-3) and np.isclose(D[5, 9], -1 + 1e-3)
    assert D[5, 4] == -1.0 and D[5, 1] == -1.0


def test_tp2_unsymmetric_positive_definite():
    """Section 4 describes TP2 as positive definite but unsymmetric: x^T A x > 0 for
    every x (its symmetric part is positive definite) while A != A^T."""
    D = dense(tp.tp2(12, 1e-3))
    assert not np.allclose(D, D.T)
    assert np.linalg.eigvalsh((D + D.T) / 2).min() > 0.0


@pytest.mark.parametrize("maker", [lambda: tp.poisson_2d(12), lambda: tp.upwind_2d(12), lambda: tp.upwind_3d(6)])
def test_normalised_two_norm(maker):
    A, sigma = tp.normalise(maker())
    s = np.linalg.svd(dense(A), compute_uv=False)[0]
    assert s <= 1.0 + 1e-12
    assert s >= 0.9


def test_csr_sorted_and_dia_roundtrip():
    A = tp.upwind_2d(7)
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    off, data = tp.csr_to_dia(A)
    assert list(off) == [-7, -1, 0, 1, 7]
    D = dense(A)
    for d, o in enumerate(off):
        for i in range(A.n):
            j = i + o
            expect = D[i, j] if 0 <= j < A.n else 0.0
            assert data[d, i] == expect


def test_random_banded_properties():
    rng = np.random.Generator(np.random.PCG64(7))
    A = tp.random_banded_system(3000, rng, band=256)
    nnz = np.diff(A.row_ptr)
    assert nnz.min() >= 7 and nnz.max() <= 15
    rows = np.repeat(np.arange(A.n), nnz)
    assert np.all(np.abs(A.col - rows) <= 256)
    assert A.val.dtype == np.float32
    d = tp.csr_diag(A).astype(np.float64)
    off = np.bincount(rows, weights=np.abs(A.val.astype(np.float64)), minlength=A.n) - np.abs(d)
    ratio = np.abs(d) / off
    assert np.all(np.abs(ratio - 1.2) < 1e-5)
    for i in range(0, A.n, 97):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_generators_deterministic():
    a = tp.problem_convdiff2d(16)
    b = tp.problem_convdiff2d(16)
    assert np.array_equal(a.b, b.b)
    c4a = tp.problem_batched_banded(nsys=3, n_lo=100, n_hi=300)
    c4b = tp.problem_batched_banded(nsys=3, n_lo=100, n_hi=300)
    for s1, s2 in zip(c4a.systems, c4b.systems):
        assert np.array_equal(s1.A.val, s2.A.val) and np.array_equal(s1.b, s2.b)


def test_workload_shapes():
    p = tp.problem_poisson2d()
    assert p.A.n == 10000 and np.allclose(p.x_star, 1 / 100.0)
    assert np.allclose(p.A.to_scipy() @ p.x_star, p.b)
    m = tp.problem_convdiff2d_multi(8, 4)
    assert m.B.shape == (64, 4) and m.X_target.shape == (64, 4)
