"""Planted mistakes in the preconditioner and adjoint oracles (``oracle/precond.py``,
``oracle/adjoint.py``): each mutant is the module's source with one slip and must fail a
pin.  CPU only.

Preconditioner pins (properties, not the formulas retyped):
* Jacobi inverts a diagonal matrix exactly;
* where I - D^{-1}A is nilpotent (A = D + strictly lower bidiagonal part, varying D), the
  Neumann polynomial of degree n-1 is A^{-1}: A (M^{-1} v) = v;
* for lower degrees, M^{-1} v and the explicit matrix equal the closed-form power sum
  sum_j (I - D^{-1}A)^j D^{-1} built with dense matrix powers (a different evaluation from
  the oracle's sweep recursion), and the norm and row-count bounds hold for that matrix.
Adjoint pins: the existing central-difference and dense-versus-sparse pins of
``test_oracle_adjoint.py``, run against the mutant."""
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp

import test_oracle_adjoint as TA
from oracle import adjoint, precond

PRECOND_SOURCE = open(precond.__file__).read()
ADJOINT_SOURCE = open(adjoint.__file__).read()

PRECOND_MUTANTS = [
    ("Jacobi: reciprocal dropped", "dinv64 = 1.0 / diag.astype(np.float64)", "dinv64 = diag.astype(np.float64)"),
    ("Neumann sweep: sign of A y", "y = y + self.dinv * (v - self.A @ y)", "y = y + self.dinv * (v + self.A @ y)"),
    ("Neumann sweep: v -> y", "y = y + self.dinv * (v - self.A @ y)", "y = y + self.dinv * (y - self.A @ y)"),
    ("Neumann: one sweep short", "for _ in range(self.degree):\n            y = y",
     "for _ in range(self.degree - 1):\n            y = y"),
    ("explicit: sign of D^-1 A", 'N = sp.identity(self.n, format="csr") - Dinv @ A',
     'N = sp.identity(self.n, format="csr") + Dinv @ A'),
    ("explicit: N^j D^-1 -> D^-1 N^j", "term = (N @ term).tocsr()", "term = (term @ N).tocsr()"),
    ("explicit: starts at I", "M = Dinv.tocsr()\n", 'M = sp.identity(self.n, format="csr")\n'),
    ("make_precond: Neumann -> Jacobi", "return Neumann(A64.astype(dtype), diag, degree, dtype)", "return Jacobi(diag, dtype)"),
    ("Neumann norm bound: min", "return float(np.sqrt(a.sum(axis=0).max() * a.sum(axis=1).max()))",
     "return float(np.sqrt(a.sum(axis=0).min() * a.sum(axis=1).min()))"),
]

ADJOINT_MUTANTS = [
    ("value gradient: sign", "return -np.sum(Lam2[rows, :] * X2[col, :], axis=1)",
     "return np.sum(Lam2[rows, :] * X2[col, :], axis=1)"),
    ("value gradient: row and column swapped", "return -np.sum(Lam2[rows, :] * X2[col, :], axis=1)",
     "return -np.sum(Lam2[col, :] * X2[rows, :], axis=1)"),
    ("dense adjoint: A instead of A^T", "Lam = np.linalg.solve(Ad.T, G)", "Lam = np.linalg.solve(Ad, G)"),
    ("dense adjoint: factor 2 dropped", "G = 2.0 * (X - Xt)\n    Lam = np.linalg.solve", "G = (X - Xt)\n    Lam = np.linalg.solve"),
    ("sparse adjoint: A instead of A^T", "AT = A.T.tocsr()", "AT = A.tocsr()"),
    ("sparse adjoint: factor 2 dropped", "G = 2.0 * (X - Xt)\n    Lam = np.zeros_like", "G = (X - Xt)\n    Lam = np.zeros_like"),
    ("loss: absolute instead of squared", "return float(np.sum((X - Xt) ** 2))", "return float(np.sum(np.abs(X - Xt)))"),
]


def _load(src, like):
    mod = types.ModuleType("oracle._mutant_" + like.__name__.split(".")[-1])
    mod.__package__ = "oracle"
    mod.__file__ = like.__file__
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src, "<oracle mutant>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _mutated(source, old, new, like):
    assert source.count(old) == 1, "mutation site not unique or missing: %r" % old
    return _load(source.replace(old, new), like)


# ---------------------------------------------------------------- preconditioner pins
def _precond_pins(mod):
    rng = np.random.Generator(np.random.PCG64(8))
    # Jacobi on a diagonal matrix is its inverse
    d = rng.uniform(0.5, 3.0, 7) * rng.choice([-1.0, 1.0], 7)
    Ad = sp.diags(d).tocsr()
    v = rng.standard_normal(7)
    if not np.allclose(Ad @ mod.make_precond("jacobi", Ad).apply(v), v, rtol=1e-15, atol=1e-15):
        return False
    # nilpotent I - D^{-1}A: degree n - 1 Neumann is the inverse
    n = 5
    L = sp.diags([rng.uniform(0.5, 2.0, n), rng.uniform(-1.0, 1.0, n - 1)], [0, -1]).tocsr()
    v = rng.standard_normal(n)
    if not np.allclose(L @ mod.make_precond("neumann", L, n - 1).apply(v), v, rtol=1e-12, atol=1e-12):
        return False
    # lower degrees: the closed-form power sum on an unsymmetric matrix with a varying diagonal
    A = sp.random(12, 12, density=0.3, random_state=np.random.RandomState(3), format="csr")
    A = (A + sp.diags(rng.uniform(2.0, 4.0, 12))).tocsr()
    Adense = A.toarray()
    Dinv = np.diag(1.0 / np.diag(Adense))
    N = np.eye(12) - Dinv @ Adense
    v = rng.standard_normal(12)
    for deg in (1, 2, 3):
        want = sum(np.linalg.matrix_power(N, j) for j in range(deg + 1)) @ Dinv
        M = mod.make_precond("neumann", A, deg)
        if not np.allclose(M.apply(v), want @ v, rtol=1e-12, atol=1e-14):
            return False
        if not np.allclose(M.explicit().toarray(), want, rtol=1e-12, atol=1e-14):
            return False
        if M.norm2_bound() < np.linalg.norm(want, 2) * (1 - 1e-12):
            return False
        if M.max_row_nnz() != int(np.max(np.sum(np.abs(want) > 0, axis=1))):
            return False
    return True


def test_unmutated_precond_passes():
    assert _precond_pins(_load(PRECOND_SOURCE, precond))


@pytest.mark.parametrize("name,old,new", PRECOND_MUTANTS, ids=[m[0] for m in PRECOND_MUTANTS])
def test_precond_mutant_fails_a_pin(name, old, new):
    with np.errstate(all="ignore"):
        assert not _precond_pins(_mutated(PRECOND_SOURCE, old, new, precond)), name


# ---------------------------------------------------------------- adjoint pins
def _adjoint_failures(monkeypatch, mod):
    monkeypatch.setattr(TA, "adjoint", mod)
    failed = []
    for fn in (TA.test_dense_adjoint_matches_central_differences, TA.test_sparse_adjoint_matches_dense):
        try:
            fn()
        except (AssertionError, np.linalg.LinAlgError, ValueError):
            failed.append(fn.__name__)
    return failed


def test_unmutated_adjoint_passes(monkeypatch):
    assert _adjoint_failures(monkeypatch, _load(ADJOINT_SOURCE, adjoint)) == []


@pytest.mark.parametrize("name,old,new", ADJOINT_MUTANTS, ids=[m[0] for m in ADJOINT_MUTANTS])
def test_adjoint_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert _adjoint_failures(monkeypatch, _mutated(ADJOINT_SOURCE, old, new, adjoint)), name
