"""Adjoint gradients of a linear solve (test infrastructure only).

Not in the paper: standard linear algebra for the differentiable solve.  For
X = A^{-1} B (one column per right-hand side) and the loss
L = sum_c ||X[:, c] - X_t[:, c]||^2:

    dL/dX   = 2 (X - X_t)
    Lambda  = A^{-T} dL/dX          (adjoint solve with the transposed matrix)
    dL/dB   = Lambda
    dL/dA_e = - sum_c Lambda[row_e, c] * X[col_e, c]   for every stored entry e.
"""
from __future__ import annotations

import numpy as np

from .krylov import pbicgstab


def loss(X, Xt) -> float:
    return float(np.sum((X - Xt) ** 2))


def grad_values(row_ptr, col, Lam, X) -> np.ndarray:
    """dL/dA over the CSR pattern: -sum_c Lam[row_e, c] X[col_e, c]."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    Lam2 = Lam.reshape(n, -1)
    X2 = X.reshape(n, -1)
    return -np.sum(Lam2[rows, :] * X2[col, :], axis=1)


def dense_adjoint(A_csr, B, Xt):
    """Dense LAPACK solves: returns X, dL/dB, dL/d(values) for a small system."""
    Ad = A_csr.to_scipy(np.float64).toarray()
    X = np.linalg.solve(Ad, B)
    G = 2.0 * (X - Xt)
    Lam = np.linalg.solve(Ad.T, G)
    return X, Lam, grad_values(A_csr.row_ptr, A_csr.col, Lam, X)


def sparse_adjoint(A_csr, B, Xt, precond="jacobi", tol=1e-13, maxit=20000, rr_period=100):
    """Forward and adjoint solves with the oracle's p-BiCGStab (one column at a time)."""
    A = A_csr.to_scipy(np.float64)
    AT = A.T.tocsr()
    nrhs = B.shape[1]
    X = np.zeros_like(B)
    for c in range(nrhs):
        X[:, c] = pbicgstab(A, B[:, c], precond=precond, tol=tol, maxit=maxit, rr_period=rr_period).x
    G = 2.0 * (X - Xt)
    Lam = np.zeros_like(B)
    for c in range(nrhs):
        Lam[:, c] = pbicgstab(AT, G[:, c], precond=precond, tol=tol, maxit=maxit, rr_period=rr_period).x
    return X, Lam, grad_values(A_csr.row_ptr, A_csr.col, Lam, X)
