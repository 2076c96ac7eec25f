"""Preconditioners M^{-1} for the oracle (test infrastructure only).

The paper's algorithms take an abstract preconditioner application
``M^{-1} v`` (PREC, Section 1 and Algorithms 1-2).  Its own experiments use
ICC(0), which is out of scope here; the solver's configurations use:

* identity (no preconditioner, as in the paper's timing runs, Section 4.1);
* Jacobi: M^{-1} v = D^{-1} v with D = diag(A), d_inv = 1/a_jj in FP64;
* Neumann polynomial of degree d in D^{-1}A:
      M^{-1} = sum_{j=0..d} (I - D^{-1} A)^j D^{-1},
  applied by the Horner / Jacobi-sweep recursion
      y_0 = D^{-1} v,   y_j = y_{j-1} + D^{-1} (v - A y_{j-1}),  j = 1..d.

In mixed mode (``dtype=float32``) every step is evaluated in FP32 with the
FP32-rounded matrix and d_inv32 = fl32(1/a_jj computed in FP64).
"""
from __future__ import annotations

import numpy as np


class Identity:
    kind = "none"
    degree = 0

    def __init__(self, n: int, dtype=np.float64):
        self.n = n
        self.dtype = dtype
        self.dinv = np.ones(n, dtype=dtype)

    def apply(self, v: np.ndarray) -> np.ndarray:
        return v.copy()

    def max_row_nnz(self) -> int:
        return 1

    def norm2_bound(self) -> float:
        return 1.0


class Jacobi:
    kind = "jacobi"
    degree = 0

    def __init__(self, diag: np.ndarray, dtype=np.float64):
        if np.any(diag == 0):
            raise ValueError("Jacobi needs a non-zero diagonal")
        dinv64 = 1.0 / diag.astype(np.float64)
        self.dinv = dinv64.astype(dtype)
        self.dtype = dtype
        self.n = len(diag)

    def apply(self, v: np.ndarray) -> np.ndarray:
        return self.dinv * v

    def max_row_nnz(self) -> int:
        return 1

    def norm2_bound(self) -> float:
        return float(np.max(np.abs(self.dinv.astype(np.float64))))


class Neumann:
    kind = "neumann"

    def __init__(self, A, diag: np.ndarray, degree: int, dtype=np.float64):
        """A: scipy CSR matrix in the working precision ``dtype``."""
        if np.any(diag == 0):
            raise ValueError("Neumann needs a non-zero diagonal")
        self.A = A
        self.degree = int(degree)
        self.dinv = (1.0 / diag.astype(np.float64)).astype(dtype)
        self.dtype = dtype
        self.n = len(diag)

    def apply(self, v: np.ndarray) -> np.ndarray:
        y = self.dinv * v
        for _ in range(self.degree):
            y = y + self.dinv * (v - self.A @ y)
        return y

    def explicit(self):
        """M^{-1} as an explicit sparse matrix (for norms and nnz counts in the error bounds)."""
        import scipy.sparse as sp
        Dinv = sp.diags(self.dinv.astype(np.float64))
        A = self.A.astype(np.float64)
        N = sp.identity(self.n, format="csr") - Dinv @ A
        M = Dinv.tocsr()
        term = Dinv.tocsr()
        for _ in range(self.degree):
            term = (N @ term).tocsr()
            M = (M + term).tocsr()
        return M

    def max_row_nnz(self) -> int:
        M = self.explicit()
        return int(np.max(np.diff(M.indptr)))

    def norm2_bound(self) -> float:
        M = self.explicit()
        a = abs(M)
        return float(np.sqrt(a.sum(axis=0).max() * a.sum(axis=1).max()))


def make_precond(kind: str, A64, degree: int = 0, dtype=np.float64):
    """Build a preconditioner for the FP64 scipy matrix ``A64`` in precision ``dtype``."""
    diag = A64.diagonal()
    if kind == "none":
        return Identity(A64.shape[0], dtype)
    if kind == "jacobi":
        return Jacobi(diag, dtype)
    if kind == "neumann":
        return Neumann(A64.astype(dtype), diag, degree, dtype)
    raise ValueError("unknown preconditioner %r" % kind)
