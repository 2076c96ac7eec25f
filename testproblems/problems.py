"""Generators for the synthetic linear systems (see the package docstring)."""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclass
class CSR:
    """Compressed sparse row matrix: int32 row_ptr[n+1], int32 col[nnz], values[nnz]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self, dtype=None):
        import scipy.sparse as sp
        v = self.val if dtype is None else self.val.astype(dtype)
        return sp.csr_matrix((v, self.col, self.row_ptr), shape=(self.n, self.n))

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.row_ptr, self.col, self.val.astype(dtype))

    def max_row_nnz(self) -> int:
        return int(np.max(np.diff(self.row_ptr))) if self.n else 0


@dataclass
class Problem:
    """One linear system A x = b with its solver settings."""
    name: str
    A: CSR
    b: np.ndarray
    x0: np.ndarray
    x_star: Optional[np.ndarray]
    precond: str = "none"          # "none" | "jacobi" | "neumann"
    degree: int = 0                # Neumann polynomial degree
    tol: float = 1e-10
    maxit: int = 10000
    fmt: str = "csr"               # storage the solver is asked to use: "csr" | "dia"
    grid: Tuple[int, ...] = ()
    sigma: float = 1.0             # normalisation factor the matrix was divided by


@dataclass
class BatchProblem:
    """Many independent systems, concatenated.  Offsets are int64."""
    name: str
    systems: List[Problem]
    tol: float = 1e-8
    maxit: int = 1000

    def concat(self):
        """Concatenated arrays: row offsets, nnz offsets, row_ptr (local per system), col, val, b, x0."""
        n = np.array([s.A.n for s in self.systems], dtype=np.int64)
        nnz = np.array([s.A.nnz for s in self.systems], dtype=np.int64)
        row_off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
        nnz_off = np.concatenate([[0], np.cumsum(nnz)]).astype(np.int64)
        rp_off = np.concatenate([[0], np.cumsum(n + 1)]).astype(np.int64)
        row_ptr = np.concatenate([s.A.row_ptr for s in self.systems]).astype(np.int32)
        col = np.concatenate([s.A.col for s in self.systems]).astype(np.int32)
        val = np.concatenate([s.A.val for s in self.systems])
        b = np.concatenate([s.b for s in self.systems])
        x0 = np.concatenate([s.x0 for s in self.systems])
        return dict(row_off=row_off, nnz_off=nnz_off, rp_off=rp_off, row_ptr=row_ptr,
                    col=col, val=val, b=b, x0=x0)


@dataclass
class MultiProblem:
    """One matrix with several right-hand sides (column-major N x nrhs) plus targets."""
    name: str
    A: CSR
    B: np.ndarray        # (n, nrhs), float64
    X_target: np.ndarray  # (n, nrhs)
    precond: str = "jacobi"
    tol: float = 1e-10
    maxit: int = 20000
    grid: Tuple[int, ...] = ()
    sigma: float = 1.0


# ---------------------------------------------------------------- stencils
def stencil_2d(nx: int, ny: int, c: Dict[str, float]) -> CSR:
    """5-point stencil on an nx x ny interior grid; keys centre, west, east, south, north.

    Columns of every row are sorted ascending: south (-nx), west (-1), centre,
    east (+1), north (+nx).  Neighbours outside the grid (Dirichlet) are dropped.
    """
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = idx // nx
    entries = [(-nx, j > 0, c["south"]), (-1, i > 0, c["west"]), (0, np.ones(n, bool), c["centre"]),
               (1, i < nx - 1, c["east"]), (nx, j < ny - 1, c["north"])]
    return _assemble(n, entries)


def stencil_3d(nx: int, ny: int, nz: int, c: Dict[str, float]) -> CSR:
    """7-point stencil; keys centre, west, east, south, north, down, up (down = -nx*ny)."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    pl = nx * ny
    entries = [(-pl, k > 0, c["down"]), (-nx, j > 0, c["south"]), (-1, i > 0, c["west"]),
               (0, np.ones(n, bool), c["centre"]), (1, i < nx - 1, c["east"]),
               (nx, j < ny - 1, c["north"]), (pl, k < nz - 1, c["up"])]
    return _assemble(n, entries)


def _assemble(n: int, entries) -> CSR:
    # entries are in ascending offset order, so per-row columns come out sorted.
    counts = np.zeros(n, dtype=np.int64)
    for _, mask, _ in entries:
        counts += mask
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    fill = row_ptr[:-1].copy()
    idx = np.arange(n, dtype=np.int64)
    for off, mask, coef in entries:
        rows = idx[mask]
        pos = fill[rows]
        col[pos] = (rows + off).astype(np.int32)
        val[pos] = coef
        fill[rows] += 1
    return CSR(n, row_ptr.astype(np.int32), col, val)


def csr_diag(A: CSR) -> np.ndarray:
    """Main diagonal of A (zero where absent)."""
    d = np.zeros(A.n, dtype=A.val.dtype)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    m = A.col == rows
    d[rows[m]] = A.val[m]
    return d


def csr_to_dia(A: CSR) -> Tuple[np.ndarray, np.ndarray]:
    """Diagonal storage: offsets[ndiag] (ascending) and data[ndiag, n] with data[d, i] = A[i, i+off[d]]."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.row_ptr))
    offs_all = A.col.astype(np.int64) - rows
    offsets = np.unique(offs_all)
    data = np.zeros((len(offsets), A.n), dtype=A.val.dtype)
    d_idx = np.searchsorted(offsets, offs_all)
    data[d_idx, rows] = A.val
    return offsets.astype(np.int32), data


def normalise(A: CSR) -> Tuple[CSR, float]:
    """Divide A by sigma = sqrt(||A||_1 ||A||_inf) >= ||A||_2 (see the package docstring)."""
    absval = np.abs(A.val)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    row_sums = np.bincount(rows, weights=absval, minlength=A.n)
    col_sums = np.bincount(A.col, weights=absval, minlength=A.n)
    sigma = float(np.sqrt(row_sums.max() * col_sums.max()))
    return CSR(A.n, A.row_ptr, A.col, A.val / sigma), sigma


def _spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    return A.to_scipy() @ x


# ---------------------------------------------------------------- problems
def poisson_2d(n: int) -> CSR:
    return stencil_2d(n, n, dict(centre=4.0, west=-1.0, east=-1.0, south=-1.0, north=-1.0))


def tp2(n: int = 1000, eps: float = 1e-3) -> CSR:
    """Paper TP2: Poisson with the upper-triangle (east, north) couplings -1+eps."""
    return stencil_2d(n, n, dict(centre=4.0, west=-1.0, east=-1.0 + eps, south=-1.0, north=-1.0 + eps))


def upwind_2d(n: int, peclet: float = 0.5) -> CSR:
    hb = peclet  # h * beta_x = h * beta_y
    return stencil_2d(n, n, dict(centre=4.0 + 2 * hb, west=-1.0 - hb, east=-1.0,
                                 south=-1.0 - hb, north=-1.0))


def upwind_3d(n: int, scale: float = 0.8) -> CSR:
    hb = np.array([1.0, 0.5, 0.25]) * scale
    return stencil_3d(n, n, n, dict(centre=6.0 + hb.sum(), west=-1.0 - hb[0], east=-1.0,
                                    south=-1.0 - hb[1], north=-1.0, down=-1.0 - hb[2], up=-1.0))


def problem_poisson2d(n: int = 100) -> Problem:
    """2D Poisson 5-point, x* = 1/sqrt(N), b = A x*, x0 = 0, no preconditioner, tol 1e-12."""
    A, sigma = normalise(poisson_2d(n))
    N = A.n
    xs = np.full(N, 1.0 / np.sqrt(N))
    return Problem("poisson2d_%dx%d" % (n, n), A, _spmv(A, xs), np.zeros(N), xs,
                   precond="none", tol=1e-12, maxit=1000, fmt="csr", grid=(n, n), sigma=sigma)


def problem_convdiff2d(n: int = 1024, seed: int = 2) -> Problem:
    """2D upwind convection-diffusion (cell Peclet 0.5), 5 diagonals, x* ~ U[0,1], Jacobi, tol 1e-10."""
    A, sigma = normalise(upwind_2d(n, 0.5))
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(0.0, 1.0, A.n)
    return Problem("convdiff2d_%dx%d" % (n, n), A, _spmv(A, xs), np.zeros(A.n), xs,
                   precond="jacobi", tol=1e-10, maxit=20000, fmt="dia", grid=(n, n), sigma=sigma)


def problem_convdiff3d(n: int = 256, seed: int = 3, degree: int = 2) -> Problem:
    """3D upwind convection-diffusion 7-point as CSR, x* ~ U[-1,1], Jacobi + Neumann(degree), tol 1e-10."""
    A, sigma = normalise(upwind_3d(n, 0.8))
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(-1.0, 1.0, A.n)
    return Problem("convdiff3d_%d^3" % n, A, _spmv(A, xs), np.zeros(A.n), xs,
                   precond="neumann", degree=degree, tol=1e-10, maxit=20000, fmt="csr",
                   grid=(n, n, n), sigma=sigma)


def random_banded_system(N: int, rng: np.random.Generator, band: int = 256,
                         nnz_lo: int = 7, nnz_hi: int = 15) -> CSR:
    """Random unsymmetric banded system with FP32 values.

    Each row has nnz ~ U{nnz_lo..nnz_hi} entries including the diagonal; the
    off-diagonal columns are distinct, uniform in [i-band, i+band] within
    [0, N) excluding i, and sorted.  Off-diagonals ~ N(0,1) rounded to FP32;
    the diagonal is +-1.2 * sum|off-diagonals| (random sign), rounded to FP32.
    """
    k_off = rng.integers(nnz_lo - 1, nnz_hi, size=N)          # off-diagonals per row, 6..14
    ncand = 24
    rows = np.arange(N, dtype=np.int64)[:, None]
    lo = np.maximum(rows - band, 0)
    hi = np.minimum(rows + band, N - 1)
    # candidates uniform in [lo, hi] \ {i}: draw from a window one smaller and skip i
    width = (hi - lo)  # number of admissible columns (window size minus the diagonal)
    u = rng.random((N, ncand))
    cand = lo + np.floor(u * width).astype(np.int64)
    cand = cand + (cand >= rows)
    cand.sort(axis=1)
    dup = np.zeros_like(cand, dtype=bool)
    dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
    # keep first k_off unique candidates (in a random order, then re-sort)
    keys = rng.random((N, ncand)) + dup * 2.0       # duplicates sort last
    order = np.argsort(keys, axis=1)
    picked = np.take_along_axis(cand, order, axis=1)
    picked_dup = np.take_along_axis(dup, order, axis=1)
    take = (np.arange(ncand)[None, :] < k_off[:, None]) & ~picked_dup
    n_off = take.sum(axis=1)
    offv = rng.standard_normal((N, ncand)).astype(np.float32)
    # assemble rows: off-diagonals + diagonal, sorted by column
    counts = n_off + 1
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cols_all = np.where(take, picked, -1)
    vals_all = np.where(take, offv, np.float32(0))
    diag_mag = 1.2 * np.abs(vals_all.astype(np.float64)).sum(axis=1)
    sign = np.where(rng.random(N) < 0.5, -1.0, 1.0)
    diag = (sign * diag_mag).astype(np.float32)
    cols_all = np.concatenate([cols_all, rows], axis=1)
    vals_all = np.concatenate([vals_all, diag[:, None]], axis=1)
    valid = np.concatenate([take, np.ones((N, 1), bool)], axis=1)
    sort_key = np.where(valid, cols_all, np.int64(1) << 40)
    o = np.argsort(sort_key, axis=1, kind="stable")
    cols_sorted = np.take_along_axis(cols_all, o, axis=1)
    vals_sorted = np.take_along_axis(vals_all, o, axis=1)
    valid_sorted = np.take_along_axis(valid, o, axis=1)
    col = cols_sorted[valid_sorted].astype(np.int32)
    val = vals_sorted[valid_sorted].astype(np.float32)
    return CSR(N, row_ptr.astype(np.int32), col, val)


def problem_batched_banded(nsys: int = 512, seed: int = 4, n_lo: int = 2048, n_hi: int = 65536,
            band: int = 256) -> BatchProblem:
    """Batched random banded systems, N_k ~ U{n_lo..n_hi}, FP32 values, x* ~ U[-1,1], b = A x* in FP64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(n_lo, n_hi + 1, size=nsys)
    systems = []
    for k, N in enumerate(sizes):
        A = random_banded_system(int(N), rng, band=band)
        xs = rng.uniform(-1.0, 1.0, int(N))
        b = A.to_scipy(np.float64) @ xs
        systems.append(Problem("sys%d" % k, A, b, np.zeros(int(N)), xs, precond="jacobi",
                               tol=1e-8, maxit=1000, fmt="csr"))
    return BatchProblem("batched_%d" % nsys, systems, tol=1e-8, maxit=1000)


def problem_convdiff2d_multi(n: int = 512, nrhs: int = 16, seed: int = 5) -> MultiProblem:
    """2D upwind convection-diffusion CSR FP64 with nrhs right-hand sides ~ N(0,1), targets ~ U[0,1]."""
    A, sigma = normalise(upwind_2d(n, 0.5))
    rng = np.random.Generator(np.random.PCG64(seed))
    B = rng.standard_normal((A.n, nrhs))
    Xt = rng.uniform(0.0, 1.0, (A.n, nrhs))
    return MultiProblem("convdiff2d_%dx%d_x%d" % (n, n, nrhs), A, B, Xt, precond="jacobi",
                        tol=1e-10, grid=(n, n), sigma=sigma)
