"""Error propagation in p-BiCGStab, Section 2.4 of the paper (test infrastructure only).

* ``gap_operator``          -- the 4 x 4 matrix of Eq. (system) that maps the gaps
  (Delta^r_i, Delta^s_{i-1}, Delta^w_i, Delta^z_{i-1}) to
  (Delta^r_{i+1}, Delta^s_i, Delta^w_{i+1}, Delta^z_i).
* ``local_error_terms``     -- the local additions epsilon^r, ^s, ^w, ^z of Eq. (local).
* ``propagation_matrices``  -- the error propagation matrices A, B, E, P, C, D, O, U of
  Eq. (all_matrices), as dense upper-triangular arrays.
* ``error_matrix_products`` -- the nine products of Eq. (all_error_matrices).
* ``column_max_norms``      -- max_k |M_kj| for every column j (the curves the paper
  plots for these products).

Scalar sequences: ``alpha[i]`` = alpha_i, ``omega[i]`` = omega_i and ``beta_next[i]`` =
beta_{i+1}, i = 0 .. m-2, exactly as one iteration i of Algorithm 2 produces them
(beta_{i+1} is computed at the end of iteration i).  Matrices for m columns (the
paper's subscript i+1 = m) need m-1 iterations of scalars.

Index reading (the printed Eq. (thetas) and Eq. (auxrec) disagree by one): in
Eq. (auxrec) the error delta^x_i belongs to x_{i+1} (likewise r, k, w), so column k of
Theta^x, Theta^r, Theta^k, Theta^w holds the error made in iteration k-1; the columns of
Theta^s, Theta^z, Theta^l hold the error of s_k, z_k, l_k made in iteration k, and
Theta^u, Theta^p, Theta^y hold iteration k-1's delta^u, delta^q, delta^y, as printed.
The local term of the S expression is A Theta^g + Theta^s (the printed Theta^q is the
same typo as in Eq. (DDs), whose local term is A delta^g - delta^s by Eq. (Ds)).
These readings are pinned by reproducing measured gaps (tests/test_oracle_propagation.py).
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

PRODUCT_NAMES = ("U", "OU", "BA", "UEA", "BAEA", "BPA", "UC", "BAC", "BD")


def gap_operator(alpha_i: float, beta_i: float, omega_i: float, omega_im1: float) -> np.ndarray:
    """Eq. (system): the iteration-i propagation operator of the four gaps."""
    a, b, o, op = alpha_i, beta_i, omega_i, omega_im1
    return np.array([
        [1.0, -a * b, -(a + o), a * b * (o + op)],
        [0.0, b, 1.0, -b * op],
        [0.0, 0.0, 1.0, -a * b],
        [0.0, 0.0, 0.0, b],
    ])


def local_error_terms(A_, d: Dict[str, np.ndarray], alpha_i: float, omega_i: float) -> Dict[str, np.ndarray]:
    """Eq. (local): epsilon^r_i, epsilon^s_i, epsilon^w_i, epsilon^z_i from the local
    rounding errors ``d`` (keys x r q u y g s l z k w, Eq. (auxrec)) of iteration i;
    ``A_`` applies the matrix."""
    a, o = alpha_i, omega_i
    Ag_s = A_(d["g"]) - d["s"]
    Al_z = A_(d["l"]) - d["z"]
    return {
        "r": -A_(d["x"]) - o * A_(d["u"]) + o * d["y"] - d["r"] - d["q"] - a * Ag_s + o * a * Al_z,
        "s": Ag_s,
        "w": -a * Al_z + A_(d["k"]) - d["y"] - d["w"] + A_(d["u"]),
        "z": Al_z,
    }


def _check(alpha, beta_next, omega):
    alpha = np.asarray(alpha, dtype=np.float64)
    beta_next = np.asarray(beta_next, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    if not (alpha.shape == beta_next.shape == omega.shape and alpha.ndim == 1):
        raise ValueError("alpha, beta_next and omega must be 1-D of equal length")
    return alpha, beta_next, omega


def propagation_matrices(alpha: Sequence[float], beta_next: Sequence[float],
                         omega: Sequence[float]) -> Dict[str, np.ndarray]:
    """Eq. (all_matrices) for m = len(alpha) + 1 columns, written out entry by entry."""
    alpha, beta_next, omega = _check(alpha, beta_next, omega)
    m = alpha.size + 1
    beta = np.concatenate([[np.nan], beta_next])     # beta[j] = beta_j, j >= 1

    def bprod(k, j):   # beta_{k+1} ... beta_j (empty product = 1)
        return float(np.prod(beta[k + 1:j + 1]))

    Am, Bm, Em, Pm, Cm, Dm, Om, Um = (np.zeros((m, m)) for _ in range(8))
    for j in range(m):
        for k in range(j + 1):
            Bm[k, j] = bprod(k, j)
            Um[k, j] = 1.0
            if k >= 1:
                Em[k, j] = bprod(k, j)
            if k < j:
                Am[k, j] = -alpha[k]
                Pm[k, j] = -omega[k] * bprod(k, j)
                Cm[k, j] = -omega[k]
                Dm[k, j] = omega[k] * alpha[k]
        if j >= 1:
            Om[j, j] = -omega[j - 1]
    return dict(A=Am, B=Bm, E=Em, P=Pm, C=Cm, D=Dm, O=Om, U=Um)


def error_matrix_products(mats: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Eq. (all_error_matrices): U, OU, BA, UEA, BAEA, BPA, UC, BAC, BD."""
    A, B, E, P, C, D, O, U = (mats[k] for k in "ABEPCDOU")
    return {
        "U": U,
        "OU": O @ U,
        "BA": B @ A,
        "UEA": U @ E @ A,
        "BAEA": B @ A @ E @ A,
        "BPA": B @ P @ A,
        "UC": U @ C,
        "BAC": B @ A @ C,
        "BD": B @ D,
    }


def column_max_norms(M: np.ndarray) -> np.ndarray:
    """max_k |M_kj| for each column j."""
    return np.max(np.abs(M), axis=0)


def propagation_column_norms(alpha, beta_next, omega) -> np.ndarray:
    """(9, m) array: column max-norms of the nine products, in PRODUCT_NAMES order."""
    prods = error_matrix_products(propagation_matrices(alpha, beta_next, omega))
    return np.stack([column_max_norms(prods[k]) for k in PRODUCT_NAMES])
