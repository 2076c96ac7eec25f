"""Rounding-error diagnostics of Sections 2-3 of the paper (test infrastructure only).

* ``bound_constants``  -- mu (max nnz per row of A), mu~ (of M^{-1}), sqrt(N),
  upper bounds of ||A||_2 and ||M^{-1}||_2 (sqrt(||.||_1 ||.||_inf)).
* ``delta_bounds``     -- the local rounding-error bounds Eq. (errbounds1)-(errbounds4)
  for iteration i of Algorithm 2, from vector norms and scalars.
* ``PipelinedProbe``   -- an observer for ``krylov.pbicgstab`` that measures, in
  extended precision, the local rounding errors delta of Eq. (auxrec), the gaps
  Delta^r, Delta^s, Delta^w, Delta^z of Eqs. (res_gap)/(DsDwDz), and how well the
  gap recurrences Eqs. (Dr), (Ds), (Dw), (Dz) hold.
* ``ClassicProbe``     -- the same for Algorithm 1 and Eq. (classic_nomatrix).

Measured local errors are "stored result minus the exact value of the
recurrence's formula applied to the stored inputs", where the explicitly
computed products m = M^{-1} w, n = M^{-1} z, t = A m, v = A n (Eq. auxvars2)
enter the formula as the exact operators applied to the stored w and z; this is
the convention under which the paper's bounds include the SpMV and PREC
round-off terms and under which the gap recurrences hold exactly.  "Exact" is
evaluated in numpy's extended ``longdouble`` (64-bit mantissa on x86); the
probes refuse to run where longdouble is no wider than double.

Parity status: the local-error definitions, the gaps and the gap recurrences are
pinned by equalities (the recurrences hold to the extended precision on real runs).
``delta_bounds`` and ``bound_constants`` are upper bounds and are pinned by
inequalities only (measured errors below them): "parity partially pinned" -- a term
that does not dominate its bound could be dropped without a pin failing.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

LD = np.longdouble


def extended_available() -> bool:
    return np.finfo(LD).eps < 1e-17


def _norm2_bound(A) -> float:
    a = abs(A)
    return float(np.sqrt(a.sum(axis=0).max() * a.sum(axis=1).max()))


def bound_constants(A64, M) -> Dict[str, float]:
    """Constants of the bounds: mu, mu~, sqrt(N), ||A|| and ||M^{-1}|| (upper bounds)."""
    n = A64.shape[0]
    return dict(mu=float(np.max(np.diff(A64.indptr))), mut=float(M.max_row_nnz()),
                sqrtN=math.sqrt(n), nA=_norm2_bound(A64), nM=float(M.norm2_bound()))


def delta_bounds(cur: Dict[str, float], prev: Dict[str, float], alpha, beta, omega, omega_prev,
                 c: Dict[str, float], eps: float) -> Dict[str, float]:
    """Eq. (errbounds1)-(errbounds4): bounds on ||delta^*_i|| for iteration i.

    ``cur`` holds norms of the iteration-i vectors x_i, r_i, k_i, w_i, g_i, s_i,
    l_i, z_i, q_i, u_i, y_i, m_i, t_i, n_i, v_i; ``prev`` those of iteration i-1
    (g, s, l, z, n, v)."""
    msn = c["mu"] * c["sqrtN"]
    tmsn = c["mut"] * c["sqrtN"]
    nA, nM = c["nA"], c["nM"]
    a, b, o, op = abs(alpha), abs(beta), abs(omega), abs(omega_prev)
    bo = b * op
    oa = o * a
    d = {}
    d["g"] = (cur["k"] + 3 * b * prev["g"] + 4 * bo * prev["l"]) * eps
    d["x"] = (2 * cur["x"] + 3 * a * cur["g"] + 2 * o * cur["u"]) * eps
    d["s"] = (cur["w"] + 3 * b * prev["s"] + 4 * bo * prev["z"]) * eps
    d["r"] = (cur["q"] + 2 * o * cur["y"]) * eps
    d["l"] = (cur["m"] + tmsn * nM * cur["w"] + 3 * b * prev["l"] + 4 * bo * prev["n"]
              + tmsn * nM * bo * prev["z"]) * eps
    d["z"] = (cur["t"] + msn * nA * cur["m"] + tmsn * nA * nM * cur["w"] + 3 * b * prev["z"]
              + 4 * bo * prev["v"] + msn * nA * bo * prev["n"] + tmsn * nA * nM * bo * prev["z"]) * eps
    d["k"] = (cur["u"] + 3 * o * cur["m"] + tmsn * nM * o * cur["w"] + 4 * oa * cur["n"]
              + tmsn * nM * oa * cur["z"]) * eps
    d["w"] = (cur["y"] + 3 * o * cur["t"] + msn * nA * o * cur["m"] + tmsn * nA * nM * o * cur["w"]
              + 4 * oa * cur["v"] + msn * nA * oa * cur["n"] + tmsn * nA * nM * oa * cur["z"]) * eps
    d["q"] = (cur["r"] + 2 * a * cur["s"]) * eps
    d["u"] = (cur["k"] + 2 * a * cur["l"]) * eps
    d["y"] = (cur["w"] + 2 * a * cur["z"]) * eps
    return d


class _ExactOps:
    """A and M^{-1} applied in extended precision to stored (FP64) vectors."""

    def __init__(self, A64, precond_kind: str, dinv: np.ndarray, degree: int):
        if not extended_available():
            raise RuntimeError("numpy longdouble is not wider than double on this platform")
        self.A = A64.astype(LD)
        self.kind = precond_kind
        self.dinv = np.asarray(dinv, dtype=np.float64).astype(LD)
        self.degree = degree

    def A_(self, v):
        return self.A @ v.astype(LD)

    def M_(self, v):
        v = v.astype(LD)
        if self.kind == "none":
            return v
        y = self.dinv * v
        if self.kind == "neumann":
            for _ in range(self.degree):
                y = y + self.dinv * (v - self.A @ y)
        return y


def _nrm(v) -> float:
    return float(np.sqrt(np.sum(v.astype(LD) ** 2)))


class PipelinedProbe:
    """Observer for ``krylov.pbicgstab`` (FP64 mode) measuring deltas, gaps and gap identities.

    After the solve, ``records[i]`` holds for iteration i:
      ``delta``  -- dict of measured ||delta^*_i|| (Eq. auxrec),
      ``bound``  -- dict of the bounds Eq. (errbounds1)-(errbounds4),
      ``gap``    -- ||Delta^r_i||, ||Delta^s_i||, ||Delta^w_i||, ||Delta^z_i||,
      ``gap_r_next`` -- ||Delta^r_{i+1}||,
      ``ident``  -- relative residuals of Eqs. (Dr), (Ds), (Dw), (Dz),
      ``replaced``;
    with ``keep_vectors`` also the delta and gap vectors (``delta_vec``, ``gap_vec``,
    ``gap_next_vec``) and the iteration's scalars alpha_i, beta_i, omega_i, omega_{i-1}.
    """

    def __init__(self, A64, b, precond_kind: str, dinv, degree: int, M, keep_vectors: bool = False):
        self.keep_vectors = keep_vectors
        self.ops = _ExactOps(A64, precond_kind, dinv, degree)
        self.b = np.asarray(b, dtype=np.float64).astype(LD)
        self.c = bound_constants(A64, M)
        self.records: List[dict] = []
        self.Ds_prev = None
        self.Dz_prev = None
        self.Dw_cur = None
        self.prev_norms = None
        self.after_replace = []

    def __call__(self, stage, i, d):
        A_, M_ = self.ops.A_, self.ops.M_
        if stage == "init":
            self.Dw_cur = A_(d["k"]) - d["w"].astype(LD)          # Delta^w_0
            return
        if stage == "replace":
            x = d["x"]
            Dr = (self.b - A_(x)) - d["r"].astype(LD)
            self.after_replace.append(dict(i=i, gap_r=_nrm(Dr), x=_nrm(x)))
            # gaps restart: w_{i+1}, s_i, z_i
            self.Dw_cur = A_(d["k"]) - d["w"].astype(LD)
            self.Ds_prev = A_(d["g"]) - d["s"].astype(LD)
            self.Dz_prev = A_(d["l"]) - d["z"].astype(LD)
            if self.records:
                self.records[-1]["replaced"] = True
            if self.prev_norms is not None:
                self.prev_norms = dict(self.prev_norms, s=_nrm(d["s"]), l=_nrm(d["l"]), z=_nrm(d["z"]))
            return
        L = lambda key: d[key].astype(LD)
        al, be, om, op = LD(d["alpha"]), LD(d["beta"]), LD(d["omega"]), LD(d["omega_prev"])
        mex, nex = M_(d["w"]), M_(d["z"])            # exact M^{-1} w_i, M^{-1} z_i
        tex, vex = A_(mex), A_(nex)                  # exact A M^{-1} w_i, A M^{-1} z_i
        nprev_ex = M_(d["z_prev"])
        vprev_ex = A_(nprev_ex)
        delta = {}
        delta["g"] = L("g") - (L("k") + be * (L("g_prev") - op * L("l_prev")))
        delta["s"] = L("s") - (L("w") + be * (L("s_prev") - op * L("z_prev")))
        delta["l"] = L("l") - (mex + be * (L("l_prev") - op * nprev_ex))
        delta["z"] = L("z") - (tex + be * (L("z_prev") - op * vprev_ex))
        delta["q"] = L("q") - (L("r") - al * L("s"))
        delta["u"] = L("u") - (L("k") - al * L("l"))
        delta["y"] = L("y") - (L("w") - al * L("z"))
        delta["x"] = L("x_new") - (L("x") + al * L("g") + om * L("u"))
        delta["r"] = L("r_new") - (L("q") - om * L("y"))
        delta["k"] = L("k_new") - (L("u") - om * (mex - al * nex))
        delta["w"] = L("w_new") - (L("y") - om * (tex - al * vex))
        # gaps at iteration i
        Dr = (self.b - A_(d["x"])) - L("r")
        Ds = A_(d["g"]) - L("s")
        Dz = A_(d["l"]) - L("z")
        Dw = self.Dw_cur
        Dr_next = (self.b - A_(d["x_new"])) - L("r_new")
        Dw_next = A_(d["k_new"]) - L("w_new")
        ident = {}
        pred_r = Dr - al * Ds - om * Dw + om * al * Dz - A_(delta["x"]) - delta["r"] - om * A_(delta["u"]) \
            - delta["q"] + om * delta["y"]                                                # Eq. (Dr)
        ident["r"] = _nrm(Dr_next - pred_r) / max(_nrm(Dr_next), 1e-300)
        pred_w = Dw - al * Dz + A_(delta["k"]) - delta["w"] + A_(delta["u"]) - delta["y"]   # Eq. (Dw)
        ident["w"] = _nrm(Dw_next - pred_w) / max(_nrm(Dw_next), 1e-300)
        if self.Ds_prev is not None:
            pred_s = Dw + be * self.Ds_prev - be * op * self.Dz_prev + A_(delta["g"]) - delta["s"]  # Eq. (Ds)
            pred_z = be * self.Dz_prev + A_(delta["l"]) - delta["z"]                              # Eq. (Dz)
        else:   # i = 0: Delta_{-1} = 0
            pred_s = Dw + A_(delta["g"]) - delta["s"]
            pred_z = A_(delta["l"]) - delta["z"]
        ident["s"] = _nrm(Ds - pred_s) / max(_nrm(Ds), 1e-300)
        ident["z"] = _nrm(Dz - pred_z) / max(_nrm(Dz), 1e-300)
        nrm64 = lambda key: float(np.linalg.norm(d[key]))
        cur = {key: nrm64(key) for key in ("x", "r", "k", "w", "g", "s", "l", "z", "q", "u", "y", "m", "t", "n", "v")}
        prev = dict(g=nrm64("g_prev"), s=nrm64("s_prev"), l=nrm64("l_prev"), z=nrm64("z_prev"),
                    n=nrm64("n_prev"), v=nrm64("v_prev"))
        bounds = delta_bounds(cur, prev, d["alpha"], d["beta"], d["omega"], d["omega_prev"], self.c, 2.0 ** -52)
        self.records.append(dict(i=i, delta={k_: _nrm(v_) for k_, v_ in delta.items()}, bound=bounds,
                                 gap=dict(r=_nrm(Dr), s=_nrm(Ds), w=_nrm(Dw), z=_nrm(Dz)),
                                 gap_r_next=_nrm(Dr_next), ident=ident, replaced=bool(d["replaced"])))
        if self.keep_vectors:   # the vectors themselves, extended precision
            self.records[-1].update(delta_vec=delta, gap_vec=dict(r=Dr, s=Ds, w=Dw, z=Dz),
                                    gap_next_vec=dict(r=Dr_next, w=Dw_next),
                                    scalars=dict(alpha=d["alpha"], beta=d["beta"], omega=d["omega"],
                                                 omega_prev=d["omega_prev"]))
        self.Ds_prev, self.Dz_prev, self.Dw_cur = Ds, Dz, Dw_next


class ClassicProbe:
    """Observer for ``krylov.bicgstab``: local errors of Eq. (auxrec0) and Eq. (classic_nomatrix).

    delta^x = x_{i+1} - (x_i + alpha M^{-1} p_i + omega M^{-1} q_i),
    delta^r = r_{i+1} - (q_i - omega A M^{-1} q_i),
    delta^q = q_i - (r_i - alpha A M^{-1} p_i)
    (the explicit products enter exactly, so their round-off is part of the deltas,
    as in the paper's bounds for Algorithm 1).  ``records[i]`` holds the gap
    ||Delta^r_{i+1}|| measured directly and predicted by the superposition
    Delta^r_0 - sum_j (A delta^x_j + delta^r_j + delta^q_j).
    """

    def __init__(self, A64, b, x0, precond_kind: str, dinv, degree: int):
        self.ops = _ExactOps(A64, precond_kind, dinv, degree)
        self.b = np.asarray(b, dtype=np.float64).astype(LD)
        self.sum = None
        self.records: List[dict] = []

    def __call__(self, stage, i, d):
        A_, M_ = self.ops.A_, self.ops.M_
        L = lambda key: d[key].astype(LD)
        al, om = LD(d["alpha"]), LD(d["omega"])
        if self.sum is None:
            self.sum = (self.b - A_(d["x"])) - L("r")       # Delta^r_0
        gex, uex = M_(d["p"]), M_(d["q"])
        dx = L("x_new") - (L("x") + al * gex + om * uex)
        dr = L("r_new") - (L("q") - om * A_(uex))
        dq = L("q") - (L("r") - al * A_(gex))
        self.sum = self.sum - (A_(dx) + dr + dq)
        gap = (self.b - A_(d["x_new"])) - L("r_new")
        self.records.append(dict(i=i, gap=_nrm(gap), pred=_nrm(self.sum),
                                 ident=_nrm(gap - self.sum) / max(_nrm(gap), 1e-300)))
