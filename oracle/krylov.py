"""Classic and pipelined preconditioned BiCGStab -- the oracle (test infrastructure only).

Written from arXiv 1809.01948:

* Algorithm 1 (classic preconditioned BiCGStab, Section 2.1).
* Algorithm 2 (preconditioned pipelined BiCGStab, Section 3), with the
  auxiliary vectors of Eq. (auxvars) and the evaluation order of Eq. (auxrec):
  left to right except where the paper brackets (numpy evaluates each binary
  operation with one IEEE rounding and never contracts into an FMA).
* The residual replacement step of Eq. (rr), executed after the w-update of
  Algorithm 2 (Section 3.6), with the periodic policy (replace every P
  iterations while ||r_i|| >= sqrt(eps) ||r_0||, Section 3.6 / 4.3) and the
  automated policy of Eq. (criterion) driven by the gap bound f^r of
  Eq. (DDr_bound).

Readings of points the paper leaves open (each one is also listed in the
design notes of the repository):

R1  Preconditioning side: both algorithms keep r = b - A x and update x with
    g = M^{-1} p, u = M^{-1} q (right preconditioning); the stop test uses the
    unpreconditioned ||r||.
R2  Shadow vector r_hat = the computed r_0 (stored separately).
R3  Vectors at i = -1 (g, s, l, z, n, v) are zero and omega_{-1} = 0.
R5  Stop: after iteration i, if ||r_{i+1}|| <= tol ||b||, the true residual
    ||b - A x_{i+1}|| is evaluated in FP64; if it also meets tol the solve has
    converged; otherwise, with a replacement policy enabled a replacement is
    forced and the iteration continues, and without one the solve returns
    STAGNATED.  b = 0 returns x = 0 after 0 iterations.
R6  Replacement placement (right after the w update): r_{i+1}, k_{i+1}, w_{i+1} are
    recomputed from x_{i+1}, and s_i, l_i, z_i from g_i, before the second
    global reduction; n_i and v_i are kept.
R7  Periodic policy: replace in iteration i when i > 0, i mod P == 0 and
    ||r_i|| >= sqrt(eps) ||r_0||, eps = 2^-52.
R8  Mixed mode adds a relative trigger: replace when ||r_i|| <= theta * (the
    recursive residual norm right after the previous replacement, or ||r_0||).
R15 Breakdown: a zero or non-finite alpha denominator, omega, (r_hat, r_i) or
    beta returns BREAKDOWN with the last finite x.  (y, y) == 0 sets omega = 0
    (y = 0 only when q = 0 in exact arithmetic), so the stop test decides.
    With max_restarts > 0 (not in the paper) a breakdown instead restarts the initialisation
    from the current iterate, with the new residual as the shadow vector; the
    iteration in which the breakdown was found counts as completed.
R20 Periodic restart (not in the paper; for the FP32 recurrences of mixed mode):
    with restart_period = P > 0, after every P completed iterations since the last
    (re)start the method restarts its initialisation from the current iterate: r = b - A x
    in FP64, the new r as the shadow vector, beta = 0 and zero g, s, l, z, n, v (reading
    R3).  It bounds how long the auxiliary recurrences' rounding errors can grow and is an
    FP64 outer correction around the inner FP32 iteration.  A failed R5 verification then
    restarts instead of returning STAGNATED.  The stop test at every (re)start uses the
    FP64 norm ||b - A x|| (identical to ||r_0|| in FP64 mode).
R21 Progress-based stagnation (stag_window = W > 0; the second half of the stop rule
    R5): at every (re)start the FP64 true residual is compared with a reference value;
    when it is at most half of it, it becomes the new reference, and when W or more
    iterations have passed since the reference was set without that, the solve returns
    STAGNATED with the iterate of the smallest true residual seen at a (re)start.  At
    max_it (NOT_CONVERGED) that iterate is also returned when its true residual is
    smaller than the last iterate's.

Mixed emulation (``mixed=True``): every vector except x and b is stored in
FP32 and every vector operation is evaluated in FP32 with the FP32-rounded
scalars; the SpMV and preconditioner use FP32 values; dot products are
accumulated in FP64 from the FP32 vectors; alpha, beta, omega are FP64; the
replacement residual r = b - A x uses FP64 values and FP64 x.  Parity of this
mode is partially pinned only (its pins are the FP64 oracle's attainable
accuracy and the replacement identities); the paper itself is FP64-only.
"""
from __future__ import annotations

import enum
import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from .precond import make_precond

EPS64 = 2.0 ** -52


class Status(enum.IntEnum):
    OK = 0
    INVALID_ARG = 1
    CUDA_ERROR = 2
    OUT_OF_MEMORY = 3
    NOT_CONVERGED = 4
    BREAKDOWN = 5
    STAGNATED = 6
    TIMEOUT = 7


@dataclass
class SolveResult:
    x: np.ndarray
    status: Status
    iterations: int
    n_replacements: int
    rel_res_recursive: float
    rel_res_true: float
    # per-iteration history (index i = iteration i):
    alpha: List[float] = field(default_factory=list)
    omega: List[float] = field(default_factory=list)
    beta: List[float] = field(default_factory=list)          # beta_{i+1}
    rnorm: List[float] = field(default_factory=list)         # ||r_{i+1}|| after any replacement
    replaced: List[bool] = field(default_factory=list)
    fr: List[float] = field(default_factory=list)            # gap bound f^r_{i+1} (auto policy)
    xs: List[np.ndarray] = field(default_factory=list)       # x_{i+1}, first `record` iterations
    n_restarts: int = 0


def _as_scipy(A):
    import scipy.sparse as sp
    if sp.issparse(A):
        return A.tocsr().astype(np.float64)
    return A.to_scipy(np.float64)


def spmv(A, v):
    """y = A v with the library's sparse matrix-vector product (row-wise, in column order)."""
    return A @ v


def _dot(a, b) -> float:
    """FP64 dot product of the stored vectors (FP32 inputs are widened exactly)."""
    return float(np.dot(a.astype(np.float64, copy=False), b.astype(np.float64, copy=False)))


def _true_res(A64, b, x) -> float:
    return float(np.linalg.norm(b - A64 @ x))


# ---------------------------------------------------------------------------
# Algorithm 1: classic preconditioned BiCGStab
# ---------------------------------------------------------------------------
def bicgstab(A, b, x0=None, precond: str = "none", degree: int = 0, tol: float = 1e-10,
             maxit: int = 1000, record: int = 0, observer: Optional[Callable] = None) -> SolveResult:
    """Algorithm 1 of the paper, FP64, shadow vector r_hat = r_0 (reading R2), stop rule R5
    without replacement."""
    A64 = _as_scipy(A)
    n = A64.shape[0]
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    M = make_precond(precond, A64, degree, np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return SolveResult(np.zeros(n), Status.OK, 0, 0, 0.0, 0.0)
    r = b - A64 @ x                     # r_0
    p = r.copy()
    rhat = r.copy()
    rho = _dot(rhat, r)
    res = SolveResult(x, Status.NOT_CONVERGED, 0, 0, 0.0, 0.0)
    rn = math.sqrt(_dot(r, r))
    if rn <= tol * bnorm:
        res.status, res.rel_res_recursive, res.rel_res_true = Status.OK, rn / bnorm, rn / bnorm
        return res
    for i in range(maxit):
        g = M.apply(p)                  # g_i = M^{-1} p_i
        s = A64 @ g                     # s_i = A g_i
        sig = _dot(rhat, s)             # (r_0, s_i)
        alpha = rho / sig if sig != 0.0 else math.inf   # alpha_i
        if sig == 0.0 or not math.isfinite(alpha):
            res.status = Status.BREAKDOWN
            break
        q = r - alpha * s               # q_i
        u = M.apply(q)                  # u_i = M^{-1} q_i
        y = A64 @ u                     # y_i = A u_i
        qy, yy = _dot(q, y), _dot(y, y)  # (q_i, y_i), (y_i, y_i)
        omega = 0.0 if yy == 0.0 else qy / yy  # omega_i
        if not math.isfinite(omega):
            res.status = Status.BREAKDOWN
            break
        x_old, r_old = x, r
        x = (x + alpha * g) + omega * u  # x_{i+1}
        r = q - omega * y                # r_{i+1}
        rho_new = _dot(rhat, r)          # (r_0, r_{i+1})
        rr = _dot(r, r)
        res.iterations = i + 1
        res.alpha.append(alpha)
        res.omega.append(omega)
        rn = math.sqrt(rr)
        res.rnorm.append(rn)
        res.replaced.append(False)
        if i < record:
            res.xs.append(x.copy())
        if observer is not None:
            observer("iter", i, dict(x=x_old, x_new=x, r=r_old, r_new=r, p=p, g=g, s=s, q=q, u=u, y=y,
                                     alpha=alpha, omega=omega))
        if rn <= tol * bnorm:
            tr = _true_res(A64, b, x)
            res.status = Status.OK if tr <= tol * bnorm else Status.STAGNATED
            break
        if omega == 0.0 or rho == 0.0:
            res.status = Status.BREAKDOWN
            break
        beta = (alpha / omega) * (rho_new / rho)   # beta_i
        if not math.isfinite(beta):
            res.status = Status.BREAKDOWN
            break
        res.beta.append(beta)
        p = r + beta * (p - omega * s)   # p_{i+1}
        rho = rho_new
    res.x = x
    res.rel_res_recursive = math.sqrt(_dot(r, r)) / bnorm
    res.rel_res_true = _true_res(A64, b, x) / bnorm
    return res


# ---------------------------------------------------------------------------
# Algorithm 2: preconditioned pipelined BiCGStab with residual replacement
# ---------------------------------------------------------------------------
def pbicgstab(A, b, x0=None, precond: str = "none", degree: int = 0, tol: float = 1e-10,
              maxit: int = 1000, rr_period: int = 0, rr_theta: float = 0.0, rr_auto: bool = False,
              rr_tau: Optional[float] = None, mixed: bool = False, record: int = 0,
              observer: Optional[Callable] = None, track_bound: bool = False,
              max_restarts: int = 0, restart_period: int = 0, stag_window: int = 0,
              contract: bool = False) -> SolveResult:
    """Algorithm 2 of the paper (lines cited as "l.N"), plus Eq. (rr) replacements.

    Replacement policies (any combination; all off means plain p-BiCGStab):
      rr_period = P > 0  periodic, reading R7;
      rr_theta  > 0      relative trigger, reading R8;
      rr_auto            Eq. (criterion) with tau = rr_tau (default sqrt(eps)).
    With any policy enabled, reading R5's forced replacement is also active.
    restart_period = P > 0 restarts the method every P iterations (reading R20);
    stag_window = W > 0 stops a solve that no longer makes progress (reading R21).
    ``contract`` (mixed mode only) evaluates every FP32 operation a + s c of the
    recurrences, and every FP32 row product, with one rounding, as a fused multiply-add
    does (reading R11): another equally valid evaluation, used to measure how much the
    FP32 iterates depend on the rounding of single operations.
    ``track_bound`` computes f^r (history ``fr``) without acting on it.
    ``observer(stage, i, vectors)`` is called with stage "init", "iter" (after
    the w update, before any replacement) and "replace" (after Eq. (rr)).
    """
    A64 = _as_scipy(A)
    n = A64.shape[0]
    T = np.float32 if mixed else np.float64
    AT = A64.astype(T)
    contract = contract and mixed
    if contract:
        AT = _OneRounding(AT)
    M = make_precond(precond, A64, degree, T)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    any_rr = rr_period > 0 or rr_theta > 0 or rr_auto
    bnorm = float(np.linalg.norm(b))
    res = SolveResult(x, Status.NOT_CONVERGED, 0, 0, 0.0, 0.0)
    if bnorm == 0.0:
        res.x, res.status = np.zeros(n), Status.OK
        return res
    sc = (lambda a: T(a))                     # scalar in the vector precision

    it = 0
    n_restarts = 0                          # breakdown restarts (bounded by max_restarts)
    n_periodic = 0                          # periodic restarts (reading R20)
    first = True
    rn0 = 0.0
    ref_true, ref_it = math.inf, 0          # reading R21
    best_true, x_best = math.inf, None
    eps = EPS64
    tau = math.sqrt(eps) if rr_tau is None else rr_tau
    fbound = _GapBound(A64, M, b, eps, mixed) if (rr_auto or track_bound) else None
    while True:                             # restarts after breakdowns (max_restarts)
        # initialisation of Algorithm 2
        r64 = b - A64 @ x
        r = r64.astype(T)
        rhat = r.copy()
        k = M.apply(r)
        w = AT @ k
        m = M.apply(w)
        t = AT @ m
        rho = _dot(rhat, r)
        rw = _dot(rhat, w)
        rn = math.sqrt(_dot(r, r))
        rt = math.sqrt(_dot(r64, r64))      # FP64 ||b - A x|| (= rn in FP64 mode)
        if first:
            rn0 = rn
        it_start = it
        if rt <= tol * bnorm:
            res.status, res.rel_res_recursive = Status.OK, rn / bnorm
            res.x, res.rel_res_true, res.iterations = x, _true_res(A64, b, x) / bnorm, it
            res.n_restarts = n_restarts + n_periodic
            return res
        if stag_window > 0:                 # reading R21
            if rt <= 0.5 * ref_true:
                ref_true, ref_it = rt, it
            elif it - ref_it >= stag_window:
                res.status, res.rel_res_recursive = Status.STAGNATED, rn / bnorm
                res.x = x_best if (x_best is not None and best_true < rt) else x
                res.rel_res_true, res.iterations = _true_res(A64, b, res.x) / bnorm, it
                res.n_restarts = n_restarts + n_periodic
                return res
            if rt < best_true:
                best_true, x_best = rt, x.copy()
        alpha = rho / rw if rw != 0.0 else math.inf
        if rw == 0.0 or not math.isfinite(alpha):
            res.status = Status.BREAKDOWN
            res.x, res.rel_res_recursive, res.rel_res_true = x, rn / bnorm, _true_res(A64, b, x) / bnorm
            return res
        beta = 0.0
        omega_prev = 0.0
        zero = np.zeros(n, dtype=T)
        g, s, l, z, nv, v = zero, zero, zero, zero, zero, zero   # reading R3
        rn_last_rr = rn
        if fbound is not None:
            fbound.start(x, rn)
        first = False
        restart = False

        def replace(x_, g_):
            """Eq. (rr): r = b - A x, k = M^{-1} r, w = A k, s = A g, l = M^{-1} s, z = A l."""
            r_ = (b - A64 @ x_).astype(T)
            k_ = M.apply(r_)
            w_ = AT @ k_
            s_ = (A64 @ g_.astype(np.float64)).astype(T)
            l_ = M.apply(s_)
            z_ = AT @ l_
            return r_, k_, w_, s_, l_, z_

        if observer is not None:
            observer("init", -1, dict(x=x, r=r, k=k, w=w, m=m, t=t))
        fr_hist = [fbound.f] if fbound is not None else None   # f^r_i, i = 0, 1, ...
        rn_hist = [rn]                                          # ||r_i||
        while it < maxit:
            i = it
            a_, b_, wp_ = sc(alpha), sc(beta), sc(omega_prev)
            g_prev, l_prev, s_prev, z_prev, n_prev, v_prev = g, l, s, z, nv, v
            if not contract:
                g = k + b_ * (g - wp_ * l)          # g_i
                s = w + b_ * (s - wp_ * z)          # s_i
                l = m + b_ * (l - wp_ * nv)         # l_i
                z = t + b_ * (z - wp_ * v)          # z_i
                q = r - a_ * s                      # q_i
                u = k - a_ * l                      # u_i
                y = w - a_ * z                      # y_i
            else:                                   # the same with one rounding per a + s c
                g = _fma(k, b_, _fma(g, -wp_, l))
                s = _fma(w, b_, _fma(s, -wp_, z))
                l = _fma(m, b_, _fma(l, -wp_, nv))
                z = _fma(t, b_, _fma(z, -wp_, v))
                q = _fma(r, -a_, s)
                u = _fma(k, -a_, l)
                y = _fma(w, -a_, z)
            qy, yy = _dot(q, y), _dot(y, y)     # first global reduction
            nv = M.apply(z)                     # n_i = M^{-1} z_i
            v = AT @ nv                         # v_i = A n_i
            omega = 0.0 if yy == 0.0 else qy / yy   # omega_i
            if not math.isfinite(omega):
                if n_restarts < max_restarts:
                    n_restarts += 1
                    it += 1
                    restart = True
                    break
                res.status = Status.BREAKDOWN
                break
            o_ = sc(omega)
            # replacement decision for this iteration (uses only quantities known now)
            do_rr = False
            if rr_period > 0 and i > 0 and i % rr_period == 0 and rn >= math.sqrt(eps) * rn0:
                do_rr = True                                             # reading R7
            if rr_theta > 0 and rn <= rr_theta * rn_last_rr:
                do_rr = True                                             # reading R8
            if rr_auto and len(fr_hist) >= 2 and (fr_hist[-2] <= tau * rn_hist[-2] and fr_hist[-1] > tau * rn_hist[-1]):
                do_rr = True                                             # Eq. (criterion)
            x_old = x
            x = (x + alpha * g.astype(np.float64)) + omega * u.astype(np.float64)   # x_{i+1}
            if not contract:
                r_new = q - o_ * y                  # r_{i+1}
                k_new = u - o_ * (m - a_ * nv)      # k_{i+1}
                w_new = y - o_ * (t - a_ * v)       # w_{i+1}
            else:
                r_new = _fma(q, -o_, y)
                k_new = _fma(u, -o_, _fma(m, -a_, nv))
                w_new = _fma(y, -o_, _fma(t, -a_, v))
            if observer is not None:
                observer("iter", i, dict(x=x_old, x_new=x, r=r, k=k, w=w, g=g, s=s, l=l, z=z, q=q, u=u,
                                         y=y, m=m, t=t, n=nv, v=v, r_new=r_new, k_new=k_new,
                                         w_new=w_new, g_prev=g_prev, l_prev=l_prev, s_prev=s_prev,
                                         z_prev=z_prev, n_prev=n_prev, v_prev=v_prev, alpha=alpha,
                                         beta=beta, omega=omega, omega_prev=omega_prev, replaced=do_rr))
            if fbound is not None:
                fbound.step(alpha, beta, omega, omega_prev, x_old, r, k, w, g, s, l, z, q, u, y, m, t, nv, v)
            r, k, w = r_new, k_new, w_new
            if do_rr:                           # Eq. (rr), right after the w update (reading R6)
                r, k, w, s, l, z = replace(x, g)
                res.n_replacements += 1
                if observer is not None:
                    observer("replace", i, dict(x=x, r=r, k=k, w=w, g=g, s=s, l=l, z=z))
                if fbound is not None:
                    fbound.reset(x, k, g, s, l, z)
            # second global reduction, overlapped with m = M^{-1} w, t = A m
            rho_new, rw, rs, rz = _dot(rhat, r), _dot(rhat, w), _dot(rhat, s), _dot(rhat, z)
            rr = _dot(r, r)
            m = M.apply(w)                      # m_{i+1}
            t = AT @ m                          # t_{i+1}
            res.iterations = i + 1
            rn = math.sqrt(rr)
            if rn <= tol * bnorm:               # reading R5
                tr = _true_res(A64, b, x)
                if tr <= tol * bnorm:
                    res.status = Status.OK
                    _log(res, alpha, omega, None, rn, do_rr, x, i, record, fbound)
                    break
                if not any_rr:
                    _log(res, alpha, omega, None, rn, do_rr, x, i, record, fbound)
                    if restart_period > 0:          # reading R20: restart from x instead
                        n_periodic += 1
                        it += 1
                        restart = True
                        break
                    res.status = Status.STAGNATED
                    break
                r, k, w, s, l, z = replace(x, g)     # forced replacement
                res.n_replacements += 1
                do_rr = True
                if observer is not None:
                    observer("replace", i, dict(x=x, r=r, k=k, w=w, g=g, s=s, l=l, z=z))
                if fbound is not None:
                    fbound.reset(x, k, g, s, l, z)
                rho_new, rw, rs, rz = _dot(rhat, r), _dot(rhat, w), _dot(rhat, s), _dot(rhat, z)
                rn = math.sqrt(_dot(r, r))
                m = M.apply(w)
                t = AT @ m
            if do_rr:
                rn_last_rr = rn
            rn_hist.append(rn)
            if fbound is not None:
                fr_hist.append(fbound.f)
            if omega == 0.0 or rho == 0.0:
                _log(res, alpha, omega, None, rn, do_rr, x, i, record, fbound)
                if n_restarts < max_restarts:
                    n_restarts += 1
                    it += 1
                    restart = True
                    break
                res.status = Status.BREAKDOWN
                break
            beta_new = (alpha / omega) * (rho_new / rho)                        # beta_{i+1}
            den = (rw + beta_new * rs) - (beta_new * omega) * rz                # alpha_{i+1} = rho_new / den
            alpha_new = rho_new / den if den != 0.0 else math.inf
            _log(res, alpha, omega, beta_new, rn, do_rr, x, i, record, fbound)
            if not (math.isfinite(beta_new) and den != 0.0 and math.isfinite(alpha_new)):
                if n_restarts < max_restarts:
                    n_restarts += 1
                    it += 1
                    restart = True
                    break
                res.status = Status.BREAKDOWN
                break
            alpha, beta, omega_prev, rho = alpha_new, beta_new, omega, rho_new
            it += 1
            if restart_period > 0 and it - it_start >= restart_period:   # reading R20
                n_periodic += 1
                restart = True
                break
        if not restart:
            break
    res.n_restarts = n_restarts + n_periodic
    if res.status == Status.NOT_CONVERGED and x_best is not None and best_true < _true_res(A64, b, x):
        x = x_best                          # reading R21
    res.x = x
    res.rel_res_recursive = rn / bnorm
    res.rel_res_true = _true_res(A64, b, x) / bnorm
    return res


def _fma(a, s, c):
    """a + s c for FP32 vectors a, c and an FP32 scalar s, rounded once to FP32 (the FP32
    product is exact in FP64; the FP64 sum is then rounded to FP32)."""
    return (a.astype(np.float64) + np.float64(s) * c.astype(np.float64)).astype(np.float32)


class _OneRounding:
    """An FP32 matrix whose row products are accumulated in FP64 and rounded once to FP32."""

    def __init__(self, A32):
        self.A = A32.astype(np.float64)

    def __matmul__(self, v):
        return (self.A @ v.astype(np.float64)).astype(np.float32)


def _log(res, alpha, omega, beta_new, rn, replaced, x, i, record, fbound):
    res.alpha.append(alpha)
    res.omega.append(omega)
    if beta_new is not None:
        res.beta.append(beta_new)
    res.rnorm.append(rn)
    res.replaced.append(bool(replaced))
    if fbound is not None:
        res.fr.append(fbound.f)
    if i < record:
        res.xs.append(x.copy())


class _GapBound:
    """Run-time gap bound f^r of Eq. (DDr_bound) for the automated policy, Eq. (criterion).

    The norms of the local rounding errors are replaced by their bounds from
    Eq. (errbounds1)-(errbounds4) (``diagnostics.delta_bounds``), and the gap
    norms ||Delta^s||, ||Delta^w||, ||Delta^z|| by the triangle-inequality
    bounds F^s, F^w, F^z of Eqs. (Ds), (Dw), (Dz), evaluated in iteration i as
        F^z_i     = |beta_i| F^z_{i-1} + ||A|| d^l_i + d^z_i
        F^s_i     = F^w_i + |beta_i| F^s_{i-1} + |beta_i omega_{i-1}| F^z_{i-1} + ||A|| d^g_i + d^s_i
        f^r_{i+1} = f^r_i + |alpha_i| F^s_i + |omega_i| F^w_i + |omega_i alpha_i| F^z_i
                    + ||A|| d^x_i + d^r_i + |omega_i| ||A|| d^u_i + d^q_i + |omega_i| d^y_i
        F^w_{i+1} = F^w_i + |alpha_i| F^z_i + ||A|| (d^k_i + d^u_i) + d^w_i + d^y_i
    (d^* = the bound on ||delta^*||).  Initial values, and the values after a
    replacement, are the round-off bounds of the explicitly computed vectors:
    F^z = mu sqrt(N) ||A|| ||l|| eps, F^w = mu sqrt(N) ||A|| ||k|| eps,
    F^s = mu sqrt(N) ||A|| ||g|| eps and f^r = ((mu sqrt(N) + 1) ||A|| ||x|| + ||b||) eps.

    Parity partially pinned: f^r is an upper bound and its pins are inequalities
    (||Delta^r_i|| <= f^r_i on every iteration of real runs, and after a replacement).
    """

    def __init__(self, A64, M, b, eps, mixed):
        from . import diagnostics
        self.d = diagnostics
        self.eps = 2.0 ** -23 if mixed else eps
        self.consts = diagnostics.bound_constants(A64, M)
        self.bnorm = float(np.linalg.norm(b))
        self.f = 0.0
        self.prev = None

    @staticmethod
    def _nrm(a) -> float:
        return float(np.linalg.norm(a.astype(np.float64)))

    def start(self, x, rn):
        c = self.consts
        self.f = ((c["mu"] * c["sqrtN"] + 1) * c["nA"] * self._nrm(x) + self.bnorm) * self.eps
        self.first = True

    def step(self, alpha, beta, omega, omega_prev, x, r, k, w, g, s, l, z, q, u, y, m, t, n, v):
        nrm = self._nrm
        cur = dict(x=nrm(x), r=nrm(r), k=nrm(k), w=nrm(w), g=nrm(g), s=nrm(s), l=nrm(l), z=nrm(z),
                   q=nrm(q), u=nrm(u), y=nrm(y), m=nrm(m), t=nrm(t), n=nrm(n), v=nrm(v))
        c = self.consts
        msn, nA = c["mu"] * c["sqrtN"], c["nA"]
        if self.first:
            zero = {key: 0.0 for key in cur}
            db = self.d.delta_bounds(cur, zero, alpha, beta, omega, omega_prev, c, self.eps)
            self.Fz = msn * nA * cur["l"] * self.eps     # z_0 = t_0 = fl(A m_0), l_0 = m_0
            self.Fw = msn * nA * cur["k"] * self.eps     # w_0 = fl(A k_0)
            self.Fs = msn * nA * cur["g"] * self.eps     # s_0 = w_0, g_0 = k_0
            self.first = False
        else:
            db = self.d.delta_bounds(cur, self.prev, alpha, beta, omega, omega_prev, c, self.eps)
            Fz = abs(beta) * self.Fz + nA * db["l"] + db["z"]
            Fs = self.Fw + abs(beta) * self.Fs + abs(beta * omega_prev) * self.Fz + nA * db["g"] + db["s"]
            self.Fz, self.Fs = Fz, Fs
        self.f = (self.f + abs(alpha) * self.Fs + abs(omega) * self.Fw + abs(omega * alpha) * self.Fz
                  + nA * db["x"] + db["r"] + abs(omega) * nA * db["u"] + db["q"] + abs(omega) * db["y"])
        self.Fw = self.Fw + abs(alpha) * self.Fz + nA * (db["k"] + db["u"]) + db["w"] + db["y"]
        self.prev = cur

    def reset(self, x, k, g, s, l, z):
        """After Eq. (rr): all gaps restart from the round-off of the explicit recomputation."""
        c = self.consts
        msn, nA, nrm = c["mu"] * c["sqrtN"], c["nA"], self._nrm
        self.f = ((msn + 1) * nA * nrm(x) + self.bnorm) * self.eps
        self.Fw = msn * nA * nrm(k) * self.eps
        self.Fs = msn * nA * nrm(g) * self.eps
        self.Fz = msn * nA * nrm(l) * self.eps
        if self.prev is not None:
            self.prev = dict(self.prev, s=nrm(s), l=nrm(l), z=nrm(z))
