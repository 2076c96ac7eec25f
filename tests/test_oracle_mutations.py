"""Planted mistakes in the oracle: each mutant below is the oracle's own source with one
plausible slip (a flipped sign, a wrong operand or index, a swapped scalar), and each must
fail at least one pin of this file -- evidence that the pins would have caught that slip in
the oracle itself.  Everything runs on the CPU; the CUDA path is not involved.

Pins (all independent of the oracle under test):
* Algorithm 1 and Algorithm 2 iterates equal scipy's BiCGStab iterates (same shadow vector
  r_0, right preconditioning) over the first iterations -- the exact-arithmetic equivalence
  of Section 3, on a constant-diagonal Jacobi problem and on a random unsymmetric system
  with a varying diagonal;
* the solve with periodic replacement converges to the dense LAPACK solution, replaces in
  iterations P, 2P, ... (reading R7), and every replacement of Eq. (rr) leaves
  r = b - A x, w = A k, s = A g, z = A l and k = M^{-1} r, l = M^{-1} s, checked with
  separate scipy products;
* Neumann preconditioning (degree 2) gives the same iterates as scipy's BiCGStab with the
  explicit polynomial as M.
"""
import sys
import types

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import testproblems as tp
from oracle import krylov

SOURCE = open(krylov.__file__).read()

# (name, original text, mutated text): each original occurs exactly once in the oracle.
PIPELINED = [
    ("g: sign of omega term", "g = k + b_ * (g - wp_ * l)", "g = k + b_ * (g + wp_ * l)"),
    ("g: l -> s", "g = k + b_ * (g - wp_ * l)", "g = k + b_ * (g - wp_ * s)"),
    ("s: z -> v", "s = w + b_ * (s - wp_ * z)", "s = w + b_ * (s - wp_ * v)"),
    ("l: n -> z", "l = m + b_ * (l - wp_ * nv)", "l = m + b_ * (l - wp_ * z)"),
    ("l: m -> w", "l = m + b_ * (l - wp_ * nv)", "l = w + b_ * (l - wp_ * nv)"),
    ("z: beta -> alpha", "z = t + b_ * (z - wp_ * v)", "z = t + a_ * (z - wp_ * v)"),
    ("q: s -> z", "q = r - a_ * s ", "q = r - a_ * z "),
    ("u: l -> s", "u = k - a_ * l ", "u = k - a_ * s "),
    ("y: z -> s", "y = w - a_ * z ", "y = w - a_ * s "),
    ("omega: (y,y) -> (q,q)", "qy, yy = _dot(q, y), _dot(y, y)     # first", "qy, yy = _dot(q, y), _dot(q, q)     # first"),
    ("n: M z -> M s", "nv = M.apply(z) ", "nv = M.apply(s) "),
    ("v: A n -> A z", "v = AT @ nv ", "v = AT @ z "),
    ("x: u -> q", "+ omega * u.astype(np.float64)", "+ omega * q.astype(np.float64)"),
    ("x: alpha g -> alpha k", "x = (x + alpha * g.astype(np.float64))", "x = (x + alpha * k.astype(np.float64))"),
    ("r: sign", "r_new = q - o_ * y ", "r_new = q + o_ * y "),
    ("k: n -> v", "k_new = u - o_ * (m - a_ * nv)", "k_new = u - o_ * (m - a_ * v)"),
    ("w: v -> n", "w_new = y - o_ * (t - a_ * v)", "w_new = y - o_ * (t - a_ * nv)"),
    ("m: M w -> M r", "m = M.apply(w)                      # m_{i+1}", "m = M.apply(r)                      # m_{i+1}"),
    ("t: A m -> A w", "t = AT @ m                          # t_{i+1}", "t = AT @ w                          # t_{i+1}"),
    ("(r0,s) <-> (r0,z)", "_dot(rhat, w), _dot(rhat, s), _dot(rhat, z)\n            rr",
     "_dot(rhat, w), _dot(rhat, z), _dot(rhat, s)\n            rr"),
    ("beta: alpha/omega inverted", "beta_new = (alpha / omega) * (rho_new / rho)", "beta_new = (omega / alpha) * (rho_new / rho)"),
    ("alpha denominator: sign of z term", "den = (rw + beta_new * rs) - (beta_new * omega) * rz",
     "den = (rw + beta_new * rs) + (beta_new * omega) * rz"),
    ("alpha denominator: rz -> rs", "den = (rw + beta_new * rs) - (beta_new * omega) * rz",
     "den = (rw + beta_new * rs) - (beta_new * omega) * rs"),
    ("init: alpha_0 = (r,r)/(r,r)", "rw = _dot(rhat, w)\n        rn", "rw = _dot(rhat, r)\n        rn"),
    ("init: k_0 = r_0", "k = M.apply(r)\n        w = AT @ k", "k = r.copy()\n        w = AT @ k"),
    ("Eq. rr: r = b - A g", "r_ = (b - A64 @ x_).astype(T)", "r_ = (b - A64 @ g_.astype(np.float64)).astype(T)"),
    ("Eq. rr: s = A k", "s_ = (A64 @ g_.astype(np.float64)).astype(T)", "s_ = (A64 @ k_.astype(np.float64)).astype(T)"),
    ("Eq. rr: l = M r", "l_ = M.apply(s_)", "l_ = M.apply(r_)"),
    ("Eq. rr: z = A s", "z_ = AT @ l_", "z_ = AT @ s_"),
    ("R7: period phase", "i > 0 and i % rr_period == 0 and", "i > 0 and i % rr_period == 1 and"),
    ("R7: cutoff inverted", "rn >= math.sqrt(eps) * rn0:", "rn <= math.sqrt(eps) * rn0:"),
]

CLASSIC = [
    ("Alg. 1: s = A g -> A p", "s = A64 @ g ", "s = A64 @ p "),
    ("Alg. 1: sign of alpha s in q", "q = r - alpha * s ", "q = r + alpha * s "),
    ("Alg. 1: omega = (q,y)/(y,y) -> (q,y)/(q,q)", "qy, yy = _dot(q, y), _dot(y, y)  #",
     "qy, yy = _dot(q, y), _dot(q, q)  #"),
    ("Alg. 1: x update u -> q", "x = (x + alpha * g) + omega * u ", "x = (x + alpha * g) + omega * q "),
    ("Alg. 1: beta with the rho ratio inverted", "beta = (alpha / omega) * (rho_new / rho)", "beta = (alpha / omega) * (rho / rho_new)"),
    ("Alg. 1: p update s -> y", "p = r + beta * (p - omega * s)", "p = r + beta * (p - omega * y)"),
]


def _load(src):
    """Execute oracle source text as a throw-away module of the oracle package."""
    name = "oracle._mutant"
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    mod.__file__ = krylov.__file__
    sys.modules[name] = mod   # dataclasses look their module up while the class is built
    try:
        exec(compile(src, "<oracle mutant>", "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _mutant(old, new):
    assert SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    return _load(SOURCE.replace(old, new))


# ---------------------------------------------------------------- fixed inputs and references
def _scipy_iterates(A, b, nit, minv=None):
    xs = []
    M = None if minv is None else spl.LinearOperator(A.shape, matvec=minv)
    spl.bicgstab(A, b, rtol=1e-30, maxiter=nit, M=M, callback=lambda x: xs.append(x.copy()))
    return xs


def _cases():
    p = tp.problem_convdiff2d(20)                      # constant diagonal
    A1 = p.A.to_scipy()
    rng = np.random.Generator(np.random.PCG64(21))
    A2 = tp.random_banded_system(300, rng, band=16).to_scipy(np.float64)   # varying diagonal
    b2 = A2 @ rng.uniform(-1.0, 1.0, 300)
    p3 = tp.problem_convdiff2d(12)                     # Neumann degree 2
    A3 = p3.A.to_scipy()
    d3 = 1.0 / A3.diagonal()

    def neumann2(v):   # M^{-1} = (I + (I - D^{-1}A) + (I - D^{-1}A)^2) D^{-1}
        y0 = d3 * v
        y1 = y0 + (y0 - d3 * (A3 @ y0))
        return y0 + (y1 - d3 * (A3 @ y1))
    return [
        (A1, p.b, "jacobi", 0, _scipy_iterates(A1, p.b, 10, lambda v: v / A1.diagonal())),
        (A2, b2, "jacobi", 0, _scipy_iterates(A2, b2, 10, lambda v: v / A2.diagonal())),
        (A3, p3.b, "neumann", 2, _scipy_iterates(A3, p3.b, 10, neumann2)),
    ]


CASES = None


def _iterate_pins(solver):
    """True when the first 10 iterates of `solver` match scipy's on every case."""
    global CASES
    if CASES is None:
        CASES = _cases()
    for A, b, prec, deg, ref in CASES:
        r = solver(A, b, precond=prec, degree=deg, tol=1e-30, maxit=10, record=10)
        if len(r.xs) < 10:
            return False
        for i in range(10):
            if not np.linalg.norm(r.xs[i] - ref[i]) <= 1e-8 * np.linalg.norm(ref[i]):
                return False
    return True


def _replacement_pins(mod):
    """Periodic replacement (P = 10) on the 24x24 convection-diffusion system with Jacobi
    (57 iterations, replacements in iterations 10-40): the schedule of reading R7, the
    identities Eq. (rr) establishes, and the dense solution."""
    p = tp.problem_convdiff2d(24)
    A = p.A.to_scipy()
    b, xs = p.b, p.x_star
    dinv = 1.0 / A.diagonal()
    bad = []

    def obs(stage, i, d):
        if stage != "replace":
            return
        x, g = d["x"], d["g"].astype(np.float64)
        checks = [(b - A @ x, d["r"]), (A @ d["k"], d["w"]), (A @ g, d["s"]), (A @ d["l"], d["z"]),
                  (dinv * d["r"], d["k"]), (dinv * d["s"], d["l"])]
        for want, got in checks:
            if not np.linalg.norm(want - got) <= 1e-12 * max(1.0, np.linalg.norm(want)):
                bad.append(i)
    r = mod.pbicgstab(A, b, precond="jacobi", tol=1e-12, maxit=600, rr_period=10, observer=obs)
    rep = [i for i, f in enumerate(r.replaced) if f]
    schedule_ok = len(rep) >= 3 and all(i % 10 == 0 for i in rep[:-1]) and rep[0] == 10
    solved = int(r.status) == 0 and np.linalg.norm(r.x - np.linalg.solve(A.toarray(), b)) <= 1e-9 * np.linalg.norm(xs)
    return schedule_ok and solved and not bad


def _pipelined_pins_pass(mod):
    try:
        return _iterate_pins(mod.pbicgstab) and _replacement_pins(mod)
    except (FloatingPointError, ValueError, ZeroDivisionError, OverflowError, np.linalg.LinAlgError):
        return False


def _classic_pins_pass(mod):
    try:
        return _iterate_pins(mod.bicgstab)
    except (FloatingPointError, ValueError, ZeroDivisionError, OverflowError, np.linalg.LinAlgError):
        return False


def test_unmutated_oracle_passes_every_pin():
    mod = _load(SOURCE)
    assert _pipelined_pins_pass(mod)
    assert _classic_pins_pass(mod)


@pytest.mark.parametrize("name,old,new", PIPELINED, ids=[m[0] for m in PIPELINED])
def test_pipelined_mutant_fails_a_pin(name, old, new):
    with np.errstate(all="ignore"):
        assert not _pipelined_pins_pass(_mutant(old, new)), name


@pytest.mark.parametrize("name,old,new", CLASSIC, ids=[m[0] for m in CLASSIC])
def test_classic_mutant_fails_a_pin(name, old, new):
    with np.errstate(all="ignore"):
        assert not _classic_pins_pass(_mutant(old, new)), name


# ---------------------------------------------------------------- mixed-precision emulation
MIXED = [
    ("mixed: FP64 operator in the recurrences", "AT = A64.astype(T)", "AT = A64"),
    ("mixed: preconditioner in FP64", "M = make_precond(precond, A64, degree, T)",
     "M = make_precond(precond, A64, degree, np.float64)"),
    ("mixed: replacement residual with FP32 values", "r_ = (b - A64 @ x_).astype(T)", "r_ = (b - AT @ x_).astype(T)"),
    ("mixed: replacement s with FP32 values", "s_ = (A64 @ g_.astype(np.float64)).astype(T)", "s_ = (AT @ g_).astype(T)"),
    ("mixed: x accumulated in FP32", "x = (x + alpha * g.astype(np.float64)) + omega * u.astype(np.float64)",
     "x = ((x.astype(T) + a_ * g) + o_ * u).astype(np.float64)"),
]


def _mixed_pins_fail(monkeypatch, mod):
    import oracle
    import test_oracle_replacement as TR
    monkeypatch.setattr(oracle, "pbicgstab", mod.pbicgstab)
    failed = []
    for fn in (TR.test_mixed_first_iterates_track_fp64, TR.test_mixed_with_replacement_reaches_1e10,
               TR.test_mixed_emulation_keeps_vectors_in_fp32):
        try:
            with np.errstate(all="ignore"):
                fn()
        except (AssertionError, FloatingPointError, ValueError):
            failed.append(fn.__name__)
    return failed


def test_unmutated_mixed_emulation_passes(monkeypatch):
    assert _mixed_pins_fail(monkeypatch, _load(SOURCE)) == []


@pytest.mark.parametrize("name,old,new", MIXED, ids=[m[0] for m in MIXED])
def test_mixed_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert _mixed_pins_fail(monkeypatch, _mutant(old, new)), name
