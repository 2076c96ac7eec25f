"""Pins of the oracle's rounding-error bound formulas that do not retype them.

1. Eqs. (errbounds1)-(errbounds4), the local rounding-error bounds of Algorithm 2, follow
   mechanically from the paper's floating-point model of Section 2 (the rounding error of
   a scalar product, a vector sum and an SPMV / PREC application, each bounded by the norms
   of its operands times epsilon) applied, to first order, to the expressions of
   Eq. (auxrec) with their brackets and left-to-right order, the products of Eq. (auxvars2)
   being the explicitly computed ones.  ``compose`` below implements those four rules and
   nothing else; the bounds it derives must equal ``diagnostics.delta_bounds`` term by
   term (every monomial in the norms and scalars, with its coefficient).

2. The run-time gap bound f^r of Eq. (DDr_bound) (with reading R14's F^s, F^w, F^z) is the
   triangle inequality applied to the gap identities Eqs. (Dr), (Ds), (Dw), (Dz).  The
   identities are written below once, as data; that data is first checked against the
   gaps and local errors measured in extended precision on a real solve (so a wrong sign,
   scalar or operand in it fails), then turned into the bound recurrences, which must equal
   ``krylov._GapBound`` step by step.  The initial (and post-replacement) values come from
   composing the same rules over r_0 = b - A x_0 and the explicit products.
"""
import math
from collections import Counter

import numpy as np
import pytest

import testproblems as tp
from oracle import diagnostics, krylov
from oracle.precond import make_precond

EPS = 2.0 ** -52


# --------------------------------------------------------------------------- composer
# An expression carries two linear combinations of monomials (tuples of factor names):
# ``mag`` bounds the norm of its computed value, ``err`` its accumulated rounding error
# (in units of epsilon).  Factor names: vector norms, |scalar| names, and the constants
# nA = ||A||, nM = ||M^{-1}||, msn = mu sqrt(N), tmsn = mu~ sqrt(N).
def _mul(c, f):
    return Counter({tuple(sorted(k + (f,))): v for k, v in c.items()})


def _add(*cs):
    out = Counter()
    for c in cs:
        out.update(c)
    return out


def leaf(name):
    """A stored vector: its norm is known, it carries no error of this step."""
    return (Counter({(name,): 1}), Counter())


def scale(s, e):
    """fl(s v): ||s v - fl(s v)|| <= |s| ||v|| eps."""
    mag, err = e
    return (_mul(mag, s), _add(_mul(err, s), _mul(mag, s)))


def plus(e1, e2):
    """fl(v + w) or fl(v - w): error <= (||v|| + ||w||) eps."""
    return (_add(e1[0], e2[0]), _add(e1[1], e2[1], e1[0], e2[0]))


def product(kind, e, name=None):
    """fl(A v) (kind "A") or fl(M^{-1} v) (kind "M"): error <= mu sqrt(N) ||A|| ||v|| eps
    (mu~, M^{-1} for PREC).  ``name``: the paper names the computed vector (m, n, t, v) and
    bounds later uses by its own norm; unnamed, its norm is bounded by ||A|| ||v||."""
    mag, err = e
    nrm, cst = ("nA", "msn") if kind == "A" else ("nM", "tmsn")
    new_mag = Counter({(name,): 1}) if name else _mul(mag, nrm)
    return (new_mag, _add(_mul(err, nrm), _mul(_mul(mag, nrm), cst)))


def auxrec_bounds():
    """Eq. (auxrec) as written, with Eq. (auxvars2)'s explicit products."""
    m = product("M", leaf("w"), "m")
    n = product("M", leaf("z"), "n")
    n_prev = product("M", leaf("z_prev"), "n_prev")
    t = product("A", m, "t")
    v = product("A", n, "v")
    v_prev = product("A", n_prev, "v_prev")
    tree = {
        "g": plus(leaf("k"), scale("beta", plus(leaf("g_prev"), scale("omega_prev", leaf("l_prev"))))),
        "x": plus(plus(leaf("x"), scale("alpha", leaf("g"))), scale("omega", leaf("u"))),
        "q": plus(leaf("r"), scale("alpha", leaf("s"))),
        "s": plus(leaf("w"), scale("beta", plus(leaf("s_prev"), scale("omega_prev", leaf("z_prev"))))),
        "r": plus(leaf("q"), scale("omega", leaf("y"))),
        "u": plus(leaf("k"), scale("alpha", leaf("l"))),
        "l": plus(m, scale("beta", plus(leaf("l_prev"), scale("omega_prev", n_prev)))),
        "k": plus(leaf("u"), scale("omega", plus(m, scale("alpha", n)))),
        "y": plus(leaf("w"), scale("alpha", leaf("z"))),
        "z": plus(t, scale("beta", plus(leaf("z_prev"), scale("omega_prev", v_prev)))),
        "w": plus(leaf("y"), scale("omega", plus(t, scale("alpha", v)))),
    }
    return {key: e[1] for key, e in tree.items()}


VEC_CUR = ("x", "r", "k", "w", "g", "s", "l", "z", "q", "u", "y", "m", "t", "n", "v")
VEC_PREV = ("g", "s", "l", "z", "n", "v")


def _evaluate(poly, values):
    return sum(c * math.prod(values[f] for f in mono) for mono, c in poly.items())


def _values(rng, zero_except=None):
    vals = {k: float(rng.uniform(0.1, 3.0)) for k in VEC_CUR}
    vals.update({k + "_prev": float(rng.uniform(0.1, 3.0)) for k in VEC_PREV})
    if zero_except is not None:
        for k in list(vals):
            if k != zero_except:
                vals[k] = 0.0
    consts = dict(mu=float(rng.integers(3, 16)), mut=float(rng.integers(1, 30)), sqrtN=float(rng.uniform(5, 50)),
                  nA=float(rng.uniform(0.5, 2.0)), nM=float(rng.uniform(0.1, 2.0)))
    scal = dict(alpha=float(rng.uniform(-2, 2)), beta=float(rng.uniform(-2, 2)), omega=float(rng.uniform(-2, 2)),
                omega_prev=float(rng.uniform(-2, 2)))
    return vals, consts, scal


def _oracle_bounds(vals, consts, scal):
    cur = {k: vals[k] for k in VEC_CUR}
    prev = {k: vals[k + "_prev"] for k in VEC_PREV}
    return diagnostics.delta_bounds(cur, prev, scal["alpha"], scal["beta"], scal["omega"], scal["omega_prev"],
                                    consts, EPS)


def _factor_values(vals, consts, scal):
    fv = dict(vals)
    fv.update({k: abs(v) for k, v in scal.items()})
    fv.update(nA=consts["nA"], nM=consts["nM"], msn=consts["mu"] * consts["sqrtN"],
              tmsn=consts["mut"] * consts["sqrtN"])
    return fv


def test_composed_bounds_have_the_printed_structure():
    """Spot checks against the printed coefficients: the composition gives 3|beta| ||g_{i-1}||
    and 4|beta omega_{i-1}| ||l_{i-1}|| in delta^g, and mu~ sqrt(N) ||M^{-1}|| ||w|| in delta^l."""
    b = auxrec_bounds()
    assert b["g"] == Counter({("k",): 1, ("beta", "g_prev"): 3, ("beta", "l_prev", "omega_prev"): 4})
    assert b["l"][("nM", "tmsn", "w")] == 1 and b["l"][("beta", "n_prev", "omega_prev")] == 4
    assert b["x"] == Counter({("x",): 2, ("alpha", "g"): 3, ("omega", "u"): 2})


def test_delta_bounds_equal_the_composed_bounds():
    """Polynomial identity at random points: every bound of diagnostics.delta_bounds equals
    the composition of the floating-point model over Eq. (auxrec)."""
    derived = auxrec_bounds()
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(20):
        vals, consts, scal = _values(rng)
        got = _oracle_bounds(vals, consts, scal)
        fv = _factor_values(vals, consts, scal)
        for key, poly in derived.items():
            want = _evaluate(poly, fv) * EPS
            assert abs(got[key] - want) <= 1e-13 * want, (key, got[key], want)


def test_delta_bounds_term_by_term():
    """Each vector norm alone: the terms that contain it, with their coefficients and
    scalar factors, are the composed ones (a dropped, doubled or mis-indexed term fails)."""
    derived = auxrec_bounds()
    rng = np.random.Generator(np.random.PCG64(12))
    for vec in VEC_CUR + tuple(k + "_prev" for k in VEC_PREV):
        for _ in range(3):
            vals, consts, scal = _values(rng, zero_except=vec)
            got = _oracle_bounds(vals, consts, scal)
            fv = _factor_values(vals, consts, scal)
            for key, poly in derived.items():
                want = _evaluate(poly, fv) * EPS
                assert abs(got[key] - want) <= 1e-13 * max(want, 1e-300), (vec, key, got[key], want)


# --------------------------------------------------------------------------- gap identities as data
# target: [(sign, scalar factors, operand, A applied)]; operands Dr, Ds, Dw, Dz (iteration i),
# Ds_prev, Dz_prev (iteration i-1) and the local errors d* of iteration i.
GAP_IDENTITIES = {
    "Dr_next": [(+1, (), "Dr", False), (-1, ("alpha",), "Ds", False), (-1, ("omega",), "Dw", False),
                (+1, ("omega", "alpha"), "Dz", False), (-1, (), "dx", True), (-1, (), "dr", False),
                (-1, ("omega",), "du", True), (-1, (), "dq", False), (+1, ("omega",), "dy", False)],   # Eq. (Dr)
    "Ds": [(+1, (), "Dw", False), (+1, ("beta",), "Ds_prev", False), (-1, ("beta", "omega_prev"), "Dz_prev", False),
           (+1, (), "dg", True), (-1, (), "ds", False)],                                               # Eq. (Ds)
    "Dw_next": [(+1, (), "Dw", False), (-1, ("alpha",), "Dz", False), (+1, (), "dk", True), (-1, (), "dw", False),
                (+1, (), "du", True), (-1, (), "dy", False)],                                         # Eq. (Dw)
    "Dz": [(+1, ("beta",), "Dz_prev", False), (+1, (), "dl", True), (-1, (), "dz", False)],            # Eq. (Dz)
}


def _probe_run(prob, K=25):
    if not diagnostics.extended_available():
        pytest.skip("numpy longdouble is not wider than double here")
    A = prob.A.to_scipy()
    M = make_precond(prob.precond, A, prob.degree, np.float64)
    probe = diagnostics.PipelinedProbe(A, prob.b, prob.precond, M.dinv, prob.degree, M, keep_vectors=True)
    krylov.pbicgstab(A, prob.b, precond=prob.precond, degree=prob.degree, tol=1e-300, maxit=K, observer=probe)
    return probe


@pytest.mark.parametrize("which", ["convdiff2d_24_jacobi", "convdiff3d_8_neumann2"])
def test_gap_identity_data_matches_measured_gaps(which):
    """The identity data, evaluated on the extended-precision gaps and local errors of a real
    run, predicts the gaps to within the extended precision: the gaps are about 1e-15, and
    the 64-bit longdouble leaves about 1e-4 of them (the bound is the 1e-2 of the oracle's own
    gap-recurrence pin); a wrong sign, scalar or operand in the data leaves O(1)."""
    prob = tp.problem_convdiff2d(24) if which.startswith("convdiff2d") else tp.problem_convdiff3d(8)
    probe = _probe_run(prob)
    A_ = probe.ops.A_
    zero = None
    for i, rec in enumerate(probe.records):
        gv, dv, sc = rec["gap_vec"], rec["delta_vec"], rec["scalars"]
        if zero is None:
            zero = gv["r"] * 0
        prev = probe.records[i - 1]["gap_vec"] if i > 0 else dict(s=zero, z=zero)
        ops = dict(Dr=gv["r"], Ds=gv["s"], Dw=gv["w"], Dz=gv["z"], Ds_prev=prev["s"], Dz_prev=prev["z"])
        ops.update({"d" + k: v for k, v in dv.items()})
        want = dict(Dr_next=rec["gap_next_vec"]["r"], Ds=gv["s"], Dw_next=rec["gap_next_vec"]["w"], Dz=gv["z"])
        for target, terms in GAP_IDENTITIES.items():
            pred = zero.copy()
            for sign, scal, operand, via_a in terms:
                f = np.longdouble(sign) * np.prod([np.longdouble(sc[s]) for s in scal], dtype=np.longdouble)
                val = A_(ops[operand]) if via_a else ops[operand]
                pred = pred + f * val
            err = np.sqrt(np.sum((want[target] - pred) ** 2)) / max(np.sqrt(np.sum(want[target] ** 2)), 1e-300)
            assert err <= 1e-2, (which, i, target, float(err))


def _triangle(target, F, d, sc, nA):
    """Triangle inequality of one identity: norms of gaps F, bounds d of the local errors."""
    total = 0.0
    for _, scal, operand, via_a in GAP_IDENTITIES[target]:
        f = math.prod(abs(sc[s]) for s in scal)
        total += f * (F[operand] if operand[0] == "D" else (nA if via_a else 1.0) * d[operand[1:]])
    return total


def test_gap_bound_follows_the_identities():
    """_GapBound.step (f^r, F^s, F^w, F^z) equals the triangle inequality of the identity data
    with the local-error bounds of delta_bounds, on synthetic norms and scalars."""
    rng = np.random.Generator(np.random.PCG64(13))
    A64 = 3.0 * tp.problem_convdiff2d(6).A.to_scipy()   # ||A|| bound 3, not 1
    M = make_precond("jacobi", A64, 0, np.float64)
    for trial in range(10):
        gb = krylov._GapBound(A64, M, np.ones(A64.shape[0]), EPS, False)
        c = gb.consts
        # vectors with prescribed norms (multiples of one unit vector: the norm is exact)
        e = np.zeros(A64.shape[0])
        e[0] = 1.0
        nv = {k: float(rng.uniform(0.1, 3.0)) for k in VEC_CUR}
        prev = {k: float(rng.uniform(0.1, 3.0)) for k in VEC_PREV}
        sc = dict(alpha=float(rng.uniform(-2, 2)), beta=float(rng.uniform(-2, 2)), omega=float(rng.uniform(-2, 2)),
                  omega_prev=float(rng.uniform(-2, 2)))
        # gaps on the scale real runs give them (a few eps times the vector norms), so that
        # every term of the recurrences is visible at the comparison's 1e-13
        F0 = {k: float(rng.uniform(1, 100)) * EPS for k in ("f", "Fs", "Fw", "Fz")}
        gb.f, gb.Fs, gb.Fw, gb.Fz = F0["f"], F0["Fs"], F0["Fw"], F0["Fz"]
        gb.first = False
        gb.prev = dict(prev)
        args = [nv[k] * e for k in ("x", "r", "k", "w", "g", "s", "l", "z", "q", "u", "y", "m", "t", "n", "v")]
        gb.step(sc["alpha"], sc["beta"], sc["omega"], sc["omega_prev"], *args)
        d = diagnostics.delta_bounds(nv, prev, sc["alpha"], sc["beta"], sc["omega"], sc["omega_prev"], c, EPS)
        nA = c["nA"]
        Fz = _triangle("Dz", dict(Dz_prev=F0["Fz"]), d, sc, nA)
        Fs = _triangle("Ds", dict(Dw=F0["Fw"], Ds_prev=F0["Fs"], Dz_prev=F0["Fz"]), d, sc, nA)
        fr = _triangle("Dr_next", dict(Dr=F0["f"], Ds=Fs, Dw=F0["Fw"], Dz=Fz), d, sc, nA)
        Fw = _triangle("Dw_next", dict(Dw=F0["Fw"], Dz=Fz), d, sc, nA)
        for name, got, want in (("Fz", gb.Fz, Fz), ("Fs", gb.Fs, Fs), ("f", gb.f, fr), ("Fw", gb.Fw, Fw)):
            assert abs(got - want) <= 1e-13 * want, (trial, name, got, want)


def test_gap_bound_initial_values_follow_the_model():
    """f^r_0 = ((mu sqrt(N) + 1)||A|| ||x_0|| + ||b||) eps is the composition of the model over
    r_0 = b - A x_0; F^s_0, F^w_0, F^z_0 (s_0 = fl(A g_0)-like explicit products, reading R3)
    are the SPMV rounding of g_0, k_0, l_0 -- the values _GapBound.start / reset use."""
    r0 = plus(leaf("b"), product("A", leaf("x")))[1]
    assert r0 == Counter({("b",): 1, ("nA", "x"): 1, ("msn", "nA", "x"): 1})
    A64 = 3.0 * tp.problem_convdiff2d(6).A.to_scipy()   # ||A|| bound 3, not 1
    M = make_precond("jacobi", A64, 0, np.float64)
    b = np.linspace(1.0, 2.0, A64.shape[0])
    gb = krylov._GapBound(A64, M, b, EPS, False)
    x = np.linspace(-1.0, 1.0, A64.shape[0])
    gb.start(x, 1.0)
    c = gb.consts
    fv = dict(b=float(np.linalg.norm(b)), x=float(np.linalg.norm(x)), nA=c["nA"], msn=c["mu"] * c["sqrtN"])
    assert abs(gb.f - _evaluate(r0, fv) * EPS) <= 1e-14 * gb.f
    k, g, l = (np.full(A64.shape[0], v) for v in (0.5, 0.7, 0.3))
    gb.reset(x, k, g, 2 * g, l, 3 * l)
    for attr, vec in (("Fw", k), ("Fs", g), ("Fz", l)):
        want = _evaluate(product("A", leaf("v"))[1], dict(v=float(np.linalg.norm(vec)), nA=c["nA"],
                                                          msn=c["mu"] * c["sqrtN"])) * EPS
        assert abs(getattr(gb, attr) - want) <= 1e-14 * want, attr


def test_bound_constants_closed_forms():
    """mu, mu~, sqrt(N) and the norm bounds on a hand-sized matrix: row 1 has 3 entries;
    column sums of |A| are 6, 9, 7 and row sums 5, 8, 9, so sqrt(||A||_1 ||A||_inf) = 9;
    Jacobi's ||M^{-1}|| bound is max |1/a_ii| = 1/4 with one entry per row; the degree-1
    Neumann polynomial D^{-1} + (I - D^{-1}A) D^{-1}, formed densely here, has A's
    tridiagonal pattern (3 entries in its middle row)."""
    import scipy.sparse as sp
    a = np.array([[4.0, -1.0, 0.0], [-2.0, 5.0, -1.0], [0.0, -3.0, 6.0]])
    A = sp.csr_matrix(a)
    c = diagnostics.bound_constants(A, make_precond("jacobi", A, 0, np.float64))
    assert c["mu"] == 3 and c["mut"] == 1 and abs(c["sqrtN"] - math.sqrt(3)) < 1e-15
    assert abs(c["nA"] - 9.0) < 1e-14 and abs(c["nM"] - 0.25) < 1e-15
    assert np.linalg.svd(a, compute_uv=False)[0] <= c["nA"]
    D = np.diag(1.0 / np.diag(a))
    P = D + (np.eye(3) - D @ a) @ D
    cn = diagnostics.bound_constants(A, make_precond("neumann", A, 1, np.float64))
    assert cn["mut"] == max(int(np.count_nonzero(np.abs(row) > 0)) for row in P) == 3
    ap = np.abs(P)
    assert abs(cn["nM"] - math.sqrt(ap.sum(axis=0).max() * ap.sum(axis=1).max())) < 1e-14
