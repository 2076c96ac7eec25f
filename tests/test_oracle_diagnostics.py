"""Oracle pins from the rounding-error analysis: Eq. (errbounds1)-(errbounds4), the gap
recurrences Eq. (Dr), (Ds), (Dw), (Dz), the classic superposition Eq. (classic_nomatrix),
and the gap bound f^r of Eq. (DDr_bound)."""
import numpy as np
import pytest

import oracle
from oracle import diagnostics
import testproblems as tp

pytestmark = pytest.mark.skipif(not diagnostics.extended_available(),
                                reason="needs numpy longdouble wider than double")

CASES = [("poisson", "none", 0), ("upwind", "jacobi", 0), ("upwind3d", "neumann", 2)]


def _problem(which):
    if which == "poisson":
        return tp.problem_poisson2d(40)
    if which == "upwind":
        return tp.problem_convdiff2d(40)
    return tp.problem_convdiff3d(10)


def _probe_run(which, prec, deg, maxit=40, **kw):
    p = _problem(which)
    A = p.A.to_scipy()
    M = oracle.make_precond(prec, A, deg)
    probe = diagnostics.PipelinedProbe(A, p.b, prec, M.dinv, deg, M)
    res = oracle.pbicgstab(A, p.b, precond=prec, degree=deg, tol=1e-30, maxit=maxit, observer=probe,
                           track_bound=True, **kw)
    return p, probe, res


@pytest.mark.parametrize("which,prec,deg", CASES)
def test_local_errors_within_paper_bounds(which, prec, deg):
    """Every measured ||delta_i|| of Eq. (auxrec) is below its bound in Eq. (errbounds1)-(4).
    A wrong index, sign or operand in any recurrence makes its delta O(1) and fails this."""
    _, probe, _ = _probe_run(which, prec, deg)
    assert len(probe.records) == 40
    for rec in probe.records:
        for key, val in rec["delta"].items():
            assert val <= rec["bound"][key], (rec["i"], key, val, rec["bound"][key])


@pytest.mark.parametrize("which,prec,deg", CASES)
def test_gap_recurrences_hold(which, prec, deg):
    """Eqs. (Dr), (Ds), (Dw), (Dz): the measured gaps obey the coupled recurrences to the
    precision of the extended-precision evaluation."""
    _, probe, _ = _probe_run(which, prec, deg)
    for rec in probe.records:
        for key in "rswz":
            assert rec["ident"][key] < 1e-2, (rec["i"], key, rec["ident"][key])


@pytest.mark.parametrize("which,prec,deg", CASES)
def test_gap_below_bound_fr(which, prec, deg):
    """||Delta^r_i|| <= f^r_i (Eq. DDr_bound with the bounds of Eq. errbounds)."""
    _, probe, res = _probe_run(which, prec, deg, maxit=60)
    for rec, fr in zip(probe.records, res.fr):
        assert rec["gap_r_next"] <= fr


def test_gap_bound_resets_at_replacement():
    """After Eq. (rr) the gap is the round-off of b - A x, bounded by
    ((mu sqrt(N) + 1) ||A|| ||x|| + ||b||) eps."""
    p, probe, res = _probe_run("upwind", "jacobi", 0, maxit=60, rr_period=20)
    assert len(probe.after_replace) == 2
    A = p.A.to_scipy()
    mu = np.max(np.diff(A.indptr))
    nA = diagnostics.bound_constants(A, oracle.make_precond("jacobi", A))["nA"]
    for ev in probe.after_replace:
        bound = ((mu * np.sqrt(A.shape[0]) + 1) * nA * ev["x"] + np.linalg.norm(p.b)) * 2.0 ** -52
        assert ev["gap_r"] <= bound
    for rec, fr in zip(probe.records, res.fr):
        assert rec["gap_r_next"] <= fr


@pytest.mark.parametrize("prec", ["none", "jacobi"])
def test_classic_gap_is_superposition(prec):
    """Eq. (classic_nomatrix): Delta^r_i = Delta^r_0 - sum_j (A dx_j + dr_j + dq_j)."""
    p = tp.problem_convdiff2d(30)
    A = p.A.to_scipy()
    M = oracle.make_precond(prec, A)
    probe = diagnostics.ClassicProbe(A, p.b, None, prec, M.dinv, 0)
    oracle.bicgstab(A, p.b, precond=prec, tol=1e-30, maxit=40, observer=probe)
    assert len(probe.records) == 40
    for rec in probe.records:
        assert rec["ident"] < 1e-2
