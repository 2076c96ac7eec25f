"""Planted mistakes in the rounding-error diagnostics (``oracle/diagnostics.py``): each
mutant is that module's source with one slip in a local-error definition of Eq. (auxrec),
a gap definition, a gap recurrence of Eqs. (Dr), (Ds), (Dw), (Dz), the extended-precision
preconditioner, or a leading term of an error bound of Eq. (errbounds1)-(4).  Each must
fail a pin of ``test_oracle_diagnostics.py`` run against the mutant.  CPU only.

The bound formulas are upper bounds and are pinned only by inequalities (measured
||delta|| <= bound, ||Delta^r|| <= f^r); dropping a term that does not dominate a bound
(most of them: the bounds sit about 5x above the measured errors) is not detected, so only
the dominating terms appear below."""
import sys
import types

import numpy as np
import pytest

import test_oracle_diagnostics as T
from oracle import diagnostics

pytestmark = pytest.mark.skipif(not diagnostics.extended_available(),
                                reason="needs numpy longdouble wider than double")

SOURCE = open(diagnostics.__file__).read()

MUTANTS = [
    ("delta q: sign", 'delta["q"] = L("q") - (L("r") - al * L("s"))', 'delta["q"] = L("q") - (L("r") + al * L("s"))'),
    ("delta k: n -> m", 'delta["k"] = L("k_new") - (L("u") - om * (mex - al * nex))',
     'delta["k"] = L("k_new") - (L("u") - om * (mex - al * mex))'),
    ("delta l: n_{i-1} -> n_i", 'delta["l"] = L("l") - (mex + be * (L("l_prev") - op * nprev_ex))',
     'delta["l"] = L("l") - (mex + be * (L("l_prev") - op * nex))'),
    ("delta x: u -> g", 'delta["x"] = L("x_new") - (L("x") + al * L("g") + om * L("u"))',
     'delta["x"] = L("x_new") - (L("x") + al * L("g") + om * L("g"))'),
    ("delta w: v -> t", 'delta["w"] = L("w_new") - (L("y") - om * (tex - al * vex))',
     'delta["w"] = L("w_new") - (L("y") - om * (tex - al * tex))'),
    ("delta z: beta -> omega", 'delta["z"] = L("z") - (tex + be * (L("z_prev") - op * vprev_ex))',
     'delta["z"] = L("z") - (tex + om * (L("z_prev") - op * vprev_ex))'),
    ("Eq. Dr: sign of omega Dw", "- om * Dw + om * al * Dz", "+ om * Dw + om * al * Dz"),
    ("Eq. Dr: A delta_x dropped", '- A_(delta["x"]) - delta["r"]', '- delta["r"]'),
    ("Eq. Dw: sign of A delta_u", '+ A_(delta["u"]) - delta["y"]   # Eq. (Dw)', '- A_(delta["u"]) - delta["y"]   # Eq. (Dw)'),
    ("Eq. Ds: omega_{i-1} -> omega_i", "be * self.Ds_prev - be * op * self.Dz_prev", "be * self.Ds_prev - be * om * self.Dz_prev"),
    ("Eq. Dz: beta dropped", 'pred_z = be * self.Dz_prev + A_(delta["l"]) - delta["z"]',
     'pred_z = self.Dz_prev + A_(delta["l"]) - delta["z"]'),
    ("gap s: A g -> A k", 'Ds = A_(d["g"]) - L("s")', 'Ds = A_(d["k"]) - L("s")'),
    ("gap w_{i+1}: k_{i+1} -> k_i", 'Dw_next = A_(d["k_new"]) - L("w_new")', 'Dw_next = A_(d["k"]) - L("w_new")'),
    ("exact Neumann sweep: sign", "y = y + self.dinv * (v - self.A @ y)", "y = y + self.dinv * (v + self.A @ y)"),
    ("bound x: ||x|| term dropped", 'd["x"] = (2 * cur["x"] + 3 * a * cur["g"] + 2 * o * cur["u"]) * eps',
     'd["x"] = (3 * a * cur["g"] + 2 * o * cur["u"]) * eps'),
    ("bound q: ||r|| term dropped", 'd["q"] = (cur["r"] + 2 * a * cur["s"]) * eps', 'd["q"] = (2 * a * cur["s"]) * eps'),
    ("bound u: ||k|| term dropped", 'd["u"] = (cur["k"] + 2 * a * cur["l"]) * eps', 'd["u"] = (2 * a * cur["l"]) * eps'),
]

CLASSIC_MUTANTS = [
    ("classic delta x: omega u dropped", "dx = L(\"x_new\") - (L(\"x\") + al * gex + om * uex)",
     "dx = L(\"x_new\") - (L(\"x\") + al * gex)"),
    ("classic delta r: sign", "dr = L(\"r_new\") - (L(\"q\") - om * A_(uex))", "dr = L(\"r_new\") - (L(\"q\") + om * A_(uex))"),
    ("classic delta q: M p -> p", "dq = L(\"q\") - (L(\"r\") - al * A_(gex))", "dq = L(\"q\") - (L(\"r\") - al * A_(L(\"p\")))"),
    ("classic superposition: A delta_x dropped", "self.sum = self.sum - (A_(dx) + dr + dq)", "self.sum = self.sum - (dr + dq)"),
]

PINS = [("local errors within bounds", T.test_local_errors_within_paper_bounds),
        ("gap recurrences", T.test_gap_recurrences_hold)]


def _load(src):
    mod = types.ModuleType("oracle._diagnostics_mutant")
    mod.__package__ = "oracle"
    mod.__file__ = diagnostics.__file__
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src, "<diagnostics mutant>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _failing_pins(monkeypatch, mod):
    monkeypatch.setattr(T, "diagnostics", mod)
    failed = []
    for name, fn in PINS:
        for case in T.CASES:
            try:
                with np.errstate(all="ignore"):
                    fn(*case)
            except (AssertionError, FloatingPointError, ValueError):
                failed.append((name, case[0]))
    return failed


def test_unmutated_source_passes(monkeypatch):
    assert _failing_pins(monkeypatch, _load(SOURCE)) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    assert _failing_pins(monkeypatch, _load(SOURCE.replace(old, new))), name


def _classic_pin_fails(monkeypatch, mod):
    monkeypatch.setattr(T, "diagnostics", mod)
    failed = []
    for prec in ("none", "jacobi"):
        try:
            with np.errstate(all="ignore"):
                T.test_classic_gap_is_superposition(prec)
        except (AssertionError, FloatingPointError, ValueError):
            failed.append(prec)
    return failed


def test_unmutated_classic_probe_passes(monkeypatch):
    assert _classic_pin_fails(monkeypatch, _load(SOURCE)) == []


@pytest.mark.parametrize("name,old,new", CLASSIC_MUTANTS, ids=[m[0] for m in CLASSIC_MUTANTS])
def test_classic_probe_mutant_fails_the_superposition_pin(monkeypatch, name, old, new):
    assert SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    assert _classic_pin_fails(monkeypatch, _load(SOURCE.replace(old, new))), name
