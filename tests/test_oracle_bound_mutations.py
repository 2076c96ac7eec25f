"""Planted slips in the rounding-error bound formulas: one in each local-error bound of
Eqs. (errbounds1)-(errbounds4) (``diagnostics.delta_bounds``) and in each recurrence and
initial value of the run-time gap bound f^r (``krylov._GapBound``, Eq. (DDr_bound) with
reading R14).  None of them dominates its bound, so the inequality pins cannot see them;
each must fail a pin of ``test_oracle_bound_derivation.py`` (the bounds derived from the
paper's floating-point model and from the gap identities) run against the mutant.  CPU only."""
import sys
import types

import numpy as np
import pytest

import test_oracle_bound_derivation as T
from oracle import diagnostics, krylov

DIAG_SOURCE = open(diagnostics.__file__).read()
KRYLOV_SOURCE = open(krylov.__file__).read()

DIAG_MUTANTS = [
    ("g: 3 beta g_prev -> 2", '3 * b * prev["g"] + 4 * bo * prev["l"]', '2 * b * prev["g"] + 4 * bo * prev["l"]'),
    ("x: 2 omega u -> 1", '3 * a * cur["g"] + 2 * o * cur["u"]', '3 * a * cur["g"] + o * cur["u"]'),
    ("s: 4 beta omega z_prev -> 3", '3 * b * prev["s"] + 4 * bo * prev["z"]', '3 * b * prev["s"] + 3 * bo * prev["z"]'),
    ("r: omega y -> alpha y", '(cur["q"] + 2 * o * cur["y"])', '(cur["q"] + 2 * a * cur["y"])'),
    ("l: PREC rounding of n_prev dropped", '+ tmsn * nM * bo * prev["z"]) * eps\n', ') * eps\n'),
    ("z: n_prev -> v_prev in the SPMV term", 'msn * nA * bo * prev["n"]', 'msn * nA * bo * prev["v"]'),
    ("k: n -> m", '4 * oa * cur["n"]\n', '4 * oa * cur["m"]\n'),
    ("w: ||M^-1|| dropped", 'tmsn * nA * nM * o * cur["w"]', 'tmsn * nA * o * cur["w"]'),
    ("q: s -> z", '(cur["r"] + 2 * a * cur["s"])', '(cur["r"] + 2 * a * cur["z"])'),
    ("u: 2 alpha l -> 3", '(cur["k"] + 2 * a * cur["l"])', '(cur["k"] + 3 * a * cur["l"])'),
    ("y: alpha z -> omega z", '(cur["w"] + 2 * a * cur["z"])', '(cur["w"] + 2 * o * cur["z"])'),
]

KRYLOV_MUTANTS = [
    ("F^z: ||A|| on d^l dropped", 'Fz = abs(beta) * self.Fz + nA * db["l"] + db["z"]', 'Fz = abs(beta) * self.Fz + db["l"] + db["z"]'),
    ("F^s: omega_{i-1} -> omega_i", 'abs(beta * omega_prev) * self.Fz', 'abs(beta * omega) * self.Fz'),
    ("f^r: |omega| on A d^u dropped", '+ abs(omega) * nA * db["u"]', '+ nA * db["u"]'),
    ("F^w: ||A|| on d^u dropped", 'nA * (db["k"] + db["u"])', 'nA * db["k"] + db["u"]'),
    ("f^r_0: the +1 of (mu sqrt(N) + 1) dropped", '(c["mu"] * c["sqrtN"] + 1) * c["nA"]', 'c["mu"] * c["sqrtN"] * c["nA"]'),
    ("reset F^s: g -> k", 'self.Fs = msn * nA * nrm(g) * self.eps', 'self.Fs = msn * nA * nrm(k) * self.eps'),
]

PINS = [T.test_delta_bounds_equal_the_composed_bounds, T.test_delta_bounds_term_by_term,
        T.test_gap_bound_follows_the_identities, T.test_gap_bound_initial_values_follow_the_model]


def _load(src, name, like):
    mod = types.ModuleType("oracle._%s_mutant" % name)
    mod.__package__ = "oracle"
    mod.__file__ = like.__file__
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src, "<%s mutant>" % name, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _failing(monkeypatch, diag=None, kry=None):
    if diag is not None:
        monkeypatch.setattr(T, "diagnostics", diag)
    if kry is not None:
        monkeypatch.setattr(T, "krylov", kry)
    failed = []
    for fn in PINS:
        try:
            with np.errstate(all="ignore"):
                fn()
        except AssertionError:
            failed.append(fn.__name__)
    return failed


def test_unmutated_sources_pass(monkeypatch):
    assert _failing(monkeypatch, _load(DIAG_SOURCE, "diagnostics", diagnostics),
                    _load(KRYLOV_SOURCE, "krylov", krylov)) == []


@pytest.mark.parametrize("name,old,new", DIAG_MUTANTS, ids=[m[0] for m in DIAG_MUTANTS])
def test_bound_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert DIAG_SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    assert _failing(monkeypatch, diag=_load(DIAG_SOURCE.replace(old, new), "diagnostics", diagnostics)), name


@pytest.mark.parametrize("name,old,new", KRYLOV_MUTANTS, ids=[m[0] for m in KRYLOV_MUTANTS])
def test_gap_bound_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert KRYLOV_SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    assert _failing(monkeypatch, kry=_load(KRYLOV_SOURCE.replace(old, new), "krylov", krylov)), name
