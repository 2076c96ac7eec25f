"""Planted mistakes in the error-propagation oracle (Section 2.4): each mutant is the source
of ``oracle/propagation.py`` with one plausible slip in an entry of the gap operator of
Eq. (system), the local terms of Eq. (local), the matrices of Eq. (all_matrices) or the
products of Eq. (all_error_matrices).  Each must fail at least one pin of
``test_oracle_propagation.py`` (the gaps measured in extended precision on real runs, the
hand-derived element sums and the constant-scalar closed forms), run here against the
mutant.  CPU only."""
import functools
import sys
import types

import numpy as np
import pytest

import test_oracle_propagation as T
from oracle import propagation

SOURCE = open(propagation.__file__).read()

MUTANTS = [
    ("O: sign", "Om[j, j] = -omega[j - 1]", "Om[j, j] = omega[j - 1]"),
    ("O: index", "Om[j, j] = -omega[j - 1]", "Om[j, j] = -omega[min(j, len(omega) - 1)]"),
    ("P: beta product start", "Pm[k, j] = -omega[k] * bprod(k, j)", "Pm[k, j] = -omega[k] * bprod(k + 1, j)"),
    ("D: sign", "Dm[k, j] = omega[k] * alpha[k]", "Dm[k, j] = -omega[k] * alpha[k]"),
    ("C: index", "Cm[k, j] = -omega[k]", "Cm[k, j] = -omega[max(k - 1, 0)]"),
    ("E: first row kept", "if k >= 1:\n                Em", "if k >= 0:\n                Em"),
    ("A: index", "Am[k, j] = -alpha[k]", "Am[k, j] = -alpha[max(k - 1, 0)]"),
    ("beta product: last factor dropped", "return float(np.prod(beta[k + 1:j + 1]))",
     "return float(np.prod(beta[k + 1:j]))"),
    ("B: diagonal dropped", "Bm[k, j] = bprod(k, j)", "Bm[k, j] = bprod(k, j) if k < j else 0.0"),
    ("G(0,3): omega sum sign", "a * b * (o + op)]", "a * b * (o - op)]"),
    ("G(1,3): omega_i instead of omega_i-1", "[0.0, b, 1.0, -b * op]", "[0.0, b, 1.0, -b * o]"),
    ("G(0,2): sign", "-(a + o)", "-(a - o)"),
    ("eps_r: sign of omega y", '+ o * d["y"] - d["r"]', '- o * d["y"] - d["r"]'),
    ("eps_w: sign of A u", '- d["y"] - d["w"] + A_(d["u"])', '- d["y"] - d["w"] - A_(d["u"])'),
    ("product BA -> AB", '"BA": B @ A,', '"BA": A @ B,'),
    ("product BD -> BC", '"BD": B @ D,', '"BD": B @ C,'),
]


def _load(src):
    mod = types.ModuleType("oracle._propagation_mutant")
    mod.__package__ = "oracle"
    mod.__file__ = propagation.__file__
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src, "<propagation mutant>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


_measured_run = T._run


@functools.lru_cache(maxsize=None)
def _cached_run(which, prec, K):
    # the measured runs use the Algorithm 2 oracle and the probes only, not this module
    return _measured_run(which, prec, K)


def _pins(monkeypatch, mod):
    """Names of the pins that fail with `mod` in place of oracle.propagation."""
    monkeypatch.setattr(T, "pg", mod)
    monkeypatch.setattr(T, "_run", _cached_run)
    failed = []
    checks = [("products", T.test_products_against_elementwise_sums, ()),
              ("closed forms", T.test_column_norms_constant_scalars_closed_forms, ())]
    if T.diagnostics.extended_available():
        for case in T.CASES:
            checks.append(("gap operator %s" % case[0], T.test_gap_operator_reproduces_measured_gaps, case))
            checks.append(("matrix expressions %s" % case[0], T.test_matrix_expressions_reproduce_measured_gaps, case))
    for name, fn, args in checks:
        try:
            with np.errstate(all="ignore"):
                fn(*args)
        except (AssertionError, IndexError, ValueError, FloatingPointError):
            failed.append(name)
    return failed


def test_unmutated_source_passes(monkeypatch):
    assert _pins(monkeypatch, _load(SOURCE)) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(monkeypatch, name, old, new):
    assert SOURCE.count(old) == 1, "mutation site not unique or missing: %r" % old
    assert _pins(monkeypatch, _load(SOURCE.replace(old, new))), name
