"""The C ABI library loads and exports every symbol include/pbicgstab.h declares, and the
ctypes structure layouts match the C compiler's (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pbicgstab.h")


def _declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:pbcg_status|const char\*)\s+(pbicgstab_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_01948_gb300._build import build
    build()
    from paper_1809_01948_gb300 import _capi
    return _capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1809_01948_gb300 import _capi
    assert set(_declared_functions()) <= set(_capi.PROTOTYPES)


def test_struct_layouts_match_c():
    from paper_1809_01948_gb300 import _capi
    structs = {"pbcg_matrix": _capi.Matrix, "pbcg_precond": _capi.Precond,
               "pbcg_options": _capi.Options, "pbcg_result": _capi.Result,
               "pbcg_batch": _capi.Batch, "pbcg_batch_result": _capi.BatchResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pbicgstab.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = dict(l.split() for l in subprocess.check_output([exe]).decode().splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_default_options_and_argument_errors(lib):
    from paper_1809_01948_gb300 import _capi
    o = _capi.Options()
    assert lib.pbicgstab_default_options(C.byref(o)) == 0
    assert o.tol == 1e-10 and o.max_it == 10000 and o.timeout_ms == 2000.0
    # NULL arguments are rejected on the host before any CUDA call
    assert lib.pbicgstab_create(None, None, None, None, None) == _capi.PBCG_INVALID_ARG
    assert b"NULL" in lib.pbicgstab_last_error()
    assert lib.pbicgstab_destroy(None) == 0
    assert lib.pbicgstab_solve(None, None, None, None) == _capi.PBCG_INVALID_ARG


def test_batched_neumann_degree_checked_on_the_host(lib):
    """A Neumann batch needs a degree in [1, 8]; the check runs before any CUDA call."""
    import numpy as np
    from paper_1809_01948_gb300 import _capi
    off = np.array([0, 4], dtype=np.int64)
    dummy = np.zeros(16, dtype=np.float64)
    bt = _capi.Batch()
    bt.n_sys, bt.val_dtype = 1, _capi.F64
    bt.row_off = off.ctypes.data_as(C.c_void_p)
    bt.nnz_off = off.ctypes.data_as(C.c_void_p)
    bt.row_ptr = bt.col = bt.val = dummy.ctypes.data_as(C.c_void_p)
    o = _capi.Options()
    assert lib.pbicgstab_default_options(C.byref(o)) == 0
    ctx = C.c_void_p()
    for degree in (0, 9):
        bt.precond, bt.degree = 2, degree
        assert lib.pbicgstab_batch_create(C.byref(ctx), C.byref(bt), C.byref(o), None) == _capi.PBCG_INVALID_ARG
        assert b"degree" in lib.pbicgstab_last_error()
    bt.precond = 3   # no such preconditioner
    assert lib.pbicgstab_batch_create(C.byref(ctx), C.byref(bt), C.byref(o), None) == _capi.PBCG_INVALID_ARG
