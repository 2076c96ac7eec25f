"""Host-side argument validation of the C ABI: every case below is rejected with
PBCG_INVALID_ARG before any CUDA call (no GPU needed), covering empty and oversized
systems, malformed matrix descriptions and inconsistent options."""
import ctypes as C

import pytest

from paper_1809_01948_gb300 import _capi as capi

INVALID = capi.PBCG_INVALID_ARG


@pytest.fixture(scope="module")
def lib():
    try:
        import paper_1809_01948_gb300._build as b
        b.build()
        return capi.load()
    except Exception as e:  # the toolchain is part of the image; a failure here is a real error
        pytest.fail("library did not build: %s" % e)


def _csr(n=10, nnz=10):
    m = capi.Matrix()
    m.format, m.val_dtype, m.n, m.nnz = capi.FMT_CSR, capi.F64, n, nnz
    # dummy device addresses: validation must reject before dereferencing any of them
    m.row_ptr, m.col, m.val = C.c_void_p(0x1000), C.c_void_p(0x2000), C.c_void_p(0x3000)
    return m


def _dia(offs, n=100):
    m = capi.Matrix()
    arr = (C.c_int32 * len(offs))(*offs)
    m.format, m.val_dtype, m.n, m.ndiag = capi.FMT_DIA, capi.F64, n, len(offs)
    m.val = C.c_void_p(0x3000)
    m.offsets = C.cast(arr, C.c_void_p)
    return m, arr


def _opts(lib, **kw):
    o = capi.Options()
    assert lib.pbicgstab_default_options(C.byref(o)) == 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _create(lib, m, prec=capi.PREC_JACOBI, degree=0, **kw):
    ctx = C.c_void_p()
    p = capi.Precond(prec, degree)
    st = lib.pbicgstab_create(C.byref(ctx), C.byref(m), C.byref(p), C.byref(_opts(lib, **kw)), None)
    return st, lib.pbicgstab_last_error().decode()


@pytest.mark.parametrize("n", [0, -5, 2 ** 30 + 1, 2 ** 31 - 1, 2 ** 40])
def test_system_size_outside_int32_rows(lib, n):
    st, msg = _create(lib, _csr(n=n))
    assert st == INVALID and "n must be" in msg


def test_malformed_matrix_descriptions(lib):
    m = _csr()
    m.format = 7
    assert _create(lib, m)[0] == INVALID
    m = _csr()
    m.val_dtype = 3
    assert _create(lib, m)[0] == INVALID
    m = _csr()
    m.val = None
    assert _create(lib, m)[0] == INVALID
    m = _csr(nnz=-1)
    assert _create(lib, m)[0] == INVALID
    m = _csr()
    m.col = None
    assert _create(lib, m)[0] == INVALID
    for offs in ([-1, 0, 0], [1, 2], [-100, 0], [0] * 17, []):   # not increasing, no 0, out of range, too many
        m, keep = _dia(offs)
        st, msg = _create(lib, m)
        assert st == INVALID, (offs, msg)


@pytest.mark.parametrize("prec,degree", [(7, 0), (capi.PREC_NEUMANN, 0), (capi.PREC_NEUMANN, 9)])
def test_bad_preconditioner(lib, prec, degree):
    assert _create(lib, _csr(), prec=prec, degree=degree)[0] == INVALID


@pytest.mark.parametrize("kw", [dict(precision=5), dict(max_it=-1), dict(tol=-1.0), dict(tol=float("inf")),
                                dict(rr_period=-1), dict(rr_auto=2), dict(rr_theta=1.0), dict(rr_tau=-1.0),
                                dict(block_threads=33), dict(block_threads=2048), dict(grid_blocks=-1),
                                dict(max_restarts=1001), dict(method=2), dict(operator_storage=7),
                                dict(method=capi.CLASSIC, precision=capi.MIXED),
                                dict(method=capi.CLASSIC, rr_period=10), dict(record_iterates=3)])
def test_inconsistent_options(lib, kw):
    assert _create(lib, _csr(), **kw)[0] == INVALID


def test_method_and_policy_need_their_preconditioners(lib):
    assert _create(lib, _csr(), prec=capi.PREC_NEUMANN, degree=2, method=capi.CLASSIC)[0] == INVALID
    assert _create(lib, _csr(), prec=capi.PREC_NEUMANN, degree=2, rr_auto=1)[0] == INVALID


@pytest.mark.parametrize("kw", [dict(batch_build=3), dict(batch_build=-1), dict(batch_build=2),
                                dict(batch_build=2, precision=capi.MIXED, cluster_blocks=1),
                                dict(batch_build=2, precision=capi.MIXED, block_threads=1024)])
def test_batched_build_option(lib, kw):
    """batch_build: 0, 1 or 2 only; the streaming build needs mixed precision, clusters and
    at most 512 threads per block (all checked before any CUDA call)."""
    row_off = (C.c_int64 * 2)(0, 10)
    nnz_off = (C.c_int64 * 2)(0, 10)
    bt = capi.Batch()
    bt.n_sys, bt.val_dtype, bt.precond = 1, capi.F64, capi.PREC_JACOBI
    bt.row_off, bt.nnz_off = C.cast(row_off, C.c_void_p), C.cast(nnz_off, C.c_void_p)
    bt.row_ptr, bt.col, bt.val = C.c_void_p(0x1000), C.c_void_p(0x2000), C.c_void_p(0x3000)
    ctx = C.c_void_p()
    st = lib.pbicgstab_batch_create(C.byref(ctx), C.byref(bt), C.byref(_opts(lib, **kw)), None)
    assert st == INVALID and "batch_build" in lib.pbicgstab_last_error().decode() and not ctx.value


def test_batched_and_multi_argument_errors(lib):
    ctx = C.c_void_p()
    bt = capi.Batch()
    bt.n_sys = 0
    o = _opts(lib)
    assert lib.pbicgstab_batch_create(C.byref(ctx), C.byref(bt), C.byref(o), None) == INVALID
    assert lib.pbicgstab_batch_create(None, None, None, None) == INVALID
    assert lib.pbicgstab_solve_multi(None, 2, None, None, None) == INVALID
    assert lib.pbicgstab_create_transpose(None, None) == INVALID
    assert lib.pbicgstab_propagation_norms(None, 8, 3, None, None) == INVALID
    st = C.c_int32()
    assert lib.pbicgstab_operator_storage(None, C.byref(st)) == INVALID
