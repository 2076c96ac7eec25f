"""pbicgstab_solve_noalloc: the allocation-free entry point for callers that must not
allocate GPU memory (their own allocator owns the device memory, or their loop cannot
take the implicit synchronisation of cudaMalloc/cudaFree).  Its scratch lives in a fixed
device array inside the library.  This file is collected last on purpose.

Each case calls the entry point twice in a row through the C ABI (the second call sees
the scratch left by the first) and compares it with the context-based entry point
(pbicgstab_create + pbicgstab_solve) on the same inputs."""
import ctypes as C

import numpy as np
import pytest

import testproblems as tp

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1809_01948_gb300._build as b
    b.build()
    import paper_1809_01948_gb300 as pb
    from paper_1809_01948_gb300 import _capi
    return torch, pb, _capi, _capi.load()


def _matrix(torch, capi, prob, fmt, keep):
    dev = torch.device("cuda:0")
    m = capi.Matrix()
    m.n = prob.A.n
    m.val_dtype = capi.F64
    if fmt == "dia":
        off, data = tp.csr_to_dia(prob.A)
        d = torch.from_numpy(data).to(dev).contiguous()
        offs = (C.c_int32 * len(off))(*[int(o) for o in off])
        keep += [d, offs]
        m.format, m.val, m.ndiag, m.offsets = capi.FMT_DIA, d.data_ptr(), len(off), C.cast(offs, C.c_void_p)
    else:
        rp = torch.from_numpy(prob.A.row_ptr).to(dev)
        col = torch.from_numpy(prob.A.col).to(dev)
        val = torch.from_numpy(prob.A.val).to(dev)
        keep += [rp, col, val]
        m.format, m.nnz = capi.FMT_CSR, prob.A.nnz
        m.row_ptr, m.col, m.val = rp.data_ptr(), col.data_ptr(), val.data_ptr()
    return m


CASES = [("convdiff2d_128_dia_jacobi_rr", lambda: tp.problem_convdiff2d(128), "dia", "jacobi", dict(rr_period=100)),
         ("poisson2d_100_csr_none", lambda: tp.problem_poisson2d(100), "csr", "none", dict()),
         ("convdiff2d_90_csr_jacobi_ragged", lambda: tp.problem_convdiff2d(90), "csr", "jacobi", dict(rr_period=50))]


@pytest.mark.parametrize("threads", [512, 0], ids=["fixed_512_threads", "default_shape"])
@pytest.mark.parametrize("name,maker,fmt,prec,kw", CASES)
def test_noalloc_matches_context_solver_twice(name, maker, fmt, prec, kw, threads):
    """threads = 0 leaves the launch shape to each entry point: both use the same default
    rule for a matrix kept as given (this entry point never uses the stencil storage), so
    they sum the dot products in the same order."""
    torch, pb, capi, lib = _setup()
    dev = torch.device("cuda:0")
    prob = maker()
    tol = 1e-10
    # reference: the context-based entry point
    ref = pb.Solver(prob.A.n, **(dict(offsets=tp.csr_to_dia(prob.A)[0].tolist(),
                                      dia=torch.from_numpy(tp.csr_to_dia(prob.A)[1]).to(dev)) if fmt == "dia" else
                                 dict(row_ptr=torch.from_numpy(prob.A.row_ptr).to(dev),
                                      col=torch.from_numpy(prob.A.col).to(dev),
                                      val=torch.from_numpy(prob.A.val).to(dev))),
                    precond=prec, precision="fp64", tol=tol, max_it=5000, block_threads=threads,
                    operator_storage="general", **kw)
    b = torch.from_numpy(prob.b).to(dev)
    x_ref, r_ref = ref.solve(b)
    x_ref = x_ref.cpu().numpy()
    keep = []
    m = _matrix(torch, capi, prob, fmt, keep)
    p = capi.Precond(capi.PREC_JACOBI if prec == "jacobi" else capi.PREC_NONE, 0)
    opt = capi.Options()
    lib.pbicgstab_default_options(C.byref(opt))
    opt.tol, opt.max_it = tol, 5000
    opt.block_threads = threads   # the same launch shape as the context above (same reduction order)
    opt.rr_period = kw.get("rr_period", 0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = torch.zeros(prob.A.n, dtype=torch.float64, device=dev)
        res = capi.Result()
        st = lib.pbicgstab_solve_noalloc(C.byref(m), C.byref(p), C.byref(opt), C.c_void_p(b.data_ptr()),
                                         C.c_void_p(x.data_ptr()), C.byref(res), stream)
        assert st == r_ref.status == 0, (call, st, capi.last_error())
        xn = x.cpu().numpy()
        # same kernel and launch rule: the tests' FP64 tolerance (1e-10 relative) holds
        assert np.linalg.norm(xn - x_ref) <= 1e-10 * np.linalg.norm(x_ref), call
        assert res.iterations == r_ref.iterations and res.n_replacements == r_ref.n_replacements
        true = np.linalg.norm(prob.b - prob.A.to_scipy() @ xn) / np.linalg.norm(prob.b)
        assert true <= tol and abs(true - res.rel_res_true) <= 1e-3 * true + 1e-18
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch, pb, capi, lib = _setup()
    dev = torch.device("cuda:0")
    n = capi.NOALLOC_MAX_N + 1
    A = tp.stencil_2d(n, 1, dict(centre=4.0, west=-1.0, east=-1.0, south=0.0, north=0.0))
    prob = tp.Problem("big", A, np.ones(n), np.zeros(n), None, precond="jacobi", fmt="csr")
    keep = []
    m = _matrix(torch, capi, prob, "csr", keep)
    p = capi.Precond(capi.PREC_JACOBI, 0)
    opt = capi.Options()
    lib.pbicgstab_default_options(C.byref(opt))
    b = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    res = capi.Result()
    st = lib.pbicgstab_solve_noalloc(C.byref(m), C.byref(p), C.byref(opt), C.c_void_p(b.data_ptr()),
                                     C.c_void_p(x.data_ptr()), C.byref(res), None)
    assert st == capi.PBCG_INVALID_ARG
    assert "32768" in capi.last_error() and "static scratch limit" in capi.last_error()
    opt.precision = capi.MIXED
    m.n = 100
    st = lib.pbicgstab_solve_noalloc(C.byref(m), C.byref(p), C.byref(opt), C.c_void_p(b.data_ptr()),
                                     C.c_void_p(x.data_ptr()), C.byref(res), None)
    assert st == capi.PBCG_INVALID_ARG and "FP64" in capi.last_error()
