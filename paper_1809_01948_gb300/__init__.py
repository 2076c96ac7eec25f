"""GB300 (sm_103a) p-BiCGStab: Python binding of libpbicgstab (include/pbicgstab.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  If the library is not
built, importing works but every call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import torch

from . import _capi as capi
from ._capi import Result, STATUS_NAMES  # noqa: F401

__all__ = ["Solver", "BatchSolver", "PBCGError", "build", "STATUS_NAMES", "test_barrier_timeout",
           "SparseSolve", "sparse_solve", "clear_solve_cache"]


class PBCGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def build(verbose: bool = False, force: bool = False) -> str:
    from ._build import build as _b
    return _b(verbose=verbose, force=force)


def _lib():
    return capi.load()


def _check(st: int, what: str):
    if st != capi.PBCG_OK:
        raise PBCGError(st, "%s: %s" % (what, capi.last_error()))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need_cuda(t, name: str, dtype=torch.float64, numel: Optional[int] = None):
    """The library reads these arrays on the device: reject host tensors, other dtypes,
    strided views and wrong sizes before any call into it."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and (dtype is None or t.dtype == dtype)
            and t.is_contiguous() and (numel is None or t.numel() == numel)):
        raise ValueError("%s must be a contiguous CUDA %s tensor%s" % (
            name, dtype if dtype is not None else "", "" if numel is None else " of %d elements" % numel))


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


_PREC = {"none": capi.PREC_NONE, "jacobi": capi.PREC_JACOBI, "neumann": capi.PREC_NEUMANN}
_PRECISION = {"fp64": capi.FP64, "mixed": capi.MIXED}
_BATCH_BUILD = {"auto": 0, "regs64": 1, "stream": 2}
_METHOD = {"pipelined": capi.PIPELINED, "classic": capi.CLASSIC}
_STORAGE = {"auto": capi.STORAGE_AUTO, "general": capi.STORAGE_GENERAL}


class Solver:
    """A p-BiCGStab solver context for one matrix (``pbicgstab_create``).

    CSR: ``row_ptr`` (int32, n+1), ``col`` (int32, nnz), ``val`` (float64/float32, nnz).
    DIA: ``offsets`` (ints, ascending, containing 0) and ``dia`` (ndiag x n values).
    All tensors must be on the CUDA device; the library copies what it keeps.
    """

    def __init__(self, n: int, *, row_ptr=None, col=None, val=None, offsets: Sequence[int] = None,
                 dia: torch.Tensor = None, precond: str = "jacobi", degree: int = 0,
                 precision: str = "fp64", tol: float = 1e-10, max_it: int = 10000, rr_period: int = 0,
                 rr_theta: float = 0.0, timeout_ms: float = 2000.0, grid_blocks: int = 0,
                 block_threads: int = 0, max_restarts: int = 0, rr_auto: bool = False, rr_tau: float = 0.0,
                 method: str = "pipelined", operator_storage: str = "auto", restart_period: int = 0,
                 stag_window: int = 0, rr_cutoff: float = 0.0, prefetch_trips: int = 0,
                 barrier_overlap: int = 0, staged_sweeps: int = 0,
                 stream: Optional[torch.cuda.Stream] = None):
        lib = _lib()
        self.n = int(n)
        self.stream = stream
        m = capi.Matrix()
        m.n = self.n
        self._keep = []
        if dia is not None:
            if not (dia.is_cuda and dia.dim() == 2 and dia.shape[1] == self.n):
                raise ValueError("dia must be a CUDA tensor of shape (ndiag, n)")
            dia = dia.contiguous()
            m.format = capi.FMT_DIA
            m.val_dtype = capi.F64 if dia.dtype == torch.float64 else capi.F32
            m.val = _ptr(dia)
            offs = (C.c_int32 * len(offsets))(*[int(o) for o in offsets])
            self._keep.append(offs)
            m.ndiag = len(offsets)
            m.offsets = C.cast(offs, C.c_void_p)
            self._keep.append(dia)
        else:
            for t in (row_ptr, col, val):
                if t is None or not t.is_cuda:
                    raise ValueError("CSR arrays must be CUDA tensors")
            row_ptr = row_ptr.to(torch.int32).contiguous()
            col = col.to(torch.int32).contiguous()
            val = val.contiguous()
            m.format = capi.FMT_CSR
            m.val_dtype = capi.F64 if val.dtype == torch.float64 else capi.F32
            m.nnz = int(col.numel())
            m.row_ptr, m.col, m.val = _ptr(row_ptr), _ptr(col), _ptr(val)
            self._keep += [row_ptr, col, val]
        self.nnz = int(m.nnz) if dia is None else 0
        p = capi.Precond(_PREC[precond], int(degree))
        self.opt = capi.Options()
        _check(lib.pbicgstab_default_options(C.byref(self.opt)), "default_options")
        self.opt.precision = _PRECISION[precision]
        self.opt.tol = tol
        self.opt.max_it = max_it
        self.opt.rr_period = rr_period
        self.opt.rr_theta = rr_theta
        self.opt.timeout_ms = timeout_ms
        self.opt.grid_blocks = grid_blocks
        self.opt.block_threads = block_threads
        self.opt.max_restarts = max_restarts
        self.opt.rr_auto = int(bool(rr_auto))
        self.opt.rr_tau = rr_tau
        self.opt.method = _METHOD[method]
        self.opt.operator_storage = _STORAGE[operator_storage]
        self.opt.restart_period = restart_period
        self.opt.stag_window = stag_window
        self.opt.rr_cutoff = rr_cutoff
        self.opt.prefetch_trips = prefetch_trips
        self.opt.barrier_overlap = barrier_overlap
        self.opt.staged_sweeps = staged_sweeps
        self.ctx = C.c_void_p()
        _check(lib.pbicgstab_create(C.byref(self.ctx), C.byref(m), C.byref(p), C.byref(self.opt),
                                    _stream_handle(stream)), "pbicgstab_create")
        self._keep = []   # the library keeps its own copies

    # -------------------------------------------------------------- options
    def set_options(self, **kw):
        hist_x = kw.pop("hist_x", None)
        hist_scalars = kw.pop("hist_scalars", None)
        for k, v in kw.items():
            if k == "precision":
                v = _PRECISION[v]
            elif k == "method":
                v = _METHOD[v]
            elif k == "operator_storage":
                v = _STORAGE[v]
            setattr(self.opt, k, v)
        self.opt.hist_x = _ptr(hist_x) if hist_x is not None else None
        self.opt.hist_scalars = _ptr(hist_scalars) if hist_scalars is not None else None
        if hist_x is None:
            self.opt.record_iterates = 0
        if hist_scalars is None:
            self.opt.hist_len = 0
        _check(_lib().pbicgstab_set_options(self.ctx, C.byref(self.opt)), "pbicgstab_set_options")

    # -------------------------------------------------------------- solve
    def solve(self, b: torch.Tensor, x: Optional[torch.Tensor] = None, wait: bool = True,
              raise_on_failure: bool = False):
        """x <- solution of A x = b (x is the initial guess, default 0).  Returns (x, Result|None)."""
        if not (b.is_cuda and b.dtype == torch.float64 and b.numel() == self.n and b.is_contiguous()):
            raise ValueError("b must be a contiguous CUDA float64 vector of length n")
        if x is None:
            x = torch.zeros_like(b)
        elif not (x.is_cuda and x.dtype == torch.float64 and x.numel() == self.n and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA float64 vector of length n")
        res = capi.Result() if wait else None
        st = _lib().pbicgstab_solve(self.ctx, _ptr(b), _ptr(x), C.byref(res) if wait else None)
        if st in (capi.PBCG_INVALID_ARG, capi.PBCG_CUDA_ERROR, capi.PBCG_OUT_OF_MEMORY, capi.PBCG_TIMEOUT) or (
                raise_on_failure and st != capi.PBCG_OK):
            raise PBCGError(st, capi.last_error())
        return x, res

    def solve_host(self, b_host, x_host):
        """End-to-end solve with host (numpy float64) buffers: copies in, solve, copy out."""
        import numpy as np
        b_host = np.ascontiguousarray(b_host, dtype=np.float64)
        if x_host.dtype != np.float64 or not x_host.flags.c_contiguous:
            raise ValueError("x_host must be a contiguous float64 array")
        res = capi.Result()
        st = _lib().pbicgstab_solve_host(self.ctx, b_host.ctypes.data_as(C.c_void_p),
                                         x_host.ctypes.data_as(C.c_void_p), C.byref(res))
        if st in (capi.PBCG_INVALID_ARG, capi.PBCG_CUDA_ERROR, capi.PBCG_OUT_OF_MEMORY, capi.PBCG_TIMEOUT):
            raise PBCGError(st, capi.last_error())
        return x_host, res

    def solve_multi(self, B: torch.Tensor, X: Optional[torch.Tensor] = None):
        """Columns of B (n x nrhs, float64, CUDA) solved independently; returns (X, [Result])."""
        if not (B.is_cuda and B.dtype == torch.float64 and B.dim() == 2 and B.shape[0] == self.n):
            raise ValueError("B must be a CUDA float64 tensor of shape (n, nrhs)")
        nrhs = B.shape[1]
        Bc = B.t().contiguous()                       # column-major storage: column c contiguous
        Xc = torch.zeros_like(Bc) if X is None else X.t().contiguous()
        res = (capi.Result * nrhs)()
        st = _lib().pbicgstab_solve_multi(self.ctx, nrhs, _ptr(Bc), _ptr(Xc), res)
        if st in (capi.PBCG_INVALID_ARG, capi.PBCG_CUDA_ERROR, capi.PBCG_OUT_OF_MEMORY, capi.PBCG_TIMEOUT):
            raise PBCGError(st, capi.last_error())
        return Xc.t(), list(res)

    @property
    def storage(self) -> str:
        """"stencil" when the context keeps A as a constant-coefficient stencil, else "general"."""
        v = C.c_int32(-1)
        _check(_lib().pbicgstab_operator_storage(self.ctx, C.byref(v)), "pbicgstab_operator_storage")
        return "stencil" if v.value == capi.STORAGE_STENCIL else "general"

    def transpose(self) -> "Solver":
        """A context for A^T (``pbicgstab_create_transpose``), same preconditioner and options."""
        t = Solver.__new__(Solver)
        t.n, t.stream, t._keep, t.opt = self.n, self.stream, [], capi.Options.from_buffer_copy(self.opt)
        t.ctx = C.c_void_p()
        _check(_lib().pbicgstab_create_transpose(C.byref(t.ctx), self.ctx), "pbicgstab_create_transpose")
        return t

    def update_values(self, val: torch.Tensor):
        """New matrix values, same pattern (``pbicgstab_update_values``): CSR nnz values or
        the DIA (ndiag, n) block, float64 or float32, on the device."""
        if not (isinstance(val, torch.Tensor) and val.is_cuda and val.dtype in (torch.float64, torch.float32)):
            raise ValueError("val must be a CUDA float64 or float32 tensor")
        val = val.contiguous()
        _check(_lib().pbicgstab_update_values(self.ctx, _ptr(val), capi.F64 if val.dtype == torch.float64 else capi.F32),
               "pbicgstab_update_values")

    def update_transpose(self, src: "Solver"):
        """This context was made by ``src.transpose()``: take src's current values (``pbicgstab_update_transpose``)."""
        _check(_lib().pbicgstab_update_transpose(self.ctx, src.ctx), "pbicgstab_update_transpose")

    def value_grad(self, Lam: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        """-sum_c Lam[row_e, c] X[col_e, c] over the stored CSR entries (``pbicgstab_csr_value_grad``)."""
        if not (isinstance(X, torch.Tensor) and isinstance(Lam, torch.Tensor) and X.dim() == 2
                and Lam.shape == X.shape and X.shape[0] == self.n):
            raise ValueError("Lam and X must both have shape (n, nrhs)")
        _need_cuda(Lam.contiguous(), "Lam")
        _need_cuda(X.contiguous(), "X")
        nrhs = X.shape[1]
        Lc = Lam.t().contiguous()
        Xc = X.t().contiguous()
        g = torch.empty(self.nnz, dtype=torch.float64, device=X.device)
        _check(_lib().pbicgstab_csr_value_grad(self.ctx, nrhs, _ptr(Lc), _ptr(Xc), _ptr(g)), "value_grad")
        return g

    def spmv(self, x: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        _need_cuda(x, "x", numel=self.n)
        y = torch.empty_like(x) if y is None else y
        _need_cuda(y, "y", numel=self.n)
        if y.data_ptr() == x.data_ptr():
            raise ValueError("y must not alias x")
        _check(_lib().pbicgstab_spmv(self.ctx, _ptr(x), _ptr(y)), "pbicgstab_spmv")
        return y

    VECTORS = ("r", "rhat", "k", "w", "g", "s", "l", "z")

    def launch_info(self) -> dict:
        """The last solve's launch (``pbicgstab_launch_info``)."""
        info = (C.c_int32 * 4)()
        _check(_lib().pbicgstab_launch_info(self.ctx, info), "pbicgstab_launch_info")
        return dict(grid_blocks=info[0], block_threads=info[1], rows_per_thread=info[2],
                    prefetch_trips=info[3] % 256, barrier_overlap=(info[3] // 256) % 2,
                    staged_sweeps=info[3] // 512)

    def get_vector(self, name: str) -> torch.Tensor:
        """A work vector of the last solve (``pbicgstab_get_vector``) as a CUDA float64 tensor."""
        dev = torch.device("cuda", torch.cuda.current_device())
        out = torch.empty(self.n, dtype=torch.float64, device=dev)
        _check(_lib().pbicgstab_get_vector(self.ctx, self.VECTORS.index(name), _ptr(out)), "pbicgstab_get_vector")
        return out

    def true_residual(self, b: torch.Tensor, x: torch.Tensor) -> float:
        _need_cuda(b, "b", numel=self.n)
        _need_cuda(x, "x", numel=self.n)
        out = C.c_double()
        _check(_lib().pbicgstab_true_residual(self.ctx, _ptr(b), _ptr(x), C.byref(out)), "true_residual")
        return out.value

    def close(self):
        if getattr(self, "ctx", None):
            _lib().pbicgstab_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent CSR systems solved by one persistent launch (``pbicgstab_batch_*``).

    ``row_off``/``nnz_off``: host int64 arrays (n_sys + 1); ``row_ptr`` (local per
    system, concatenated: n_k + 1 entries each), ``col`` (local indices), ``val``:
    CUDA tensors.  ``precond``: "none", "jacobi" or "neumann" (with ``degree`` 1..8), the
    same for every system.  grid_blocks = block_threads = 0 lets the library autotune.
    ``build``: "auto", "regs64" (the 64-register kernels) or "stream" (the 40-register
    cluster kernel; mixed precision).
    """

    def __init__(self, row_off, nnz_off, row_ptr, col, val, precond: str = "jacobi", degree: int = 0,
                 precision: str = "mixed",
                 tol: float = 1e-8, max_it: int = 1000, rr_period: int = 0, rr_theta: float = 0.0,
                 grid_blocks: int = 0, block_threads: int = 0, max_restarts: int = 0, cluster_blocks: int = 0,
                 lanes_per_row: int = 0, build: str = "auto", restart_period: int = 0, stag_window: int = 0,
                 stream: Optional[torch.cuda.Stream] = None):
        import numpy as np
        lib = _lib()
        self.row_off = np.ascontiguousarray(row_off, dtype=np.int64)
        self.nnz_off = np.ascontiguousarray(nnz_off, dtype=np.int64)
        self.n_sys = len(self.row_off) - 1
        self.total_rows = int(self.row_off[-1])
        for t, name in ((row_ptr, "row_ptr"), (col, "col"), (val, "val")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda):
                raise ValueError("%s must be a CUDA tensor" % name)
        if val.dtype not in (torch.float64, torch.float32):
            raise ValueError("val must be float64 or float32")
        if row_ptr.numel() != self.total_rows + self.n_sys or col.numel() != val.numel() \
                or val.numel() != int(self.nnz_off[-1]):
            raise ValueError("row_ptr needs sum(n_k) + n_sys entries and col, val nnz_off[-1] entries each")
        row_ptr = row_ptr.to(torch.int32).contiguous()
        col = col.to(torch.int32).contiguous()
        val = val.contiguous()
        bt = capi.Batch()
        bt.n_sys = self.n_sys
        bt.val_dtype = capi.F64 if val.dtype == torch.float64 else capi.F32
        bt.row_off = self.row_off.ctypes.data_as(C.c_void_p)
        bt.nnz_off = self.nnz_off.ctypes.data_as(C.c_void_p)
        bt.row_ptr, bt.col, bt.val = _ptr(row_ptr), _ptr(col), _ptr(val)
        bt.precond = _PREC[precond]
        bt.degree = int(degree)
        self.opt = capi.Options()
        _check(lib.pbicgstab_default_options(C.byref(self.opt)), "default_options")
        self.opt.precision = _PRECISION[precision]
        self.opt.tol, self.opt.max_it = tol, max_it
        self.opt.rr_period, self.opt.rr_theta = rr_period, rr_theta
        self.opt.grid_blocks, self.opt.block_threads = grid_blocks, block_threads
        self.opt.max_restarts = max_restarts
        self.opt.cluster_blocks = cluster_blocks
        self.opt.lanes_per_row = lanes_per_row
        self.opt.batch_build = _BATCH_BUILD[build]
        self.opt.restart_period = restart_period
        self.opt.stag_window = stag_window
        self.ctx = C.c_void_p()
        _check(lib.pbicgstab_batch_create(C.byref(self.ctx), C.byref(bt), C.byref(self.opt), _stream_handle(stream)),
               "pbicgstab_batch_create")

    def solve(self, b: torch.Tensor, x: Optional[torch.Tensor] = None):
        """Returns (x, info dict with per-system numpy arrays)."""
        import numpy as np
        _need_cuda(b, "b", numel=self.total_rows)
        if x is None:
            x = torch.zeros_like(b)
        _need_cuda(x, "x", numel=self.total_rows)
        st = np.zeros(self.n_sys, np.int32)
        it = np.zeros(self.n_sys, np.int32)
        nr = np.zeros(self.n_sys, np.int32)
        tr = np.zeros(self.n_sys, np.float64)
        res = capi.BatchResult()
        res.status, res.iterations = st.ctypes.data_as(C.c_void_p), it.ctypes.data_as(C.c_void_p)
        res.n_replacements, res.rel_res_true = nr.ctypes.data_as(C.c_void_p), tr.ctypes.data_as(C.c_void_p)
        code = _lib().pbicgstab_batch_solve(self.ctx, _ptr(b), _ptr(x), C.byref(res))
        if code in (capi.PBCG_INVALID_ARG, capi.PBCG_CUDA_ERROR, capi.PBCG_OUT_OF_MEMORY, capi.PBCG_TIMEOUT):
            raise PBCGError(code, capi.last_error())
        return x, dict(status=st, iterations=it, n_replacements=nr, rel_res_true=tr, time_ms=res.time_ms,
                       n_ok=res.n_ok, block_threads=res.block_threads, grid_blocks=res.grid_blocks,
                       cluster_blocks=res.cluster_blocks, lanes_per_row=res.lanes_per_row,
                       build={1: "regs64", 2: "stream"}.get(res.batch_build, "?"))

    def close(self):
        if getattr(self, "ctx", None):
            _lib().pbicgstab_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ContextCache:
    """Solver contexts of the differentiable solve, reused across calls with the same
    sparsity pattern and options: a new call refreshes the values (``update_values``) and
    the transposed context (``update_transpose``) instead of creating both again."""

    def __init__(self, size: int = 4):
        self.size = size
        self.entries = {}   # key -> [solver, transpose or None, version of its values, version, row_ptr, col]

    @staticmethod
    def key(n, row_ptr, col, opts):
        return (n, row_ptr.data_ptr(), row_ptr.numel(), col.data_ptr(), col.numel(), row_ptr.device.index,
                tuple(sorted(opts.items())))

    def forward_solver(self, n, values, row_ptr, col, opts):
        k = self.key(n, row_ptr, col, opts)
        e = self.entries.get(k)
        if e is None:
            if len(self.entries) >= self.size:
                old = self.entries.pop(next(iter(self.entries)))
                old[0].close()
                if old[1] is not None:
                    old[1].close()
            s = Solver(n, row_ptr=row_ptr, col=col, val=values.detach(), **opts)
            # the entry holds the pattern tensors, so their storage (the key) cannot be reused
            e = self.entries[k] = [s, None, -1, 0, row_ptr, col]
        else:
            e[0].update_values(values.detach())
            e[3] += 1
        return e

    @staticmethod
    def transpose_solver(e):
        if e[1] is None:
            e[1] = e[0].transpose()
        elif e[2] != e[3]:
            e[1].update_transpose(e[0])
        e[2] = e[3]
        return e[1]

    def clear(self):
        for e in self.entries.values():
            e[0].close()
            if e[1] is not None:
                e[1].close()
        self.entries.clear()


_CACHE = _ContextCache()


class SparseSolve(torch.autograd.Function):
    """X = A^{-1} B with A given by CSR values (differentiable in ``values`` and ``B``).

    forward:  p-BiCGStab on A for every column of B (``pbicgstab_solve_multi``).
    backward: adjoint p-BiCGStab on A^T (``pbicgstab_create_transpose``) for the upstream
              gradient G = dL/dX: Lam = A^{-T} G; dL/dB = Lam; dL/dvalues = -sum_c Lam[row] X[col]
              (``pbicgstab_csr_value_grad``).
    The contexts for A and A^T are kept per sparsity pattern and options and refreshed with
    the new values on later calls (``pbicgstab_update_values`` / ``pbicgstab_update_transpose``).
    A backward pass must run before the next forward with the same pattern (it reads the
    shared contexts).
    """

    @staticmethod
    def forward(ctx, values, B, row_ptr, col, opts):
        n = B.shape[0]
        e = _CACHE.forward_solver(n, values, row_ptr, col, opts)
        s = e[0]
        X, res = s.solve_multi(B.detach())
        bad = [r.status for r in res if r.status != capi.PBCG_OK]
        if bad:
            raise PBCGError(bad[0], "forward solve did not converge")
        ctx.entry = e
        ctx.version = e[3]
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, G):
        (X,) = ctx.saved_tensors
        e = ctx.entry
        if e[3] != ctx.version:
            raise RuntimeError("sparse_solve: another forward pass with the same pattern ran before this backward")
        s = e[0]
        st = _CACHE.transpose_solver(e)
        Lam, res = st.solve_multi(G.contiguous())
        bad = [r.status for r in res if r.status != capi.PBCG_OK]
        if bad:
            raise PBCGError(bad[0], "adjoint solve did not converge")
        gvals = s.value_grad(Lam, X) if ctx.needs_input_grad[0] else None
        return gvals, (Lam if ctx.needs_input_grad[1] else None), None, None, None


def sparse_solve(values, B, row_ptr, col, **opts):
    """Differentiable solve X = A^{-1} B (A in CSR with the given values)."""
    return SparseSolve.apply(values, B, row_ptr, col, opts)


def clear_solve_cache():
    """Release the contexts ``sparse_solve`` keeps between calls."""
    _CACHE.clear()


def propagation_norms(hist: torch.Tensor, iters: int, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Column max-norms of the error propagation products (``pbicgstab_propagation_norms``).

    ``hist``: CUDA float64 tensor holding at least ``iters`` rows of ``capi.HIST_STRIDE``
    doubles, as a solve writes them to ``hist_scalars``.  Returns a (9, iters + 1) CUDA
    tensor, rows in ``capi.PROPAGATION_PRODUCTS`` order."""
    if not (hist.is_cuda and hist.dtype == torch.float64 and hist.is_contiguous()):
        raise ValueError("hist must be a contiguous CUDA float64 tensor")
    if hist.numel() < iters * capi.HIST_STRIDE:
        raise ValueError("hist holds fewer than iters rows")
    out = torch.empty(len(capi.PROPAGATION_PRODUCTS), iters + 1, dtype=torch.float64, device=hist.device)
    _check(_lib().pbicgstab_propagation_norms(_ptr(hist), capi.HIST_STRIDE, int(iters), _ptr(out),
                                              _stream_handle(stream)), "pbicgstab_propagation_norms")
    return out


def test_barrier_timeout(timeout_ms: float = 200.0, extra_arrivals: int = 1) -> str:
    st = C.c_int32(-1)
    _check(_lib().pbicgstab_test_barrier_timeout(timeout_ms, extra_arrivals, C.byref(st)), "barrier test")
    return STATUS_NAMES.get(st.value, str(st.value))
