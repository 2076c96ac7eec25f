"""Helpers for the GPU tests: build solvers from test problems, oracle sensitivity."""
import math

import numpy as np
import pytest

import oracle
from oracle import krylov
import testproblems as tp


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1809_01948_gb300._build as b
    b.build()
    return torch


def make_solver(prob, precision="fp64", fmt=None, **kw):
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    dev = torch.device("cuda:0")
    fmt = fmt or prob.fmt
    common = dict(precond=prob.precond, degree=prob.degree, precision=precision)
    common.update(kw)
    if fmt == "dia":
        off, data = tp.csr_to_dia(prob.A)
        return pb.Solver(prob.A.n, offsets=off.tolist(), dia=torch.from_numpy(data).to(dev), **common)
    A = prob.A
    return pb.Solver(A.n, row_ptr=torch.from_numpy(A.row_ptr).to(dev), col=torch.from_numpy(A.col).to(dev),
                     val=torch.from_numpy(A.val).to(dev), **common)


def gpu_solve(solver, b, K=0, hist_len=0, x0=None, **opts):
    """Run one solve; returns (x numpy, Result, iterates (K, n) numpy, scalar history numpy)."""
    torch = torch_cuda()
    dev = torch.device("cuda:0")
    n = solver.n
    hx = torch.zeros(max(K, 1) * n, dtype=torch.float64, device=dev) if K else None
    hs = torch.full((max(hist_len, 1) * 8,), float("nan"), dtype=torch.float64, device=dev) if hist_len else None
    solver.set_options(record_iterates=K, hist_x=hx, hist_len=hist_len, hist_scalars=hs, **opts)
    bt = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64)).to(dev)
    xt = None if x0 is None else torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float64)).to(dev)
    x, res = solver.solve(bt, xt)
    torch.cuda.synchronize()
    its = hx.view(max(K, 1), n).cpu().numpy()[:K] if K else None
    hist = hs.view(-1, 8).cpu().numpy()[:hist_len] if hist_len else None
    return x.cpu().numpy(), res, its, hist


def oracle_sensitivity(A, b, K, method=None, **kw):
    """Per-iterate relative difference between two correct FP64 evaluations of the oracle
    that differ only in the summation order of the dot products (index order via BLAS vs
    an exactly rounded fsum).  This is the part of an iterate that the arithmetic of the
    method itself does not determine; parity tolerances are scaled from it."""
    method = method or oracle.pbicgstab
    a = method(A, b, tol=1e-300, maxit=K, record=K, **kw)
    orig = krylov._dot
    krylov._dot = lambda u, v: math.fsum(u.astype(np.float64) * v.astype(np.float64))
    try:
        c = method(A, b, tol=1e-300, maxit=K, record=K, **kw)
    finally:
        krylov._dot = orig
    return a, np.array([np.linalg.norm(a.xs[i] - c.xs[i]) / np.linalg.norm(a.xs[i]) for i in range(K)])


def iterate_tolerance(sens, floor=1e-10, factor=100.0):
    """max(1e-10, 100 * s_i): the stated 1e-10 wherever the problem's own rounding
    sensitivity allows it, else two orders of magnitude above that sensitivity."""
    return np.maximum(floor, factor * sens)


def oracle_iteration_spread(A, b, method=None, **kw):
    """Iterations the oracle needs under three dot-product summation orders (BLAS, exactly
    rounded fsum, reversed index order).  On the convection-diffusion operators the
    convergence history is sensitive enough that these differ (e.g. 192 vs 357 on a
    97x97 grid), so an independent implementation is compared against this range."""
    method = method or oracle.pbicgstab
    orig = krylov._dot
    orders = [orig,
              lambda u, v: math.fsum(u.astype(np.float64) * v.astype(np.float64)),
              lambda u, v: float(np.dot(u[::-1].astype(np.float64), v[::-1].astype(np.float64)))]
    out = []
    try:
        for f in orders:
            krylov._dot = f
            out.append(method(A, b, **kw))
    finally:
        krylov._dot = orig
    return out
