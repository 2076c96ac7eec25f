"""ctypes wrapper of the C oracle (``c_oracle.c``): Algorithm 2 with Eq. (rr), the
replacement and restart policies, FP64 or the mixed FP32/FP64 emulation, on all host
cores.  TEST INFRASTRUCTURE ONLY (tests/ and the CPU legs of bench.py).

It restates ``krylov.pbicgstab`` step for step in C so that the CPU baseline runs the
benchmark systems to completion; ``tests/test_oracle_c.py`` pins it to that oracle
(iterates, statuses, iteration counts and residuals on the test problems).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c_oracle.c")
LIB = os.path.join(HERE, "lib", "liboracle.so")
STATUS = {0: "OK", 4: "NOT_CONVERGED", 5: "BREAKDOWN", 6: "STAGNATED"}


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_it", C.c_int), ("rr_period", C.c_int), ("rr_theta", C.c_double),
                ("restart_period", C.c_int), ("stag_window", C.c_int), ("max_restarts", C.c_int)]


class Res(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("n_replacements", C.c_int), ("n_restarts", C.c_int),
                ("rel_res_recursive", C.c_double), ("rel_res_true", C.c_double)]


def build(force: bool = False) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off (portable C99: no target-specific flags)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    deps = [SRC, os.path.join(HERE, "c_oracle_body.h")]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in deps):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", LIB, SRC, "-lm"])
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.oracle_pbicgstab.restype = C.c_int
        lib.oracle_pbicgstab.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                         C.c_void_p, C.c_void_p, C.POINTER(Opts), C.POINTER(Res), C.c_int]
        lib.oracle_stream_copy_gbs.restype = C.c_double
        lib.oracle_stream_copy_gbs.argtypes = [C.c_long, C.c_int, C.c_int]
        lib.oracle_threads.restype = C.c_int
        _lib = lib
    return _lib


_KIND = {"none": 0, "jacobi": 1, "neumann": 2}


def pbicgstab(A, b, x0=None, precond="none", degree=0, mixed=False, tol=1e-10, maxit=1000, rr_period=0,
              rr_theta=0.0, restart_period=0, stag_window=0, max_restarts=0, threads=0):
    """Returns (x, dict(status, iterations, n_replacements, n_restarts, rel_res_recursive,
    rel_res_true)).  ``A``: scipy CSR (FP64 values, sorted column indices)."""
    lib = _load()
    A = A.tocsr()
    A.sort_indices()
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.shape[0]) if x0 is None else np.array(x0, dtype=np.float64)
    o = Opts(tol, maxit, rr_period, rr_theta, restart_period, stag_window, max_restarts)
    r = Res()
    rc = lib.oracle_pbicgstab(A.shape[0], rp.ctypes.data, col.ctypes.data, val.ctypes.data, _KIND[precond],
                              int(degree), int(bool(mixed)), b.ctypes.data, x.ctypes.data, C.byref(o),
                              C.byref(r), int(threads))
    if rc != 0:
        raise MemoryError("C oracle: allocation failed")
    return x, dict(status=STATUS.get(r.status, str(r.status)), iterations=r.iterations,
                   n_replacements=r.n_replacements, n_restarts=r.n_restarts,
                   rel_res_recursive=r.rel_res_recursive, rel_res_true=r.rel_res_true)


def host_copy_gbs(n: int = 1 << 26, reps: int = 5, threads: int = 0) -> float:
    """Host memory bandwidth (parallel copy, read + write bytes per second, best of reps)."""
    return _load().oracle_stream_copy_gbs(int(n), int(reps), int(threads))


def threads() -> int:
    return _load().oracle_threads()
