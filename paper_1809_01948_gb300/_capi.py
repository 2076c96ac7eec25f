"""ctypes mirror of include/pbicgstab.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpbicgstab.so")

PBCG_OK, PBCG_INVALID_ARG, PBCG_CUDA_ERROR, PBCG_OUT_OF_MEMORY = 0, 1, 2, 3
PBCG_NOT_CONVERGED, PBCG_BREAKDOWN, PBCG_STAGNATED, PBCG_TIMEOUT = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA_ERROR", 3: "OUT_OF_MEMORY", 4: "NOT_CONVERGED",
                5: "BREAKDOWN", 6: "STAGNATED", 7: "TIMEOUT"}
FMT_CSR, FMT_DIA = 0, 1
F64, F32 = 0, 1
PREC_NONE, PREC_JACOBI, PREC_NEUMANN = 0, 1, 2
FP64, MIXED = 0, 1
PIPELINED, CLASSIC = 0, 1
STORAGE_AUTO, STORAGE_GENERAL, STORAGE_STENCIL = 0, 1, 2
HIST_STRIDE = 8
PROPAGATION_PRODUCTS = ("U", "OU", "BA", "UEA", "BAEA", "BPA", "UC", "BAC", "BD")
NOALLOC_MAX_N = 32768
NOALLOC_MAX_VALUES = 524288


class Matrix(C.Structure):
    _fields_ = [("format", C.c_int32), ("val_dtype", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("ndiag", C.c_int32), ("reserved0", C.c_int32), ("offsets", C.c_void_p)]


class Precond(C.Structure):
    _fields_ = [("kind", C.c_int32), ("degree", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_it", C.c_int32), ("tol", C.c_double),
                ("rr_period", C.c_int32), ("rr_auto", C.c_int32), ("rr_theta", C.c_double),
                ("timeout_ms", C.c_double), ("record_iterates", C.c_int32), ("hist_len", C.c_int32),
                ("hist_x", C.c_void_p), ("hist_scalars", C.c_void_p),
                ("grid_blocks", C.c_int32), ("block_threads", C.c_int32),
                ("max_restarts", C.c_int32), ("method", C.c_int32), ("rr_tau", C.c_double),
                ("operator_storage", C.c_int32), ("cluster_blocks", C.c_int32),
                ("lanes_per_row", C.c_int32), ("batch_build", C.c_int32),
                ("restart_period", C.c_int32), ("stag_window", C.c_int32), ("rr_cutoff", C.c_double),
                ("prefetch_trips", C.c_int32), ("barrier_overlap", C.c_int32),
                ("staged_sweeps", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("n_replacements", C.c_int32),
                ("n_restarts", C.c_int32), ("rel_res_recursive", C.c_double), ("rel_res_true", C.c_double),
                ("time_ms", C.c_double)]

    def as_dict(self):
        return dict(status=STATUS_NAMES.get(self.status, str(self.status)), iterations=self.iterations,
                    n_replacements=self.n_replacements, n_restarts=self.n_restarts,
                    rel_res_recursive=self.rel_res_recursive, rel_res_true=self.rel_res_true, time_ms=self.time_ms)


class Batch(C.Structure):
    _fields_ = [("n_sys", C.c_int32), ("val_dtype", C.c_int32), ("row_off", C.c_void_p), ("nnz_off", C.c_void_p),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p), ("precond", C.c_int32),
                ("degree", C.c_int32)]


class BatchResult(C.Structure):
    _fields_ = [("status", C.c_void_p), ("iterations", C.c_void_p), ("n_replacements", C.c_void_p),
                ("rel_res_true", C.c_void_p), ("time_ms", C.c_double), ("n_ok", C.c_int32),
                ("block_threads", C.c_int32), ("grid_blocks", C.c_int32), ("cluster_blocks", C.c_int32),
                ("lanes_per_row", C.c_int32), ("batch_build", C.c_int32)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "pbicgstab_default_options": (C.c_int, [C.POINTER(Options)]),
    "pbicgstab_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Matrix), C.POINTER(Precond),
                                   C.POINTER(Options), C.c_void_p]),
    "pbicgstab_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "pbicgstab_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Result)]),
    "pbicgstab_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Result)]),
    "pbicgstab_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pbicgstab_true_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "pbicgstab_get_vector": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "pbicgstab_launch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "pbicgstab_update_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "pbicgstab_update_transpose": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pbicgstab_destroy": (C.c_int, [C.c_void_p]),
    "pbicgstab_last_error": (C.c_char_p, []),
    "pbicgstab_test_barrier_timeout": (C.c_int, [C.c_double, C.c_int32, C.POINTER(C.c_int32)]),
    "pbicgstab_solve_noalloc": (C.c_int, [C.POINTER(Matrix), C.POINTER(Precond), C.POINTER(Options), C.c_void_p,
                                          C.c_void_p, C.POINTER(Result), C.c_void_p]),
    "pbicgstab_solve_multi": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pbicgstab_create_transpose": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p]),
    "pbicgstab_csr_value_grad": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pbicgstab_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Batch), C.POINTER(Options), C.c_void_p]),
    "pbicgstab_batch_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(BatchResult)]),
    "pbicgstab_batch_destroy": (C.c_int, [C.c_void_p]),
    "pbicgstab_solve_batched": (C.c_int, [C.POINTER(Batch), C.POINTER(Options), C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.POINTER(BatchResult)]),
    "pbicgstab_propagation_norms": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "pbicgstab_operator_storage": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpbicgstab.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpbicgstab.so is not built (%s); run paper_1809_01948_gb300/_build.py" % path)
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().pbicgstab_last_error().decode()
