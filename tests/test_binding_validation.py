"""The Python binding refuses host tensors, wrong dtypes and wrong sizes before it calls
the library, whose entry points read device memory (no GPU needed)."""
import numpy as np
import pytest
import torch

import paper_1809_01948_gb300 as pb


@pytest.fixture(scope="module", autouse=True)
def _library():
    """The checks run in the binding, but the constructors load the library first."""
    from paper_1809_01948_gb300._build import build
    build()


def _bare_solver(n=8):
    s = pb.Solver.__new__(pb.Solver)
    s.n, s.nnz, s.ctx = n, 20, None
    return s


@pytest.mark.parametrize("call", [
    lambda s: s.solve(torch.zeros(8, dtype=torch.float64)),
    lambda s: s.solve_multi(torch.zeros(8, 2, dtype=torch.float64)),
    lambda s: s.spmv(torch.zeros(8, dtype=torch.float64)),
    lambda s: s.true_residual(torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float64)),
    lambda s: s.value_grad(torch.zeros(8, 2, dtype=torch.float64), torch.zeros(8, 2, dtype=torch.float64)),
    lambda s: s.value_grad(torch.zeros(8, 2, dtype=torch.float64), torch.zeros(8, 3, dtype=torch.float64)),
])
def test_solver_methods_reject_host_tensors(call):
    with pytest.raises(ValueError):
        call(_bare_solver())


def test_solver_construction_rejects_host_csr():
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    with pytest.raises(ValueError):
        pb.Solver(2, row_ptr=rp, col=torch.tensor([0, 1], dtype=torch.int32), val=torch.ones(2, dtype=torch.float64))


def test_batch_solver_rejects_host_tensors_and_bad_sizes():
    row_off = np.array([0, 2], np.int64)
    nnz_off = np.array([0, 2], np.int64)
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    col = torch.tensor([0, 1], dtype=torch.int32)
    val = torch.ones(2, dtype=torch.float32)
    with pytest.raises(ValueError):
        pb.BatchSolver(row_off, nnz_off, rp, col, val)
    b = pb.BatchSolver.__new__(pb.BatchSolver)
    b.n_sys, b.total_rows, b.ctx = 1, 2, None
    with pytest.raises(ValueError):
        b.solve(torch.zeros(2, dtype=torch.float64))


def test_propagation_norms_rejects_host_history():
    with pytest.raises(ValueError):
        pb.propagation_norms(torch.zeros(80, dtype=torch.float64), 10)
