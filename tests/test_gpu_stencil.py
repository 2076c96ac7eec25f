"""The constant-coefficient stencil storage of the operator (options.operator_storage):
which matrices qualify, and that solves and SpMVs with it equal the general CSR / DIA
storage bit for bit (same products, same ascending-offset order)."""
import numpy as np
import pytest

import testproblems as tp
from gpu_common import gpu_solve, make_solver, torch_cuda

pytestmark = pytest.mark.gpu


def _variable_coefficients(prob, seed=3):
    """The same sparsity, one coupling changed by a relative 1e-3: not a stencil."""
    A = prob.A
    val = A.val.copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    e = int(rng.integers(0, A.nnz))
    while A.col[e] == np.searchsorted(A.row_ptr, e, side="right") - 1:   # an off-diagonal entry
        e = int(rng.integers(0, A.nnz))
    val[e] *= 1.001
    B = tp.CSR(A.n, A.row_ptr.copy(), A.col.copy(), val)
    return tp.Problem(prob.name + "_var", B, tp.problems._spmv(B, prob.x_star), prob.x0, prob.x_star,
                      precond=prob.precond, degree=prob.degree, fmt=prob.fmt)


def test_detection():
    torch_cuda()
    assert make_solver(tp.problem_poisson2d(30), fmt="csr", precond="none").storage == "stencil"
    assert make_solver(tp.problem_convdiff2d(40), fmt="dia").storage == "stencil"
    assert make_solver(tp.problem_convdiff2d(40), fmt="csr").storage == "stencil"
    assert make_solver(tp.problem_convdiff3d(10), fmt="csr").storage == "stencil"
    T2 = tp.tp2(20)
    p2 = tp.Problem("tp2", T2, np.ones(T2.n), np.zeros(T2.n), None, precond="jacobi", fmt="csr")
    assert make_solver(p2).storage == "stencil"
    assert make_solver(tp.problem_convdiff2d(40), fmt="dia", operator_storage="general").storage == "general"
    var = _variable_coefficients(tp.problem_convdiff2d(40))
    assert make_solver(var, fmt="csr").storage == "general"
    assert make_solver(var, fmt="dia").storage == "general"
    rng = np.random.Generator(np.random.PCG64(9))
    A = tp.random_banded_system(3000, rng)
    rb = tp.Problem("rb", A, np.ones(A.n), np.zeros(A.n), None, precond="jacobi", fmt="csr")
    assert make_solver(rb).storage == "general"


CASES = {
    "poisson_csr_none": (lambda: tp.problem_poisson2d(60), "csr", "fp64", "pipelined", dict()),
    "convdiff2d_dia_jacobi": (lambda: tp.problem_convdiff2d(96), "dia", "fp64", "pipelined", dict(rr_period=50)),
    "convdiff2d_csr_jacobi_mixed": (lambda: tp.problem_convdiff2d(64), "csr", "mixed", "pipelined", dict(rr_theta=1e-3)),
    "convdiff3d_csr_neumann": (lambda: tp.problem_convdiff3d(20), "csr", "fp64", "pipelined", dict(rr_period=50)),
    "convdiff3d_csr_neumann_mixed": (lambda: tp.problem_convdiff3d(20), "csr", "mixed", "pipelined", dict(rr_theta=3e-3)),
    "convdiff2d_dia_classic": (lambda: tp.problem_convdiff2d(96), "dia", "fp64", "classic", dict()),
    "convdiff2d_dia_auto_rr": (lambda: tp.problem_convdiff2d(64), "dia", "fp64", "pipelined", dict(rr_auto=True)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_solves_bitwise_equal_to_general_storage(name):
    """Same kernel, same launch shape: 1024-thread blocks keep the stencil context on the
    one-row kernels (the four-row ones sum the dot products in another order), so the
    stencil storage must reproduce the general storage bit for bit."""
    maker, fmt, precision, method, kw = CASES[name]
    prob = maker()
    out = []
    for storage in ("auto", "general"):
        s = make_solver(prob, fmt=fmt, precision=precision, method=method, tol=1e-10, max_it=3000,
                        operator_storage=storage, block_threads=1024, **kw)
        assert s.storage == ("stencil" if storage == "auto" else "general")
        x, res, its, hist = gpu_solve(s, prob.b, K=5, hist_len=50)
        out.append((x, res, its, hist))
    (x1, r1, i1, h1), (x2, r2, i2, h2) = out
    assert r1.status == r2.status and r1.iterations == r2.iterations and r1.n_replacements == r2.n_replacements
    assert np.array_equal(x1, x2)
    assert np.array_equal(i1, i2)
    assert np.array_equal(h1, h2, equal_nan=True)


@pytest.mark.parametrize("fmt", ["csr", "dia"])
def test_spmv_and_true_residual_equal(fmt):
    torch = torch_cuda()
    prob = tp.problem_convdiff2d(50)
    sa = make_solver(prob, fmt=fmt)
    sg = make_solver(prob, fmt=fmt, operator_storage="general")
    rng = np.random.Generator(np.random.PCG64(4))
    x = torch.from_numpy(rng.standard_normal(prob.A.n)).cuda()
    assert torch.equal(sa.spmv(x), sg.spmv(x))
    b = torch.from_numpy(prob.b).cuda()
    assert sa.true_residual(b, x) == sg.true_residual(b, x)


def test_storage_fixed_at_create():
    torch_cuda()
    import paper_1809_01948_gb300 as pb
    s = make_solver(tp.problem_convdiff2d(20), fmt="dia")
    with pytest.raises(pb.PBCGError):
        s.set_options(operator_storage="general")


def test_four_row_kernels_run_where_they_apply():
    """Stencil storage, n a multiple of 4, aligned vectors and the default block size: the
    four-row kernels; a ragged n, 1024-thread blocks or general storage: the one-row ones."""
    prob = tp.problem_convdiff2d(64)                     # n = 4096
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=500)
    _, res, _, _ = gpu_solve(s, prob.b)
    assert res.status == 0 and s.launch_info()["rows_per_thread"] == 4
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=500, block_threads=1024)
    gpu_solve(s, prob.b)
    assert s.launch_info()["rows_per_thread"] == 1
    s = make_solver(prob, fmt="dia", tol=1e-10, max_it=500, operator_storage="general")
    gpu_solve(s, prob.b)
    assert s.launch_info()["rows_per_thread"] == 1
    ragged = tp.problem_convdiff2d(63)                   # n = 3969
    s = make_solver(ragged, fmt="dia", tol=1e-10, max_it=500)
    _, res, _, _ = gpu_solve(s, ragged.b)
    assert res.status == 0 and s.launch_info()["rows_per_thread"] == 1


STAGED = {
    # name: (problem, block_threads, staged): a block stages 8 x block_threads rows per trip
    "3d_40_near": (lambda: tp.problem_convdiff3d(40), 0, True),       # offsets 1, 40, 1600 within a trip
    "3d_40_far": (lambda: tp.problem_convdiff3d(40), 128, True),      # 1600 beyond a trip: its own window
    "3d_34_far": (lambda: tp.problem_convdiff3d(34), 64, True),       # 34 near, 1156 far
    "2d_130_near_odd": (lambda: tp.problem_convdiff2d(130), 32, True),    # 130 near, not a multiple of 4
    "2d_262_far_odd": (lambda: tp.problem_convdiff2d(262), 32, False),    # 262 beyond a trip, unaligned
    "2d_512_chunked": (lambda: tp.problem_convdiff2d(512), 0, True),      # chunked row order
}


@pytest.mark.parametrize("name", list(STAGED))
def test_staged_sweeps_equal_register_sweeps(name):
    """options.staged_sweeps: the Neumann sweeps of the mixed four-row kernels read their
    operands from shared-memory stages instead of registers; same products in the same
    order, so the solve is bit for bit the register form's.  Where the layout cannot stage
    an offset the option is ignored."""
    maker, threads, staged = STAGED[name]
    prob = maker()
    out = []
    for flag in (-1, 1):
        s = make_solver(prob, fmt="csr", precision="mixed", precond="neumann", degree=2, tol=1e-9, max_it=400,
                        rr_period=50, block_threads=threads, staged_sweeps=flag)
        x, res, its, hist = gpu_solve(s, prob.b, K=5, hist_len=40)
        info = s.launch_info()
        assert info["rows_per_thread"] == 4
        assert info["staged_sweeps"] == (1 if flag > 0 and staged else 0)
        out.append((x, res, its, hist))
    (x1, r1, i1, h1), (x2, r2, i2, h2) = out
    assert r1.status == r2.status and r1.iterations == r2.iterations and r1.n_replacements == r2.n_replacements
    assert np.array_equal(x1, x2)
    assert np.array_equal(i1, i2)
    assert np.array_equal(h1, h2, equal_nan=True)


def test_staged_sweeps_automatic_rule():
    """0 (the default) stages the sweeps only where their operands exceed L2: not at 40^3."""
    prob = tp.problem_convdiff3d(40)
    s = make_solver(prob, fmt="csr", precision="mixed", tol=1e-9, max_it=50)
    gpu_solve(s, prob.b)
    assert s.launch_info()["staged_sweeps"] == 0
