"""GPU parity of the error propagation diagnostics (pbicgstab_propagation_norms) against
the oracle's dense products of Eq. (all_error_matrices).  Scalar sequences come from the
oracle's own Algorithm 2 runs or from a seeded generator, never from the GPU."""
import numpy as np
import pytest

import oracle
from oracle import propagation as pg
import testproblems as tp
from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu

STRIDE = 8


def _hist(torch, alpha, omega, beta_next):
    h = np.full((len(alpha), STRIDE), np.nan)
    h[:, 0], h[:, 1], h[:, 2] = alpha, omega, beta_next
    return torch.from_numpy(h.reshape(-1)).cuda()


def _gpu_norms(alpha, omega, beta_next):
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    out = pb.propagation_norms(_hist(torch, alpha, omega, beta_next), len(alpha))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare(gpu, ref, rtol):
    assert gpu.shape == ref.shape
    scale = np.maximum(ref, 1e-300)
    err = np.abs(gpu - ref) / scale
    assert np.all((err <= rtol) | ((ref == 0) & (gpu == 0))), float(np.nanmax(np.where(ref > 0, err, 0)))


def _random_scalars(m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.uniform(0.2, 2.0, m - 1), rng.uniform(-1.0, 1.0, m - 1),
            rng.uniform(0.3, 1.2, m - 1) * rng.choice([-1, 1], m - 1))


@pytest.mark.parametrize("m", [1, 2, 3, 40, 256, 257, 300])
def test_random_scalars_match_oracle(m):
    """Ragged sizes around the 256-row block; columns of every product, relative 1e-11."""
    alpha, omega, beta_next = _random_scalars(m, 100 + m)
    ref = pg.propagation_column_norms(alpha, beta_next, omega)
    gpu = _gpu_norms(alpha, omega, beta_next)
    _compare(gpu, ref, 1e-11)


def test_convection_diffusion_run_matches_oracle():
    """The scalars of 300 iterations of the oracle's Algorithm 2 on the 2D convection-diffusion
    problem (64 x 64, Jacobi), where the products grow by orders of magnitude."""
    p = tp.problem_convdiff2d(64)
    res = oracle.pbicgstab(p.A.to_scipy(), p.b, precond="jacobi", tol=1e-30, maxit=301)
    al, om, be = np.array(res.alpha[:300]), np.array(res.omega[:300]), np.array(res.beta[:300])
    ref = pg.propagation_column_norms(al, be, om)
    gpu = _gpu_norms(al, om, be)
    assert ref[pg.PRODUCT_NAMES.index("BA")].max() > 10.0
    _compare(gpu, ref, 1e-10)


def test_long_history_columns_depend_on_their_prefix_only():
    """At the length of a full solve (3,000 iterations): the first 801 columns equal the
    oracle's 801-column products and the 801-column GPU result (column j uses rows < j)."""
    m = 3001
    alpha, omega, beta_next = _random_scalars(m, 7)
    beta_next = np.clip(beta_next, -0.98, 0.98)     # keep 3,000-fold products finite
    full = _gpu_norms(alpha, omega, beta_next)
    short = _gpu_norms(alpha[:800], omega[:800], beta_next[:800])
    assert np.array_equal(full[:, :801], short)
    ref = pg.propagation_column_norms(alpha[:800], beta_next[:800], omega[:800])
    _compare(short, ref, 1e-10)
    assert np.all(np.isfinite(full))


def test_invalid_arguments_rejected():
    torch = torch_cuda()
    import ctypes as C
    import paper_1809_01948_gb300 as pb
    from paper_1809_01948_gb300 import _capi as capi
    lib = capi.load()
    h = torch.zeros(8 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(9 * 5, dtype=torch.float64, device="cuda")
    hp, op = C.c_void_p(h.data_ptr()), C.c_void_p(out.data_ptr())
    assert lib.pbicgstab_propagation_norms(hp, 2, 4, op, None) == 1          # stride < 3
    assert lib.pbicgstab_propagation_norms(hp, 8, -1, op, None) == 1         # negative iters
    assert lib.pbicgstab_propagation_norms(hp, 8, 70000, op, None) == 1      # above the limit
    assert lib.pbicgstab_propagation_norms(None, 8, 4, op, None) == 1
    with pytest.raises(ValueError):
        pb.propagation_norms(h, 5)                                            # too few rows
    # zero iterations: one column, U = 1 and every other product 0
    n0 = pb.propagation_norms(h, 0).cpu().numpy()
    assert n0.shape == (9, 1) and n0[0, 0] == 1.0 and np.all(n0[1:, 0] == 0.0)
