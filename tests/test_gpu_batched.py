"""Batched solver (one persistent launch, one block per system) against the oracle."""
import numpy as np
import pytest

import oracle
import testproblems as tp
from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


def _batch_solver(bp, **kw):
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    c = bp.concat()
    dev = torch.device("cuda:0")
    s = pb.BatchSolver(c["row_off"], c["nnz_off"], torch.from_numpy(c["row_ptr"]).to(dev),
                       torch.from_numpy(c["col"]).to(dev), torch.from_numpy(c["val"]).to(dev), **kw)
    return s, c, torch.from_numpy(c["b"]).to(dev)


def test_batched_small_uneven_matches_oracle():
    bp = tp.problem_batched_banded(nsys=24, n_lo=50, n_hi=3000, band=64)
    s, c, b = _batch_solver(bp, precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3)
    x, info = s.solve(b)
    x = x.cpu().numpy()
    assert info["n_ok"] == 24, info["status"]
    for k, sysk in enumerate(bp.systems):
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        A = sysk.A.to_scipy(np.float64)
        true = np.linalg.norm(sysk.b - A @ xk) / np.linalg.norm(sysk.b)
        assert true <= 1e-8 and abs(true - info["rel_res_true"][k]) <= 1e-3 * true + 1e-18
        ref = oracle.pbicgstab(A, sysk.b, precond="jacobi", tol=1e-8, maxit=500, mixed=True, rr_theta=1e-3)
        assert ref.status == oracle.Status.OK
        # mixed mode: replacement points depend on FP32 rounding, so only an upper bound
        assert int(info["iterations"][k]) <= 1.5 * ref.iterations + 5


def test_batched_fp64_iterates_equal_single_solver():
    """FP64 batched solves give the same answers as the single-system solver."""
    torch = torch_cuda()
    from gpu_common import make_solver, gpu_solve
    bp = tp.problem_batched_banded(nsys=5, n_lo=500, n_hi=2000, band=40)
    s, c, b = _batch_solver(bp, precision="fp64", tol=1e-12, max_it=500, rr_period=50)
    x, info = s.solve(b)
    x = x.cpu().numpy()
    assert info["n_ok"] == 5
    for k, sysk in enumerate(bp.systems):
        single = make_solver(tp.Problem("s", sysk.A, sysk.b, sysk.x0, None, precond="jacobi", fmt="csr"),
                             tol=1e-12, max_it=500, rr_period=50)
        xs, res, _, _ = gpu_solve(single, sysk.b)
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        assert res.status == 0
        assert np.linalg.norm(xk - xs) <= 1e-10 * np.linalg.norm(xs)


def test_batched_graph_replay_and_autotune():
    bp = tp.problem_batched_banded(nsys=40, n_lo=100, n_hi=5000, band=128)
    s, c, b = _batch_solver(bp, precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3)
    x1, i1 = s.solve(b)
    x1 = x1.clone()
    x2, i2 = s.solve(b, x1.new_zeros(x1.shape))
    assert i1["n_ok"] == 40 and i2["n_ok"] == 40
    assert i1["block_threads"] in (256, 512, 1024) and i1["grid_blocks"] > 0
    assert np.array_equal(i1["iterations"], i2["iterations"])
    # same launch shape and inputs: bitwise identical solution
    assert bool((x1 == x2).all())


def test_batched_invalid_input_rejected():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    dev = torch.device("cuda:0")
    row_off = np.array([0, 2], np.int64)
    nnz_off = np.array([0, 2], np.int64)
    rp = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    col = torch.tensor([0, 7], dtype=torch.int32, device=dev)        # column out of range
    val = torch.ones(2, dtype=torch.float32, device=dev)
    with pytest.raises(pb.PBCGError) as e:
        pb.BatchSolver(row_off, nnz_off, rp, col, val)
    assert e.value.status == 1


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_batched_cluster_per_system_matches_single_solver(cluster):
    """A thread-block cluster per system (rows dealt to the cluster's blocks, cluster barrier,
    partials summed through distributed shared memory) solves every system as the
    single-system solver does; sizes include systems smaller than one block's threads."""
    torch = torch_cuda()
    from gpu_common import make_solver, gpu_solve
    import paper_1809_01948_gb300 as pb
    bp = tp.problem_batched_banded(nsys=12, n_lo=20, n_hi=6000, band=64)
    c = bp.concat()
    dev = torch.device("cuda:0")
    s = pb.BatchSolver(c["row_off"], c["nnz_off"], torch.from_numpy(c["row_ptr"]).to(dev),
                       torch.from_numpy(c["col"]).to(dev), torch.from_numpy(c["val"]).to(dev), precision="fp64",
                       tol=1e-12, max_it=800, rr_period=50, grid_blocks=4 * cluster, block_threads=256,
                       cluster_blocks=cluster)
    b = torch.from_numpy(c["b"]).to(dev)
    x, info = s.solve(b)
    assert info["cluster_blocks"] == cluster and info["grid_blocks"] == 4 * cluster
    x = x.cpu().numpy()
    assert info["n_ok"] == 12, info["status"]
    for k, sysk in enumerate(bp.systems):
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        true = np.linalg.norm(sysk.b - sysk.A.to_scipy(np.float64) @ xk) / np.linalg.norm(sysk.b)
        assert true <= 1e-11 and abs(true - info["rel_res_true"][k]) <= 1e-3 * true + 1e-18
        single = make_solver(tp.Problem("s", sysk.A, sysk.b, sysk.x0, None, precond="jacobi", fmt="csr"),
                             tol=1e-12, max_it=800, rr_period=50)
        xs, res, _, _ = gpu_solve(single, sysk.b)
        assert res.status == 0
        assert np.linalg.norm(xk - xs) <= 1e-10 * np.linalg.norm(xs)
    # replay from the captured graph: bitwise identical
    x2, info2 = s.solve(b, torch.zeros_like(b))
    assert np.array_equal(x, x2.cpu().numpy()) and np.array_equal(info["iterations"], info2["iterations"])


def test_batched_cluster_mixed_and_autotune_choice():
    bp = tp.problem_batched_banded(nsys=30, n_lo=1000, n_hi=20000, band=128)
    s, c, b = _batch_solver(bp, precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3, cluster_blocks=4)
    x, info = s.solve(b)
    assert info["n_ok"] == 30 and info["cluster_blocks"] == 4
    s2, _, _ = _batch_solver(bp, precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3)
    x2, info2 = s2.solve(b)   # autotune over one-block and cluster shapes
    assert info2["n_ok"] == 30 and info2["cluster_blocks"] in (1, 2, 4, 8) and info2["lanes_per_row"] in (1, 2, 4, 8)


def test_batched_cluster_option_rejected():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    bp = tp.problem_batched_banded(nsys=3, n_lo=100, n_hi=200, band=16)
    with pytest.raises(pb.PBCGError):
        _batch_solver(bp, cluster_blocks=3)


@pytest.mark.parametrize("lanes,cluster", [(2, 1), (4, 2), (8, 1)])
def test_batched_lanes_per_row_matches_single_solver(lanes, cluster):
    """Several threads per row in the SpMVs (shuffle-combined partial row sums) change only
    the summation order: every system still matches the single-system solver."""
    torch = torch_cuda()
    from gpu_common import make_solver, gpu_solve
    import paper_1809_01948_gb300 as pb
    bp = tp.problem_batched_banded(nsys=10, n_lo=30, n_hi=5000, band=64)
    c = bp.concat()
    dev = torch.device("cuda:0")
    s = pb.BatchSolver(c["row_off"], c["nnz_off"], torch.from_numpy(c["row_ptr"]).to(dev),
                       torch.from_numpy(c["col"]).to(dev), torch.from_numpy(c["val"]).to(dev), precision="fp64",
                       tol=1e-12, max_it=800, rr_period=50, grid_blocks=8 * cluster, block_threads=256,
                       cluster_blocks=cluster, lanes_per_row=lanes)
    b = torch.from_numpy(c["b"]).to(dev)
    x, info = s.solve(b)
    assert info["lanes_per_row"] == lanes and info["n_ok"] == 10, info["status"]
    x = x.cpu().numpy()
    for k, sysk in enumerate(bp.systems):
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        single = make_solver(tp.Problem("s", sysk.A, sysk.b, sysk.x0, None, precond="jacobi", fmt="csr"),
                             tol=1e-12, max_it=800, rr_period=50)
        xs, res, _, _ = gpu_solve(single, sysk.b)
        assert res.status == 0
        assert np.linalg.norm(xk - xs) <= 1e-10 * np.linalg.norm(xs)
    with pytest.raises(pb.PBCGError):
        pb.BatchSolver(c["row_off"], c["nnz_off"], torch.from_numpy(c["row_ptr"]).to(dev),
                       torch.from_numpy(c["col"]).to(dev), torch.from_numpy(c["val"]).to(dev), lanes_per_row=3)


def test_batched_streaming_cluster_build_equals_64_register_build():
    """The streaming cluster build (40 registers, more resident clusters) runs the same
    per-system code as the 64-register cluster kernel: identical iterates, bit for bit, at a
    fixed shape; the autotuner restricted to it solves every system; FP64, one block per
    system and 1024-thread blocks reject it."""
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    bp = tp.problem_batched_banded(nsys=24, n_lo=200, n_hi=6000, band=64)
    kw = dict(precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3, grid_blocks=16, block_threads=256,
              cluster_blocks=4)
    s1, c, b = _batch_solver(bp, build="regs64", **kw)
    s2, _, _ = _batch_solver(bp, build="stream", **kw)
    x1, i1 = s1.solve(b)
    x2, i2 = s2.solve(b)
    assert i1["build"] == "regs64" and i2["build"] == "stream"
    assert i1["n_ok"] == 24 and i2["n_ok"] == 24
    assert np.array_equal(i1["iterations"], i2["iterations"])
    assert torch.equal(x1, x2)
    s3, _, _ = _batch_solver(bp, build="stream", precision="mixed", tol=1e-8, max_it=500, rr_theta=1e-3)
    x3, i3 = s3.solve(b)
    assert i3["build"] == "stream" and i3["n_ok"] == 24 and i3["block_threads"] <= 512 and i3["cluster_blocks"] > 1
    x3 = x3.cpu().numpy()
    for k, sysk in enumerate(bp.systems):
        xk = x3[c["row_off"][k]:c["row_off"][k + 1]]
        A = sysk.A.to_scipy(np.float64)
        assert np.linalg.norm(sysk.b - A @ xk) <= 1e-7 * np.linalg.norm(sysk.b)
    for bad in (dict(build="stream", precision="fp64"), dict(build="stream", precision="mixed", cluster_blocks=1),
                dict(build="stream", precision="mixed", block_threads=1024, grid_blocks=8, cluster_blocks=2)):
        with pytest.raises(pb.PBCGError):
            _batch_solver(bp, **bad)
    s4, _, _ = _batch_solver(bp, build="stream", precision="mixed", grid_blocks=8, block_threads=256)
    with pytest.raises(pb.PBCGError):   # a fixed shape with one block per system
        s4.solve(b)


def test_batched_neumann_fp64_equals_single_solver():
    """Neumann degree 2 in the batched solver: the same answers as the single-system solver."""
    from gpu_common import make_solver, gpu_solve
    bp = tp.problem_batched_banded(nsys=5, n_lo=400, n_hi=2500, band=40)
    s, c, b = _batch_solver(bp, precond="neumann", degree=2, precision="fp64", tol=1e-12, max_it=500,
                            rr_period=50)
    x, info = s.solve(b)
    x = x.cpu().numpy()
    assert info["n_ok"] == 5, info["status"]
    for k, sysk in enumerate(bp.systems):
        single = make_solver(tp.Problem("s", sysk.A, sysk.b, sysk.x0, None, precond="neumann", degree=2, fmt="csr"),
                             tol=1e-12, max_it=500, rr_period=50)
        xs, res, _, _ = gpu_solve(single, sysk.b)
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        assert res.status == 0
        assert np.linalg.norm(xk - xs) <= 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("cluster", [1, 4])
def test_batched_neumann_mixed_matches_oracle(cluster):
    bp = tp.problem_batched_banded(nsys=12, n_lo=60, n_hi=3000, band=64)
    s, c, b = _batch_solver(bp, precond="neumann", degree=2, precision="mixed", tol=1e-8, max_it=500,
                            rr_theta=1e-3, cluster_blocks=cluster)
    x, info = s.solve(b)
    x = x.cpu().numpy()
    assert info["n_ok"] == 12, info["status"]
    for k, sysk in enumerate(bp.systems):
        xk = x[c["row_off"][k]:c["row_off"][k + 1]]
        A = sysk.A.to_scipy(np.float64)
        true = np.linalg.norm(sysk.b - A @ xk) / np.linalg.norm(sysk.b)
        assert true <= 1e-8 and abs(true - info["rel_res_true"][k]) <= 1e-3 * true + 1e-18
        ref = oracle.pbicgstab(A, sysk.b, precond="neumann", degree=2, tol=1e-8, maxit=500, mixed=True,
                               rr_theta=1e-3)
        assert ref.status == oracle.Status.OK
        assert int(info["iterations"][k]) <= 1.5 * ref.iterations + 5
