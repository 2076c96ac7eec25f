"""Multi-RHS solves, the A^T context, value gradients and the autograd Function on the GPU,
against the oracle's dense / sparse adjoint and central finite differences."""
import numpy as np
import pytest

from oracle import adjoint
import oracle
import testproblems as tp
from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


def _csr_tensors(torch, A):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col).to(dev),
            torch.from_numpy(A.val).to(dev))


def test_multi_rhs_matches_single_solves():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=48, nrhs=5)
    rp, col, val = _csr_tensors(torch, m.A)
    s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=val, precond="jacobi", tol=1e-12, max_it=5000, rr_period=100)
    B = torch.from_numpy(m.B).cuda()
    X, res = s.solve_multi(B)
    assert all(r.status == 0 for r in res)
    A = m.A.to_scipy()
    for c in range(5):
        xs, r1 = s.solve(B[:, c].contiguous())
        assert r1.status == 0
        xc = X[:, c].cpu().numpy()
        assert np.linalg.norm(xc - xs.cpu().numpy()) <= 1e-10 * np.linalg.norm(xc)
        assert np.linalg.norm(m.B[:, c] - A @ xc) / np.linalg.norm(m.B[:, c]) <= 1e-12
        ref = oracle.pbicgstab(A, m.B[:, c], precond="jacobi", tol=1e-12, maxit=5000, rr_period=100)
        assert np.linalg.norm(xc - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_more_rhs_than_teams_run_in_waves():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=16, nrhs=7)
    rp, col, val = _csr_tensors(torch, m.A)
    s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=val, precond="jacobi", tol=1e-12, max_it=2000, rr_period=100,
                  grid_blocks=3)
    X, res = s.solve_multi(torch.from_numpy(m.B).cuda())
    A = m.A.to_scipy()
    assert len(res) == 7 and all(r.status == 0 for r in res)
    Xn = X.cpu().numpy()
    for c in range(7):
        assert np.linalg.norm(m.B[:, c] - A @ Xn[:, c]) / np.linalg.norm(m.B[:, c]) <= 1e-12


def test_transpose_context():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=40, nrhs=1)
    rp, col, val = _csr_tensors(torch, m.A)
    s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=val, precond="jacobi", tol=1e-12, max_it=3000, rr_period=100)
    t = s.transpose()
    rng = np.random.Generator(np.random.PCG64(3))
    v = rng.standard_normal(m.A.n)
    AT = m.A.to_scipy().T.tocsr()
    y = t.spmv(torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.linalg.norm(y - AT @ v) <= 1e-14 * np.linalg.norm(AT @ v)
    b = m.B[:, 0]
    x, r = t.solve(torch.from_numpy(b).cuda())
    assert r.status == 0
    assert np.linalg.norm(b - AT @ x.cpu().numpy()) / np.linalg.norm(b) <= 1e-12


def test_value_grad_kernel_matches_oracle_formula():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=20, nrhs=3)
    rp, col, val = _csr_tensors(torch, m.A)
    s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=val, precond="jacobi")
    rng = np.random.Generator(np.random.PCG64(4))
    Lam = rng.standard_normal((m.A.n, 3))
    X = rng.standard_normal((m.A.n, 3))
    g = s.value_grad(torch.from_numpy(Lam).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref = adjoint.grad_values(m.A.row_ptr, m.A.col, Lam, X)
    assert np.allclose(g, ref, rtol=1e-13, atol=1e-14)


def _loss_and_grads(torch, pb, m, tol=1e-13):
    rp, col, val = _csr_tensors(torch, m.A)
    values = val.clone().requires_grad_(True)
    B = torch.from_numpy(m.B).cuda().requires_grad_(True)
    Xt = torch.from_numpy(m.X_target).cuda()
    X = pb.sparse_solve(values, B, rp, col, precond="jacobi", tol=tol, max_it=30000, rr_period=100, rr_theta=1e-3, max_restarts=3)
    L = ((X - Xt) ** 2).sum()
    L.backward()
    return X.detach().cpu().numpy(), B.grad.cpu().numpy(), values.grad.cpu().numpy()


def test_autograd_matches_dense_adjoint():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=32, nrhs=16)
    X, gB, gv = _loss_and_grads(torch, pb, m)
    Xd, gBd, gvd = adjoint.dense_adjoint(m.A, m.B, m.X_target)
    assert np.linalg.norm(X - Xd) <= 1e-10 * np.linalg.norm(Xd)
    assert np.linalg.norm(gB - gBd) <= 1e-6 * np.linalg.norm(gBd)
    assert np.linalg.norm(gv - gvd) <= 1e-6 * np.linalg.norm(gvd)
    # entrywise on the largest entries as well
    for g, gd in ((gB.ravel(), gBd.ravel()), (gv, gvd)):
        big = np.abs(gd) > 1e-3 * np.abs(gd).max()
        assert np.max(np.abs(g[big] - gd[big]) / np.abs(gd[big])) <= 1e-6


def _fd_check(torch, pb, m, n_entries, seed=0, tol=1e-14, h_b=1e-4, h_v=1e-6):
    """Central differences of L = sum ||X - X_t||^2 on random entries of B and of the CSR
    values, with every solve converged to the tolerance `tol`.

    Step sizes.  For B, L is exactly quadratic, so central differences have no truncation
    error at any h, while the solve error enters as (solve error)/h: at h = 1e-6 that is
    about 1e-5 relative even for the CPU oracle, so B uses a larger h_b.  For the values
    the truncation error grows like (h/|a_e|)^2 and the noise like (solve error)/h."""
    X, gB, gv = _loss_and_grads(torch, pb, m, tol=tol)
    rp, col, val = _csr_tensors(torch, m.A)
    Xt = m.X_target
    rng = np.random.Generator(np.random.PCG64(seed))

    def L_with(values_np, B_np, cols):
        s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=torch.from_numpy(values_np).cuda(), precond="jacobi",
                      tol=tol, max_it=30000, rr_period=100, rr_theta=1e-3, max_restarts=3)
        Bsub = torch.from_numpy(np.ascontiguousarray(B_np[:, list(cols)])).cuda()
        Xs, res = s.solve_multi(Bsub)
        assert all(r.status == 0 for r in res)
        Xs = Xs.cpu().numpy()
        s.close()
        return float(np.sum((Xs - Xt[:, list(cols)]) ** 2))

    errs_b, errs_v = [], []
    allc = range(m.B.shape[1])
    for _ in range(n_entries):
        h = h_b
        i, c = int(rng.integers(0, m.A.n)), int(rng.integers(0, m.B.shape[1]))
        Bp, Bm = m.B.copy(), m.B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (L_with(m.A.val, Bp, [c]) - L_with(m.A.val, Bm, [c])) / (2 * h)
        errs_b.append(abs(fd - gB[i, c]) / max(abs(gB[i, c]), 1e-30))
    for _ in range(n_entries):
        h = h_v
        e = int(rng.integers(0, m.A.nnz))
        vp, vm = m.A.val.copy(), m.A.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (L_with(vp, m.B, allc) - L_with(vm, m.B, allc)) / (2 * h)
        errs_v.append(abs(fd - gv[e]) / max(abs(gv[e]), 1e-30))
    return np.array(errs_b), np.array(errs_v)


def _fd_errors(torch, pb, m, n_entries, seed, tol, h_b, h_v):
    """Like _fd_check, but returns (fd, gradient) pairs so that a scaled criterion can be used."""
    X, gB, gv = _loss_and_grads(torch, pb, m, tol=tol)
    rp, col, val = _csr_tensors(torch, m.A)
    rng = np.random.Generator(np.random.PCG64(seed))

    def L_with(values_np, B_np, cols):
        s = pb.Solver(m.A.n, row_ptr=rp, col=col, val=torch.from_numpy(values_np).cuda(), precond="jacobi",
                      tol=tol, max_it=30000, rr_period=100, rr_theta=1e-3, max_restarts=3)
        Xs, res = s.solve_multi(torch.from_numpy(np.ascontiguousarray(B_np[:, list(cols)])).cuda())
        assert all(r.status == 0 for r in res)
        out = float(np.sum((Xs.cpu().numpy() - m.X_target[:, list(cols)]) ** 2))
        s.close()
        return out

    pb_, pv = [], []
    for _ in range(n_entries):
        i, c = int(rng.integers(0, m.A.n)), int(rng.integers(0, m.B.shape[1]))
        Bp, Bm = m.B.copy(), m.B.copy()
        Bp[i, c] += h_b
        Bm[i, c] -= h_b
        pb_.append(((L_with(m.A.val, Bp, [c]) - L_with(m.A.val, Bm, [c])) / (2 * h_b), gB[i, c]))
    for _ in range(n_entries):
        e = int(rng.integers(0, m.A.nnz))
        vp, vm = m.A.val.copy(), m.A.val.copy()
        vp[e] += h_v
        vm[e] -= h_v
        allc = range(m.B.shape[1])
        pv.append(((L_with(vp, m.B, allc) - L_with(vm, m.B, allc)) / (2 * h_v), gv[e]))
    return X, gB, gv, np.array(pb_), np.array(pv)


def test_autograd_matches_central_differences_small():
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    eb, ev = _fd_check(torch, pb, tp.problem_convdiff2d_multi(n=40, nrhs=4), n_entries=12)
    assert eb.max() <= 1e-6, eb
    assert ev.max() <= 1e-6, ev


def test_autograd_full_size_convdiff2d_512_16rhs():
    """512x512 convection-diffusion, 16 right-hand sides, solves to 1e-12 (on this grid the
    adjoint solves' attainable accuracy is about 1e-12, so 1e-13 stalls).  Checks that hold
    at any size: forward and adjoint true residuals recomputed on the CPU, the value
    gradient formula on sampled entries.  Then central differences on 32 random entries of
    B (h = 1e-2: exact for the quadratic dependence) and of the values (h = 1e-4).  The FD
    noise is an absolute quantity (the solves' error in L divided by 2h), so the criterion
    is scaled: |fd - g| <= 1e-5 |g| + 1e-6 max|g| over the sampled entries."""
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=512, nrhs=16)
    X, gB, gv, fb, fv = _fd_errors(torch, pb, m, n_entries=32, seed=5, tol=1e-12, h_b=1e-2, h_v=1e-4)
    A = m.A.to_scipy()
    AT = A.T.tocsr()
    G = 2 * (X - m.X_target)
    for c in range(16):
        assert np.linalg.norm(m.B[:, c] - A @ X[:, c]) / np.linalg.norm(m.B[:, c]) <= 1e-12
        assert np.linalg.norm(G[:, c] - AT @ gB[:, c]) / np.linalg.norm(G[:, c]) <= 1e-12
    rows = np.repeat(np.arange(m.A.n), np.diff(m.A.row_ptr))
    rng = np.random.Generator(np.random.PCG64(11))
    for e in rng.integers(0, m.A.nnz, 64):
        ref = -np.dot(gB[rows[e], :], X[m.A.col[e], :])
        assert abs(gv[e] - ref) <= 1e-12 * max(1.0, abs(ref))
    for pairs in (fb, fv):
        fd, g = pairs[:, 0], pairs[:, 1]
        assert np.all(np.abs(fd - g) <= 1e-5 * np.abs(g) + 1e-6 * np.abs(g).max()), np.abs(fd - g) / np.abs(g)


def test_autograd_reuses_its_contexts_across_value_updates():
    """Three calls with one sparsity pattern and changing values: the first creates the A and
    A^T contexts, the later ones refresh their values (pbicgstab_update_values /
    pbicgstab_update_transpose); every call's gradients match the dense adjoint of its own
    values (a stale value anywhere would show)."""
    import dataclasses
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    m = tp.problem_convdiff2d_multi(n=32, nrhs=16)
    rp, col, val = _csr_tensors(torch, m.A)
    rng = np.random.Generator(np.random.PCG64(21))
    pb.clear_solve_cache()
    Xt = torch.from_numpy(m.X_target).cuda()
    for call in range(3):
        scale = 1.0 + (0.0 if call == 0 else 0.05) * rng.uniform(-1.0, 1.0, m.A.nnz)
        vnp = m.A.val * scale
        values = torch.from_numpy(vnp).cuda().requires_grad_(True)
        B = torch.from_numpy(m.B).cuda().requires_grad_(True)
        X = pb.sparse_solve(values, B, rp, col, precond="jacobi", tol=1e-13, max_it=30000, rr_period=100,
                            rr_theta=1e-3, max_restarts=3)
        ((X - Xt) ** 2).sum().backward()
        Ac = dataclasses.replace(m.A, val=vnp)
        Xd, gBd, gvd = adjoint.dense_adjoint(Ac, m.B, m.X_target)
        assert np.linalg.norm(X.detach().cpu().numpy() - Xd) <= 1e-10 * np.linalg.norm(Xd), call
        assert np.linalg.norm(B.grad.cpu().numpy() - gBd) <= 1e-6 * np.linalg.norm(gBd), call
        assert np.linalg.norm(values.grad.cpu().numpy() - gvd) <= 1e-6 * np.linalg.norm(gvd), call
    assert len(pb._CACHE.entries) == 1
    pb.clear_solve_cache()


def test_autograd_full_size_against_the_oracle_adjoint():
    """512x512, 16 right-hand sides: the gradients of the differentiable solve against the
    oracle's adjoint computed independently -- forward and adjoint solves by the C oracle
    (Algorithm 2 on all host cores, tol 1e-12, the same policy) and the value gradient by
    the oracle's formula -- to 1e-6 relative (norm-wise)."""
    torch = torch_cuda()
    import paper_1809_01948_gb300 as pb
    from oracle import c_oracle
    m = tp.problem_convdiff2d_multi(n=512, nrhs=16)
    X, gB, gv = _loss_and_grads(torch, pb, m, tol=1e-12)
    A = m.A.to_scipy()
    AT = A.T.tocsr()
    kw = dict(precond="jacobi", tol=1e-12, maxit=30000, rr_period=100, rr_theta=1e-3, max_restarts=3)
    Xo = np.zeros_like(m.B)
    Lo = np.zeros_like(m.B)
    for c in range(m.B.shape[1]):
        Xo[:, c], r = c_oracle.pbicgstab(A, m.B[:, c], **kw)
        assert r["status"] == "OK", (c, r)
    G = 2.0 * (Xo - m.X_target)
    for c in range(m.B.shape[1]):
        Lo[:, c], r = c_oracle.pbicgstab(AT, G[:, c], **kw)
        assert r["status"] == "OK", (c, r)
    gvo = adjoint.grad_values(m.A.row_ptr, m.A.col, Lo, Xo)
    assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)
    assert np.linalg.norm(gB - Lo) <= 1e-6 * np.linalg.norm(Lo)
    assert np.linalg.norm(gv - gvo) <= 1e-6 * np.linalg.norm(gvo)
