"""Oracle pins for the residual replacement step (Eq. rr) and its policies, and for the
mixed-precision emulation."""
import numpy as np
import pytest

import oracle
import testproblems as tp


def test_periodic_schedule_and_cutoff():
    """Reading R7: replacements in iterations P, 2P, ... while ||r_i|| >= sqrt(eps) ||r_0||."""
    p = tp.problem_convdiff2d(48)
    A = p.A.to_scipy()
    r = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-13, maxit=400, rr_period=25)
    rep = [i for i, f in enumerate(r.replaced) if f]
    rn0 = np.linalg.norm(p.b)  # x0 = 0 so r_0 = b
    periodic = [i for i in rep if i % 25 == 0]
    assert periodic and all(i % 25 == 0 for i in rep[:-1])
    for i in periodic:
        # ||r_i|| is the norm logged at the end of iteration i-1
        assert r.rnorm[i - 1] >= np.sqrt(2.0 ** -52) * rn0


def test_replacement_resets_recursive_residual():
    """Right after Eq. (rr) the recursive residual equals b - A x up to the round-off of
    one FP64 SpMV: the logged ||r_{i+1}|| matches the true residual of x_{i+1}."""
    p = tp.problem_convdiff2d(40)
    A = p.A.to_scipy()
    seen = []

    def obs(stage, i, d):
        if stage == "replace":
            seen.append(np.linalg.norm((p.b - A @ d["x"]) - d["r"]) / np.linalg.norm(p.b))
    oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-12, maxit=300, rr_period=30, observer=obs)
    assert seen and max(seen) < 1e-15


def test_replacement_improves_attainable_accuracy():
    """Section 4.3 / Fig. 'unsymmetric': without replacement p-BiCGStab stagnates above
    the accuracy classic BiCGStab attains; with replacements it reaches the classic level."""
    p = tp.problem_convdiff2d(64)
    A = p.A.to_scipy()
    plain = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-12, maxit=2000)
    rr = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-12, maxit=2000, rr_period=100)
    assert plain.status == oracle.Status.STAGNATED and plain.rel_res_true > 1e-12
    assert rr.status == oracle.Status.OK and rr.rel_res_true <= 1e-12


def test_automated_replacement_reaches_tolerance():
    """Eq. (criterion) with tau = sqrt(eps): replacements happen, tolerance reached where
    plain p-BiCGStab stagnates (the bound f^r built from the paper's worst-case local
    error bounds is loose, so the count is larger than with a periodic policy)."""
    p = tp.problem_convdiff2d(64)
    A = p.A.to_scipy()
    r = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-12, maxit=2000, rr_auto=True)
    assert r.status == oracle.Status.OK and r.rel_res_true <= 1e-12
    assert 1 <= r.n_replacements <= r.iterations // 4
    assert all(np.isfinite(r.fr))


def test_mixed_first_iterates_track_fp64():
    """Mixed emulation: the first iterates agree with FP64 to FP32 accuracy."""
    p = tp.problem_convdiff2d(64)
    A = p.A.to_scipy()
    f = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-30, maxit=5, record=5)
    m = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-30, maxit=5, record=5, mixed=True)
    for i in range(5):
        assert np.linalg.norm(f.xs[i] - m.xs[i]) <= 1e-5 * np.linalg.norm(f.xs[i])


def test_mixed_with_replacement_reaches_1e10():
    """Mixed mode needs replacements (FP32 recurrences); with the relative trigger and FP64
    replacement residuals it reaches a 1e-10 true relative residual on this grid.  (It is
    not robust: on some grids, e.g. 96x96, no trigger threshold converges.)"""
    p = tp.problem_convdiff2d(64)
    A = p.A.to_scipy()
    m = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-10, maxit=3000, mixed=True, rr_theta=1e-3)
    assert m.status == oracle.Status.OK and m.rel_res_true <= 1e-10
    assert m.x.dtype == np.float64


def test_restart_after_breakdown_keeps_attainable_accuracy():
    """Not in the paper (its breakdown handling is silent): with max_restarts a breakdown
    restarts the initialisation of Algorithm 2 from the current iterate.  On TP2 pushed to an
    unreachable tolerance the plain iteration diverges after stagnating and breaks down;
    with restarts the true residual stays at the attainable level."""
    A, _ = tp.normalise(tp.tp2(200))
    N = A.n
    As = A.to_scipy()
    b = As @ np.full(N, 1 / np.sqrt(N))
    plain = oracle.pbicgstab(As, b, tol=1e-16, maxit=1000, rr_period=100)
    rs = oracle.pbicgstab(As, b, tol=1e-16, maxit=1000, rr_period=100, max_restarts=3)
    assert plain.status == oracle.Status.BREAKDOWN and plain.n_restarts == 0
    assert rs.n_restarts >= 1 and rs.status == oracle.Status.NOT_CONVERGED
    assert rs.rel_res_true <= 1e-10 < plain.rel_res_true


@pytest.mark.parametrize("mixed", [False, True])
def test_power_of_two_scaling_gives_identical_iterates(mixed):
    """Metamorphic pin: with A -> 2^k A and b -> 2^k b every Jacobi-preconditioned
    quantity of Algorithm 2 is either unchanged (k, g, u, l, m, n, alpha, omega, beta,
    x) or scaled exactly by 2^k (r, w, s, z, q, y, t, v), in FP64 and in the FP32
    emulation alike, so the iterates and the replacement schedule are bit-identical.
    Applying M^{-1} to a wrong vector, or dropping it, breaks the equality."""
    p = tp.problem_convdiff2d(24)
    A = p.A.to_scipy()
    kw = dict(precond="jacobi", tol=1e-30, maxit=60, rr_period=20, mixed=mixed, record=60)
    r1 = oracle.pbicgstab(A, p.b, **kw)
    r2 = oracle.pbicgstab(A * 4.0, p.b * 4.0, **kw)
    assert r1.iterations == r2.iterations == 60
    assert r1.replaced == r2.replaced and any(r1.replaced)
    for a, b in zip(r1.xs, r2.xs):
        assert np.array_equal(a, b)
    assert np.array_equal(np.array(r1.alpha), np.array(r2.alpha))
    assert np.array_equal(np.array(r1.rnorm) * 4.0, np.array(r2.rnorm))


def test_mixed_emulation_keeps_vectors_in_fp32():
    """The mixed mode's definition (FP32 values, vectors and preconditioner; FP64 x, dots,
    scalars and replacement residual): every recurrence vector the oracle hands to its
    observer is FP32, before and after replacements, and x stays FP64."""
    p = tp.problem_convdiff2d(20)
    A = p.A.to_scipy()
    seen = []

    def obs(stage, i, d):
        for key, v in d.items():
            if isinstance(v, np.ndarray):
                want = np.float64 if key in ("x", "x_new") else np.float32
                seen.append((stage, key, v.dtype == want))
    r = oracle.pbicgstab(A, p.b, precond="jacobi", tol=1e-30, maxit=30, rr_period=10, mixed=True, observer=obs)
    assert r.x.dtype == np.float64 and any(r.replaced)
    assert seen and all(ok for _, _, ok in seen), [s for s in seen if not s[2]][:5]
    assert {"init", "iter", "replace"} <= {s[0] for s in seen}
