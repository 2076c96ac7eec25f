"""Oracle pins for the error propagation analysis of Section 2.4: the 4 x 4 gap operator of
Eq. (system) with the local terms of Eq. (local), the propagation matrices of
Eq. (all_matrices) through the matrix expressions of Eq. (matrix_expr), and the products
of Eq. (all_error_matrices) against closed forms.

The strong pins reproduce gaps MEASURED in extended precision on real runs of the oracle's
Algorithm 2 (``diagnostics.PipelinedProbe``) from the measured local errors, so a wrong
sign, index or operand in any operator entry or matrix moves the prediction off the
measurement."""
import numpy as np
import pytest

import oracle
from oracle import diagnostics, propagation as pg
import testproblems as tp

LD = np.longdouble
ext = pytest.mark.skipif(not diagnostics.extended_available(), reason="needs numpy longdouble wider than double")

CASES = [("poisson", "none"), ("upwind", "jacobi")]


def _run(which, prec, K):
    p = tp.problem_poisson2d(16) if which == "poisson" else tp.problem_convdiff2d(16)
    A = p.A.to_scipy()
    M = oracle.make_precond(prec, A, 0)
    probe = diagnostics.PipelinedProbe(A, p.b, prec, M.dinv, 0, M, keep_vectors=True)
    res = oracle.pbicgstab(A, p.b, precond=prec, tol=1e-30, maxit=K, observer=probe)
    assert res.iterations == K and not any(res.replaced)
    A_ld = A.astype(LD)
    return probe.records, (lambda v: A_ld @ v)


def _rel(a, b):
    a = np.asarray(a, dtype=LD)
    b = np.asarray(b, dtype=LD)
    return float(np.sqrt(np.sum((a - b) ** 2)) / max(np.sqrt(np.sum(b ** 2)), 1e-300))


@ext
@pytest.mark.parametrize("which,prec", CASES)
def test_gap_operator_reproduces_measured_gaps(which, prec):
    """Eq. (system) + Eq. (local): G_i applied to the iteration-i gaps plus epsilon_i gives
    the measured (Delta^r_{i+1}, Delta^s_i, Delta^w_{i+1}, Delta^z_i), every iteration."""
    recs, A_ = _run(which, prec, 30)
    n = recs[0]["gap_vec"]["r"].size
    zero = np.zeros(n, dtype=LD)
    for i, rec in enumerate(recs):
        sc = rec["scalars"]
        G = pg.gap_operator(sc["alpha"], sc["beta"], sc["omega"], sc["omega_prev"])
        prev_s = recs[i - 1]["gap_vec"]["s"] if i > 0 else zero   # Delta_{-1} = 0 (R3)
        prev_z = recs[i - 1]["gap_vec"]["z"] if i > 0 else zero
        old = [rec["gap_vec"]["r"], prev_s, rec["gap_vec"]["w"], prev_z]
        eps = pg.local_error_terms(A_, rec["delta_vec"], LD(sc["alpha"]), LD(sc["omega"]))
        new = [rec["gap_next_vec"]["r"], rec["gap_vec"]["s"], rec["gap_next_vec"]["w"], rec["gap_vec"]["z"]]
        for row, key in enumerate("rswz"):
            pred = sum(LD(G[row, c]) * old[c] for c in range(4)) + eps[key]
            assert _rel(pred, new[row]) < 1e-2, (i, key, _rel(pred, new[row]))


@ext
@pytest.mark.parametrize("which,prec", CASES)
def test_matrix_expressions_reproduce_measured_gaps(which, prec):
    """Eq. (matrix_expr) with the matrices of Eq. (all_matrices) and the Theta matrices of
    Eq. (thetas) (index reading in ``oracle/propagation.py``): the columns of R, S, W, Z
    equal the measured gaps Delta_0 .. Delta_{m-1}."""
    m = 25
    recs, A_ = _run(which, prec, m)
    n = recs[0]["gap_vec"]["r"].size
    alpha = [recs[j]["scalars"]["alpha"] for j in range(m - 1)]
    omega = [recs[j]["scalars"]["omega"] for j in range(m - 1)]
    beta_next = [recs[j + 1]["scalars"]["beta"] for j in range(m - 1)]
    mats = {k: v.astype(LD) for k, v in pg.propagation_matrices(alpha, beta_next, omega).items()}
    dv = lambda key, j: recs[j]["delta_vec"][key]

    def theta(first, cols):
        T = np.zeros((n, m), dtype=LD)
        if first is not None:
            T[:, 0] = first
        for k in range(1, m):
            T[:, k] = cols(k)
        return T

    g0 = recs[0]["gap_vec"]
    Tx = theta(None, lambda k: -dv("x", k - 1))
    Tr = theta(g0["r"], lambda k: -dv("r", k - 1))
    Tu = theta(None, lambda k: dv("u", k - 1))
    Tp = theta(None, lambda k: -dv("q", k - 1))
    Ty = theta(None, lambda k: -dv("y", k - 1))
    Tg = theta(None, lambda k: dv("g", k))
    Ts = theta(g0["s"], lambda k: -dv("s", k))
    Tk = theta(None, lambda k: dv("k", k - 1))
    Tw = theta(g0["w"], lambda k: -dv("w", k - 1))
    Tl = theta(None, lambda k: dv("l", k))
    Tz = theta(g0["z"], lambda k: -dv("z", k))
    AM = lambda T: np.stack([A_(T[:, k]) for k in range(m)], axis=1)
    Am, Bm, Em, Pm, Cm, Dm, Om, Um = (mats[k] for k in "ABEPCDOU")
    Z = (AM(Tl) + Tz) @ Bm
    W = (AM(Tk) + Tw + AM(Tu) + Ty) @ Um + Z @ Am
    S = (AM(Tg) + Ts) @ Bm + W @ Em + Z @ Pm
    R = (AM(Tx) + Tr + AM(Tu) @ Om + Tp + Ty @ Om) @ Um + S @ Am + W @ Cm + Z @ Dm
    for j in range(m):
        gv = recs[j]["gap_vec"]
        for key, M_ in (("z", Z), ("w", W), ("s", S), ("r", R)):
            assert _rel(M_[:, j], gv[key]) < 1e-2, (j, key, _rel(M_[:, j], gv[key]))


def _random_scalars(m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.uniform(0.2, 2.0, m - 1), rng.uniform(0.3, 1.5, m - 1) * rng.choice([-1, 1], m - 1),
            rng.uniform(-1.0, 1.0, m - 1))


def test_products_against_elementwise_sums():
    """Entries of BA, UC, BD, OU and UEA from hand-derived scalar sums over the definitions:
    (BA)_rj = -sum_{r<=k<j} alpha_k prod_{r<l<=k} beta_l, (UC)_rj = -sum_{r<=k<j} omega_k,
    (BD)_rj = sum_{r<=k<j} omega_k alpha_k prod_{r<l<=k} beta_l, (OU)_rj = -omega_{r-1}
    (1 <= r <= j), (UEA)_rj = -sum_{1<=k<j} alpha_k sum_{max(r,1)<=l<=k} prod_{l<t<=k} beta_t."""
    m = 9
    alpha, beta_next, omega = _random_scalars(m, 11)
    beta = np.concatenate([[np.nan], beta_next])
    P = pg.error_matrix_products(pg.propagation_matrices(alpha, beta_next, omega))
    bp = lambda a, b: np.prod(beta[a + 1:b + 1]) if b > a else 1.0   # beta_{a+1} .. beta_b
    for r in range(m):
        for j in range(m):
            ba = -sum(alpha[k] * bp(r, k) for k in range(r, j))
            uc = -sum(omega[k] for k in range(r, j))
            bd = sum(omega[k] * alpha[k] * bp(r, k) for k in range(r, j))
            ou = -omega[r - 1] if 1 <= r <= j else 0.0
            uea = -sum(alpha[k] * sum(bp(l, k) for l in range(max(r, 1), k + 1)) for k in range(1, j))
            for name, want in (("BA", ba), ("UC", uc), ("BD", bd), ("OU", ou), ("UEA", uea)):
                assert abs(P[name][r, j] - want) <= 1e-12 * (1 + abs(want)), (name, r, j)


def test_column_norms_constant_scalars_closed_forms():
    """Constant alpha = a, beta = b, omega = w: column j of BA has max-norm a (1 - b^j)/(1 - b),
    of UC |w| j, of BD |w| a (1 - b^j) / (1 - b), of U 1 and of OU |w| (j >= 1)."""
    m, a, b, w = 40, 0.7, 0.9, -0.4
    N = pg.propagation_column_norms(np.full(m - 1, a), np.full(m - 1, b), np.full(m - 1, w))
    idx = {k: i for i, k in enumerate(pg.PRODUCT_NAMES)}
    j = np.arange(m)
    geo = (1 - b ** j) / (1 - b)
    assert np.allclose(N[idx["U"]], 1.0)
    assert np.allclose(N[idx["OU"]], np.where(j >= 1, abs(w), 0.0))
    assert np.allclose(N[idx["BA"]], a * geo, rtol=1e-13)
    assert np.allclose(N[idx["UC"]], abs(w) * j, rtol=1e-13)
    assert np.allclose(N[idx["BD"]], abs(w) * a * geo, rtol=1e-13)


def test_omega_zero_removes_the_stabilising_terms():
    """omega = 0 (the p-CG limit the paper describes): P, C, D and O vanish, so OU, BPA, UC,
    BAC and BD are zero and the gap operator loses its omega couplings."""
    m = 12
    alpha, beta_next, _ = _random_scalars(m, 5)
    N = pg.propagation_column_norms(alpha, beta_next, np.zeros(m - 1))
    for name in ("OU", "BPA", "UC", "BAC", "BD"):
        assert np.all(N[pg.PRODUCT_NAMES.index(name)] == 0.0), name
    G = pg.gap_operator(0.5, 0.8, 0.0, 0.0)
    assert G[0, 3] == 0.0 and G[1, 3] == 0.0 and G[0, 2] == -0.5


def test_growth_on_a_real_run_is_reported_per_column():
    """On the convection-diffusion run the products grow by orders of magnitude (the
    paper's observation), and column j depends on the first j iterations only (up to the
    rounding of differently blocked dense products)."""
    p = tp.problem_convdiff2d(64)
    res = oracle.pbicgstab(p.A.to_scipy(), p.b, precond="jacobi", tol=1e-30, maxit=120)
    al, om, be = np.array(res.alpha), np.array(res.omega), np.array(res.beta)
    N = pg.propagation_column_norms(al[:119], be[:119], om[:119])
    N_short = pg.propagation_column_norms(al[:59], be[:59], om[:59])
    assert np.allclose(N[:, :60], N_short, rtol=1e-12, atol=0)
    assert N[pg.PRODUCT_NAMES.index("BA")].max() > 10.0
