"""Pins of the oracle's nonlinear Schwarz layer (Eqs. 4-13) against facts outside the oracle.

* A single subdomain covering the whole mesh: T_1(u) = u - u* exactly (u* the solution of
  F = 0 by plain global Newton), so F_1(u) = u - u*, DF_1 = I, and the outer loop stops
  after one iteration with one GMRES iteration.
* The fixed point: F_x(u*) = 0 for every coupling, and the converged outer iterate equals
  the plain-Newton solution of F(u) = 0 (the definition of the discrete solution).
* The tangents of Eqs. 6 and 12 are derivatives: they must match central finite
  differences of F_x with the local and coarse problems re-solved.
* A tiny brute force: the tangent assembled densely from explicit inverses
  (R_i, P_i, P~_i and P_0 as dense matrices) equals the matrix-free tangent, and GMRES
  reproduces a dense direct solve of Eq. 13.
* GMRES(m) with restarts reproduces numpy's dense solve.
* The shape of Fig. 1: one-level GMRES counts grow with the number of subdomains while the
  two-level counts stay flat.
"""
import numpy as np
import pytest

from oracle import fem, schwarz as S
from paper_2410_24138_gb300 import inputs as I

TIGHT = dict(inner_rtol=1e-13, inner_atol=1e-15)


def _problem(n=16, nb=2, overlap=1):
    return I.diffusion_problem(n, I.box_partition(n, nb, nb), nb * nb, overlap)


def test_single_subdomain_reduces_to_plain_newton():
    p = _problem(16, 1)
    ustar, _ = S.plain_newton(p, tol=1e-15)
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, **TIGHT))
    rng = np.random.default_rng(4)
    u = np.where(sw.free, 0.02 * rng.standard_normal(sw.N), 0.0)
    Fx, st = sw.evaluate(u)
    np.testing.assert_allclose(Fx, u - ustar, atol=1e-13)
    A = sw.tangent(st)
    v = np.where(sw.free, rng.standard_normal(sw.N), 0.0)
    np.testing.assert_allclose(A(v), v, atol=1e-12)
    sw2 = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, outer_atol=1e-13, **TIGHT))
    usol, hist, _ = sw2.solve()
    its = [h for h in hist if "gmres_its" in h]
    assert len(its) == 1 and its[0]["gmres_its"] == 1
    np.testing.assert_allclose(usol, ustar, atol=1e-14)


@pytest.mark.parametrize("coupling", [S.ONE_LEVEL, S.ADDITIVE, S.HYBRID])
def test_fixed_point_and_converged_solution(coupling):
    p = _problem(32, 4, 1)
    ustar, _ = S.plain_newton(p, tol=1e-15)
    sw = S.Schwarz(p, S.Options(coupling=coupling, **TIGHT))
    Fx, _ = sw.evaluate(ustar)
    assert np.linalg.norm(Fx) < 1e-11
    sw = S.Schwarz(p, S.Options(coupling=coupling, outer_atol=1e-13, inner_atol=1e-15))
    u, hist, _ = sw.solve()
    outer = [h for h in hist if "gmres_its" in h]
    assert 2 <= len(outer) <= 5
    assert np.linalg.norm(u - ustar) / np.linalg.norm(ustar) < 1e-10


@pytest.mark.parametrize("coupling", [S.ONE_LEVEL, S.ADDITIVE, S.HYBRID])
def test_tangent_is_derivative_of_Fx(coupling):
    p = _problem(16, 2, 1)
    sw = S.Schwarz(p, S.Options(coupling=coupling, **TIGHT))
    rng = np.random.default_rng(5)
    u = np.where(sw.free, 0.05 * rng.random(sw.N), 0.0)
    v = np.where(sw.free, rng.standard_normal(sw.N), 0.0)
    _, st = sw.evaluate(u)
    Av = sw.tangent(st)(v)
    h = 1e-6
    fd = (sw.evaluate(u + h * v)[0] - sw.evaluate(u - h * v)[0]) / (2 * h)
    assert np.linalg.norm(Av - fd) <= 1e-8 * np.linalg.norm(fd)


def test_neohooke_tangent_is_derivative_of_Fx():
    p = I.neohooke_problem(8, I.box_partition(8, 2, 2), 4, 1, traction_max=4.0)
    sw = S.Schwarz(p, S.Options(coupling=S.HYBRID, **TIGHT))
    rng = np.random.default_rng(6)
    u = np.where(sw.free, 0.01 * rng.standard_normal(sw.N), 0.0)
    v = np.where(sw.free, rng.standard_normal(sw.N), 0.0)
    _, st = sw.evaluate(u)
    Av = sw.tangent(st)(v)
    h = 1e-6
    fd = (sw.evaluate(u + h * v)[0] - sw.evaluate(u - h * v)[0]) / (2 * h)
    assert np.linalg.norm(Av - fd) <= 1e-7 * np.linalg.norm(fd)


@pytest.mark.parametrize("coupling", [S.ADDITIVE, S.HYBRID])
def test_dense_brute_force_tangent_and_gmres(coupling):
    p = _problem(8, 2, 1)
    sw = S.Schwarz(p, S.Options(coupling=coupling, gmres_rtol=1e-13, **TIGHT))
    rng = np.random.default_rng(7)
    u = np.where(sw.free, 0.1 * rng.random(sw.N), 0.0)
    Fx, st = sw.evaluate(u)
    N = sw.N
    free = np.nonzero(sw.free)[0]
    model = fem.Model(p)
    I_N = np.eye(N)
    P0 = sw.cs.P0.toarray()
    J0 = fem.global_jacobian(model, st["u0"]).toarray()
    Q0 = P0 @ np.linalg.inv(P0.T @ J0 @ P0) @ P0.T @ J0
    local = np.zeros((N, N))
    for lp, res in zip(sw.locals, st["local"]):
        R = I_N[lp.sub.dofs]
        Pt = (R * lp.sub.owned[:, None]).T
        x = st["points"].copy()
        x[lp.sub.dofs] = res.w
        J = fem.global_jacobian(model, x).toarray()
        local += Pt @ np.linalg.inv(R @ J @ R.T) @ R @ J
    D = local + Q0 if coupling == S.ADDITIVE else local @ (I_N - Q0) + Q0
    Dff = D[np.ix_(free, free)]
    A = sw.tangent(st)
    cols = np.stack([A(I_N[:, k])[free] for k in free], axis=1)
    np.testing.assert_allclose(cols, Dff, atol=1e-11 * np.abs(Dff).max())
    du, its, rel = S.gmres(A, Fx, 1e-13, 20, 500)
    np.testing.assert_allclose(du[free], np.linalg.solve(Dff, Fx[free]), rtol=1e-9, atol=1e-14)


def test_gmres_with_restarts_matches_dense_solve():
    rng = np.random.default_rng(8)
    n = 60
    M = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, its, rel = S.gmres(lambda v: M @ v, b, 1e-12, 7, 2000)
    assert rel < 1e-11 and its > 7
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-9)


def test_newton_line_search_on_scalar_root():
    opts = S.Options(inner_atol=1e-14, inner_rtol=0.0)
    x, its, status, _, rn = S.newton(np.array([10.0]), lambda x: (np.arctan(x - 1.0), True),
                                     lambda x, r: r * (1.0 + (x - 1.0) ** 2), opts)
    assert status == S.STATUS_CONVERGED and abs(x[0] - 1.0) < 1e-13


def test_fig1_shape_one_level_grows_two_level_flat():
    counts = {}
    for nb in (2, 8):
        p = I.diffusion_problem(64, I.box_partition(64, nb, nb), nb * nb, 1)
        for coupling in (S.ONE_LEVEL, S.HYBRID):
            _, hist, _ = S.Schwarz(p, S.Options(coupling=coupling)).solve()
            counts[nb, coupling] = sum(h["gmres_its"] for h in hist if "gmres_its" in h)
    assert counts[8, S.ONE_LEVEL] > 2 * counts[2, S.ONE_LEVEL]
    assert counts[8, S.HYBRID] < 1.3 * counts[2, S.HYBRID]


@pytest.mark.parametrize("coupling", [S.ADDITIVE, S.HYBRID])
def test_rebuilt_coarse_basis_keeps_the_fixed_point(coupling):
    """The coarse space only accelerates: rebuilt from DF(u) at every outer iterate, the outer
    iteration still converges to the plain Newton solution of F(u) = 0 (the beam of Section 1, large
    deformation), and a basis fitted to the current tangent does not need more GMRES iterations."""
    p = I.beam_problem(6, 2, 3, 7.5)
    ustar, _ = S.plain_newton(p, tol=1e-12)
    its = {}
    for rebuild in (False, True):
        sw = S.Schwarz(p, S.Options(coupling=coupling, outer_atol=1e-10, gmres_maxit=100, coarse_rebuild=rebuild))
        u, hist, _ = sw.solve()
        assert np.linalg.norm(u - ustar) <= 1e-9 * np.linalg.norm(ustar)
        its[rebuild] = sum(h["gmres_its"] for h in hist if "gmres_its" in h)
    assert its[True] <= its[False]
