"""Pins of the oracle's finite-element layer (Eqs. 1-3) against facts fixed outside the oracle.

* Jacobians against central finite differences of the residual.
* Eq. 1 at k = 1 on this triangulation is the classical 5-point stencil; its small-load
  limit is the finite-difference Poisson solution, computed here in closed form by a
  discrete sine transform (scipy.fft), not by the oracle's assembly.
* Eq. 1 is Kirchhoff-transformable: G(u) = u + u^3/3 satisfies -Laplace G(u) = f, so the
  FE solution must approach G^-1 of the Poisson solution at second order in h.
* A manufactured solution converges at second order in h.
* Eq. 2: the residual is the gradient of the stored energy
  W(F) = mu/2 (|F|^2 - 2) - mu ln J + lambda/2 (ln J)^2, evaluated by an independent routine
  in this file; a rigid rotation is stress free; a uniaxial stretch gives the closed-form
  stress; the tangent is symmetric.
"""
import numpy as np
import pytest
from scipy.fft import dstn, idstn

from oracle import fem, schwarz
from paper_2410_24138_gb300 import inputs as I


def _random_p1(rng, E=20):
    X = np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.9]])[None] + 0.2 * rng.random((E, 3, 2))
    return X, rng.standard_normal((E, 3)), 0.5 + rng.random(E), rng.random(E)


def test_p1_jacobian_matches_finite_differences():
    rng = np.random.default_rng(1)
    X, ue, k, f = _random_p1(rng)
    _, K = fem.diffusion_p1(X, ue, k, f)
    h = 1e-6
    for b in range(3):
        d = np.zeros_like(ue)
        d[:, b] = h
        rp, _ = fem.diffusion_p1(X, ue + d, k, f, want_jac=False)
        rm, _ = fem.diffusion_p1(X, ue - d, k, f, want_jac=False)
        fd = (rp - rm) / (2 * h)
        assert np.max(np.abs(fd - K[:, :, b])) <= 1e-7 * np.max(np.abs(K))


def test_p1_reference_element_by_hand():
    # unit right triangle, u = (1, 2, 3) = 1 + x + 2y: grad u = (1, 2); midpoints 1.5, 2.5, 2 -> int(1+u^2) = (1/6)(3 + 2.25 + 6.25 + 4)
    X = np.array([[[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]])
    ue = np.array([[1.0, 2.0, 3.0]])
    r, _ = fem.diffusion_p1(X, ue, np.array([1.0]), np.array([0.0]))
    Q = (3.0 + 2.25 + 6.25 + 4.0) / 6.0
    grads = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    np.testing.assert_allclose(r[0], Q * grads @ np.array([1.0, 2.0]), rtol=1e-14)


def test_p1_linearisation_is_five_point_stencil():
    n = 8
    p = I.diffusion_problem(n, I.box_partition(n, 1, 1), 1, 1)
    model = fem.Model(p)
    K = fem.global_jacobian(model, np.zeros(p.n_nodes)).toarray()
    m = n + 1
    for j in range(1, n):
        for i in range(1, n):
            a = j * m + i
            expect = np.zeros(p.n_nodes)
            expect[a] = 4.0
            for b in (a - 1, a + 1, a - m, a + m):
                expect[b] = -1.0
            np.testing.assert_allclose(K[a], expect, atol=1e-13)
    F0 = fem.global_residual(model, np.zeros(p.n_nodes))
    free = fem.free_mask(p)
    np.testing.assert_allclose(F0[free], -(1.0 / n) ** 2, rtol=1e-13)


def _fd_poisson(n, f=1.0):
    """Finite-difference Poisson solution of -Laplace v = f, v = 0 on the boundary (interior nodes)."""
    h = 1.0 / n
    k = np.arange(1, n)
    s = (4.0 / h ** 2) * np.sin(np.pi * k / (2 * n)) ** 2
    lam = s[:, None] + s[None, :]
    rhs = np.full((n - 1, n - 1), f)
    return idstn(dstn(rhs, type=1) / lam, type=1)


def _interior(u, n):
    return u.reshape(n + 1, n + 1)[1:-1, 1:-1]


def test_small_load_limit_is_fd_poisson():
    n, eps = 16, 1e-3
    p = I.diffusion_problem(n, I.box_partition(n, 1, 1), 1, 1, f_cell=np.full(n * n, eps))
    u, _ = schwarz.plain_newton(p, tol=1e-16)
    v = _fd_poisson(n)
    err = np.max(np.abs(_interior(u, n) / eps - v)) / np.max(np.abs(v))
    assert err < 1e-5   # the cubic term contributes O(eps^2) relative


def _g_inverse(v):
    u = v.copy()
    for _ in range(60):
        u -= (u + u ** 3 / 3.0 - v) / (1.0 + u ** 2)
    return u


def test_kirchhoff_transform_second_order():
    errs = []
    for n in (16, 32, 64):
        p = I.diffusion_problem(n, I.box_partition(n, 1, 1), 1, 1)
        u, _ = schwarz.plain_newton(p, tol=1e-14)
        errs.append(np.max(np.abs(_interior(u, n) - _g_inverse(_fd_poisson(n)))))
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.2 < r < 4.8 for r in rates), (errs, rates)


def test_manufactured_solution_second_order():
    errs = []
    for n in (8, 16, 32):
        xy, conn = I.structured_mesh(n, I.P1_TRI)
        c = xy[conn].mean(axis=1)
        x, y = c[:, 0], c[:, 1]
        us = np.sin(np.pi * x) * np.sin(np.pi * y)
        grad2 = np.pi ** 2 * ((np.cos(np.pi * x) * np.sin(np.pi * y)) ** 2 + (np.sin(np.pi * x) * np.cos(np.pi * y)) ** 2)
        fval = 2 * np.pi ** 2 * us * (1 + us ** 2) - 2 * us * grad2
        p = I.diffusion_problem(n, I.box_partition(n, 1, 1), 1, 1)
        p.f_elem = fval
        u, _ = schwarz.plain_newton(p, tol=1e-13)
        exact = np.sin(np.pi * p.xy[:, 0]) * np.sin(np.pi * p.xy[:, 1])
        errs.append(np.sqrt(np.mean((u - exact) ** 2)))
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.0 < r < 5.0 for r in rates), (errs, rates)


# ---------------------------------------------------------------------------------------------
# Eq. 2
# ---------------------------------------------------------------------------------------------

def _stored_energy(Fd, mu, lam):
    J = Fd[..., 0, 0] * Fd[..., 1, 1] - Fd[..., 0, 1] * Fd[..., 1, 0]
    return 0.5 * mu * (np.sum(Fd * Fd, axis=(-1, -2)) - 2.0) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2


def _element_energy(X, U, mu, lam):
    """sum over 2x2 Gauss points of W(F) det(dX/dxi): an independent Q1 implementation."""
    g = 1.0 / np.sqrt(3.0)
    total = 0.0
    for xi in (-g, g):
        for eta in (-g, g):
            dN = 0.25 * np.array([[-(1 - eta), -(1 - xi)], [(1 - eta), -(1 + xi)],
                                  [(1 + eta), (1 + xi)], [-(1 + eta), (1 - xi)]])
            Jm = X.T @ dN
            B = dN @ np.linalg.inv(Jm)
            Fd = np.eye(2) + U.T @ B
            total += _stored_energy(Fd, mu, lam) * np.linalg.det(Jm)
    return total


def _random_q1(rng):
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.1, 0.9], [0.05, 1.0]]) + 0.05 * rng.random((4, 2))
    U = 0.1 * rng.standard_normal((4, 2))
    return X, U


def test_neohooke_residual_is_energy_gradient():
    rng = np.random.default_rng(2)
    mu, lam = fem.lame(210.0, 0.3)
    for _ in range(5):
        X, U = _random_q1(rng)
        r, _, _ = fem.neohooke_q1(X[None], U.reshape(1, 8), mu, lam, want_jac=False)
        h = 1e-6
        grad = np.zeros(8)
        for d in range(8):
            e = np.zeros(8)
            e[d] = h
            grad[d] = (_element_energy(X, (U.ravel() + e).reshape(4, 2), mu, lam)
                       - _element_energy(X, (U.ravel() - e).reshape(4, 2), mu, lam)) / (2 * h)
        np.testing.assert_allclose(r[0], grad, rtol=1e-6, atol=1e-6 * np.max(np.abs(grad)))


def test_neohooke_tangent_fd_and_symmetric():
    rng = np.random.default_rng(3)
    mu, lam = fem.lame(210.0, 0.3)
    X, U = _random_q1(rng)
    _, K, _ = fem.neohooke_q1(X[None], U.reshape(1, 8), mu, lam)
    h = 1e-6
    for d in range(8):
        e = np.zeros(8)
        e[d] = h
        rp, _, _ = fem.neohooke_q1(X[None], (U.ravel() + e)[None], mu, lam, want_jac=False)
        rm, _, _ = fem.neohooke_q1(X[None], (U.ravel() - e)[None], mu, lam, want_jac=False)
        np.testing.assert_allclose((rp - rm)[0] / (2 * h), K[0, :, d], rtol=1e-6, atol=1e-6 * np.abs(K).max())
    np.testing.assert_allclose(K[0], K[0].T, atol=1e-10 * np.abs(K).max())


def test_neohooke_rigid_rotation_is_stress_free():
    mu, lam = fem.lame(210.0, 0.3)
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    U = X @ R.T - X + np.array([0.3, -0.2])
    r, _, det = fem.neohooke_q1(X[None], U.reshape(1, 8), mu, lam, want_jac=False)
    assert np.max(np.abs(r)) < 1e-12
    np.testing.assert_allclose(det, 1.0, rtol=1e-14)


def test_neohooke_uniaxial_stretch_closed_form():
    mu, lam = fem.lame(210.0, 0.3)
    s = 1.3
    P, _, _ = fem.neohooke_stress(np.array([[s, 0.0], [0.0, 1.0]]), mu, lam)
    np.testing.assert_allclose(P[0, 0], mu * (s - 1.0 / s) + lam * np.log(s) / s, rtol=1e-14)
    np.testing.assert_allclose(P[1, 1], 0.0 + lam * np.log(s), rtol=1e-14)
    assert abs(P[0, 1]) < 1e-14 and abs(P[1, 0]) < 1e-14
    np.testing.assert_allclose(fem.lame(210.0, 0.3), (210.0 / 2.6, 210.0 * 0.3 / (1.3 * 0.4)), rtol=1e-15)


def test_plane_stress_lambda_is_the_textbook_constant():
    """The plane-stress reduction lambda* = 2 mu lambda / (lambda + 2 mu) equals the textbook
    plane-stress Lame constant E nu / (1 - nu^2); mu is unchanged."""
    for E, nu in ((210.0, 0.3), (1.0, 0.45), (70.0, 0.0)):
        mu, lam = fem.lame(E, nu, plane_stress=True)
        np.testing.assert_allclose(lam, E * nu / (1.0 - nu * nu), rtol=1e-14, atol=1e-300)
        np.testing.assert_allclose(mu, fem.lame(E, nu)[0], rtol=1e-15)


@pytest.mark.parametrize("plane_stress", [True, False])
def test_uniaxial_stress_modulus_and_contraction(plane_stress):
    """A small uniaxial stress state: stretch eps along x, the transverse stretch eta found from
    P_yy = 0.  With the plane-stress lambda the 2D modulus P_xx / eps is Young's E and the
    contraction -eta / eps is nu; with the printed (plane-strain) lambda they are E / (1 - nu^2)
    and nu / (1 - nu) (both to O(eps))."""
    from scipy.optimize import brentq
    E, nu, eps = 210.0, 0.3, 1e-6
    mu, lam = fem.lame(E, nu, plane_stress=plane_stress)

    def stress(eta):
        return fem.neohooke_stress(np.array([[1.0 + eps, 0.0], [0.0, 1.0 + eta]]), mu, lam)[0]

    eta = brentq(lambda t: stress(t)[1, 1], -10 * eps, 10 * eps, xtol=1e-18, rtol=1e-15)
    modulus, contraction = stress(eta)[0, 0] / eps, -eta / eps
    if plane_stress:
        np.testing.assert_allclose([modulus, contraction], [E, nu], rtol=1e-4)
    else:
        np.testing.assert_allclose([modulus, contraction], [E / (1 - nu * nu), nu / (1 - nu)], rtol=1e-4)


def test_traction_load_total_force():
    p = I.neohooke_c3(n=8, per_side=2, traction_max=2.0)
    model = fem.Model(p)
    F = fem.global_residual(model, np.zeros(p.n_nodes * 2), load=0.5)
    # zero displacement: internal forces vanish, so F = -(external load); total vertical load = -tau * 1 * 0.5
    np.testing.assert_allclose(F[1::2].sum(), 1.0, rtol=1e-14)
    assert abs(F[0::2].sum()) < 1e-14


def test_volume_load_nodal_shares_and_total():
    """Constant volume force f on Q1 elements: each element gives each of its nodes f |e| / 4 on a
    parallelogram, so on the uniform beam mesh an interior node carries f h_x h_y, an edge node half
    and a corner a quarter; on a distorted quad mesh the total is f times the area (sum_a N_a = 1),
    the area taken from the shoelace formula."""
    m, fx = 4, 3.0
    p = I.beam_problem(m, 2, 2, fx)
    hx, hy = 1.0 / m, I.BEAM_LENGTH / (I.BEAM_LENGTH * m)
    model = fem.Model(p)
    F = fem.global_residual(model, np.zeros(p.n_nodes * 2), load=0.5)
    # zero displacement: internal forces vanish, F = -(external load) on the free dofs
    nx = m + 1
    i, j = np.arange(p.n_nodes) % nx, np.arange(p.n_nodes) // nx
    ny = int(round(I.BEAM_LENGTH * m))
    share = np.where((i == 0) | (i == m), 0.5, 1.0) * np.where((j == 0) | (j == ny), 0.5, 1.0)
    free = fem.free_mask(p).reshape(-1, 2)[:, 0]
    np.testing.assert_allclose(F[0::2][free], 0.5 * fx * hx * hy * share[free], rtol=1e-13)
    assert np.all(F[1::2] == 0.0)
    # distorted mesh: total force = f * area
    rng = np.random.default_rng(4)
    X = p.xy[p.conn] + 0.2 * hx * rng.uniform(-1, 1, (p.conn.shape[0], 4, 2))
    f = np.tile([[1.5, -2.0]], (p.conn.shape[0], 1))
    fe = fem.volume_load(X, f).reshape(-1, 4, 2)
    x, y = X[..., 0], X[..., 1]
    area = 0.5 * np.abs(np.sum(x * np.roll(y, -1, axis=1) - np.roll(x, -1, axis=1) * y, axis=1))
    np.testing.assert_allclose(fe.sum(axis=1), area[:, None] * f, rtol=1e-13)
