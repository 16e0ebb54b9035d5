"""Pins of the oracle's learned-guess maps (oracle/guess.py) against facts outside them:
* on a field that is linear in x and y, the side samples are the field at the sample points, and
  the decoded proposal with a zero network output reproduces the field at every local unknown
  (the Coons patch is exact on bilinear data, and the correction vanishes);
* a constant k gives log k in every k feature, f enters times the load factor, and the box size is
  the ring rectangle's in mesh units;
* with k = 1 the smoothing diagonal of an interior node is 4 (the P1 stiffness on this mesh is the
  five-point stencil) and it scales with k;
* a local solution of Eq. 4 is a fixed point of the smoothing, and one sweep from another start
  is the damped Jacobi formula written out with the five-point stencil at small amplitude.
Eq. 2 (Q1, two displacement components):
* on a displacement field linear in x and y, each component's side samples are that component at
  the sample points and the decode with a zero correction reproduces both components at every local
  unknown, also for subdomains whose box is clamped to a Neumann edge of the mesh;
* the feature layout (both components' samples, load factor, box size) and the clamped box;
* the smoothing diagonal in closed form on the uniform mesh: each element adds (lambda + 3 mu) / 3
  (int (dN_a/dx)^2 = int (dN_a/dy)^2 = 1/3 for a bilinear N_a on a square), so 4 (lambda + 3 mu) / 3
  at an interior node, 2 (lambda + 3 mu) / 3 on a free edge, (lambda + 3 mu) / 3 at a free corner;
  and it equals the diagonal of the tangent at zero displacement;
* a local solution is a fixed point of the smoothing, and at small amplitude one sweep is
  w - omega (K_0 w) / d with K_0 the tangent at zero displacement (the law is linear there)."""
import numpy as np

from oracle import decomposition as dec, fem, guess as G, schwarz as S
from paper_2410_24138_gb300 import inputs as I

N = 24


def problem(k=None, f=None):
    return I.diffusion_problem(N, I.brick_partition(N, 2, 3, 7), 6, 2, k_cell=k, f_cell=f)


def test_linear_field_samples_and_exact_decode():
    p = problem()
    a, bx, by = 0.3, -1.2, 0.7
    x = a + bx * p.xy[:, 0] + by * p.xy[:, 1]
    subs, _ = dec.decompose(p)
    h = 1.0 / N
    for sub in subs:
        nodes = sub.vnodes
        i0, i1, j0, j1 = G.ring_box(p, nodes)
        S_ = G.side_samples(p, (i0, i1, j0, j1), x)
        u = np.arange(G.KSIDE) / (G.KSIDE - 1)
        X = (i0 + u * (i1 - i0)) * h
        Y = (j0 + u * (j1 - j0)) * h
        np.testing.assert_allclose(S_[0], a + bx * X + by * j0 * h, rtol=0, atol=1e-14)
        np.testing.assert_allclose(S_[1], a + bx * X + by * j1 * h, rtol=0, atol=1e-14)
        np.testing.assert_allclose(S_[2], a + bx * i0 * h + by * Y, rtol=0, atol=1e-14)
        np.testing.assert_allclose(S_[3], a + bx * i1 * h + by * Y, rtol=0, atol=1e-14)
        w = G.decode(p, nodes, x, np.zeros(G.KGRID * G.KGRID), 1.0)
        np.testing.assert_allclose(w, x[nodes], rtol=0, atol=1e-13)


def test_scalar_features():
    k = np.full(N * N, 3.0)
    f = np.full(N * N, 0.75)
    p = problem(k, f)
    subs, _ = dec.decompose(p)
    for sub in subs:
        nodes = sub.vnodes
        i0, i1, j0, j1 = G.ring_box(p, nodes)
        ft = G.features(p, nodes, np.zeros(p.n_nodes), 0.4)
        assert ft.shape == (G.N_FEATURES,)
        np.testing.assert_allclose(ft[4 * G.KSIDE:4 * G.KSIDE + G.KKS ** 2], np.log(3.0), rtol=0, atol=1e-15)
        assert ft[-3] == 0.4 * 0.75
        np.testing.assert_allclose(ft[-2:], [(i1 - i0) / N, (j1 - j0) / N], rtol=1e-15)


def test_jacobi_diagonal_is_the_five_point_stencil():
    p = problem()
    subs, _ = dec.decompose(p)
    nodes = subs[0].vnodes
    np.testing.assert_allclose(G.jacobi_diagonal(p, nodes), 4.0, rtol=1e-14)
    p2 = problem(k=np.full(N * N, 2.5))
    np.testing.assert_allclose(G.jacobi_diagonal(p2, nodes), 10.0, rtol=1e-14)


def test_smoothing_fixed_point_and_one_sweep():
    p = problem()
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, inner_rtol=0.0, inner_atol=1e-14), with_coarse=False, which=[2])
    lp = sw.locals[0]
    nodes = lp.sub.vnodes
    x = np.zeros(p.n_nodes)
    d = G.jacobi_diagonal(p, nodes)
    wstar, _, st, _, _ = lp.solve_newton(x, x[lp.sub.dofs], sw.opts, 1.0)
    assert st == 0
    np.testing.assert_allclose(G.smooth(lp, x, wstar, 1.0, 6, 0.8, d), wstar, rtol=0, atol=1e-13)
    # one sweep at small amplitude (load 1e-6: 1 + w^2 = 1 to 1e-12) with the five-point stencil
    # h^-2-free form: r_a = 4 w_a - sum of the four neighbours - h^2 f (f = load)
    rng = np.random.default_rng(1)
    w0 = 1e-6 * rng.random(len(nodes))
    load = 1e-6
    w1 = G.smooth(lp, x, w0, load, 1, 0.8, d)
    full = np.zeros(p.n_nodes)
    full[nodes] = w0
    m = N + 1
    r = np.array([4 * full[v] - full[v - 1] - full[v + 1] - full[v - m] - full[v + m] - load / N ** 2 for v in nodes])
    np.testing.assert_allclose(w1, w0 - 0.8 * r / 4.0, rtol=0, atol=1e-17)


def nh_problem(n=16):
    return I.neohooke_problem(n, I.brick_partition(n, 2, 3, 7), 6, 2, 0.0)


def test_displacement_linear_field_samples_and_exact_decode():
    n = 16
    p = nh_problem(n)
    coef = [(0.3, -1.2, 0.7), (-0.1, 0.4, 2.0)]
    X, Y = p.xy[:, 0], p.xy[:, 1]
    x = np.zeros(2 * p.n_nodes)
    for c, (a, bx, by) in enumerate(coef):
        x[c::2] = a + bx * X + by * Y
    subs, _ = dec.decompose(p)
    h = 1.0 / n
    clamped = 0
    for sub in subs:
        nodes = sub.vnodes
        i0, i1, j0, j1 = G.ring_box(p, nodes)
        assert 0 <= i0 < i1 <= n and 0 <= j0 < j1 <= n
        gi, gj = nodes % (n + 1), nodes // (n + 1)
        clamped += (gi.max() == n) + (gj.min() == 0) + (gj.max() == n)
        u = np.arange(G.KSIDE) / (G.KSIDE - 1)
        Xs, Ys = (i0 + u * (i1 - i0)) * h, (j0 + u * (j1 - j0)) * h
        for c, (a, bx, by) in enumerate(coef):
            S_ = G.side_samples(p, (i0, i1, j0, j1), x, c)
            np.testing.assert_allclose(S_[0], a + bx * Xs + by * j0 * h, rtol=0, atol=1e-14)
            np.testing.assert_allclose(S_[1], a + bx * Xs + by * j1 * h, rtol=0, atol=1e-14)
            np.testing.assert_allclose(S_[2], a + bx * i0 * h + by * Ys, rtol=0, atol=1e-14)
            np.testing.assert_allclose(S_[3], a + bx * i1 * h + by * Ys, rtol=0, atol=1e-14)
        w = G.decode(p, nodes, x, np.zeros(2 * G.KGRID * G.KGRID), 1.0)
        np.testing.assert_allclose(w, x[sub.dofs], rtol=0, atol=1e-13)
    assert clamped > 0  # some boxes sit on the free edges


def test_displacement_features_layout():
    n = 16
    p = nh_problem(n)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(2 * p.n_nodes)
    subs, _ = dec.decompose(p)
    for sub in subs:
        box = G.ring_box(p, sub.vnodes)
        ft = G.features(p, sub.vnodes, x, 0.6)
        assert ft.shape == (G.N_FEATURES_DISP,)
        np.testing.assert_array_equal(ft[:4 * G.KSIDE], G.side_samples(p, box, x, 0).ravel())
        np.testing.assert_array_equal(ft[4 * G.KSIDE:8 * G.KSIDE], G.side_samples(p, box, x, 1).ravel())
        assert ft[-3] == 0.6
        np.testing.assert_allclose(ft[-2:], [(box[1] - box[0]) / n, (box[3] - box[2]) / n], rtol=1e-15)


def test_elasticity_diagonal_closed_form_and_tangent():
    n = 16
    p = nh_problem(n)
    mu, lam = fem.lame(p.young, p.poisson)
    unit = (lam + 3 * mu) / 3
    nodes = np.arange(p.n_nodes)
    nodes = nodes[nodes % (n + 1) > 0]  # free nodes (the left edge is clamped)
    d = G.jacobi_diagonal(p, nodes).reshape(-1, 2)
    gi, gj = nodes % (n + 1), nodes // (n + 1)
    nel = (np.where((gi == 0) | (gi == n), 1, 2) * np.where((gj == 0) | (gj == n), 1, 2))
    np.testing.assert_allclose(d, (nel * unit)[:, None] * np.ones((1, 2)), rtol=1e-13)
    K0 = fem.global_jacobian(fem.Model(p), np.zeros(2 * p.n_nodes))
    dofs = (nodes[:, None] * 2 + np.arange(2)).ravel()
    np.testing.assert_allclose(d.ravel(), K0.diagonal()[dofs], rtol=1e-13)


def test_displacement_smoothing_fixed_point_and_one_sweep():
    p = nh_problem()
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL, inner_rtol=0.0, inner_atol=1e-14), with_coarse=False, which=[4])
    lp = sw.locals[0]
    nodes = lp.sub.vnodes
    d = G.jacobi_diagonal(p, nodes)
    rng = np.random.default_rng(2)
    x = np.where(fem.free_mask(p), 1e-3 * rng.standard_normal(2 * p.n_nodes), 0.0)
    wstar, _, st, _, _ = lp.solve_newton(x, x[lp.sub.dofs], sw.opts, 1.0)
    assert st == 0
    np.testing.assert_allclose(G.smooth(lp, x, wstar, 1.0, 6, 0.8, d), wstar, rtol=0, atol=1e-13)
    # small amplitude, no traction: r(w) = K_0 w to O(|w|^2) (relative O(1e-5 |w| n^2) here)
    x0 = np.zeros(2 * p.n_nodes)
    w0 = 1e-10 * rng.standard_normal(lp.sub.n)
    w1 = G.smooth(lp, x0, w0, 0.0, 1, 0.8, d)
    K0 = fem.global_jacobian(fem.Model(p), x0)
    full = np.zeros(2 * p.n_nodes)
    full[lp.sub.dofs] = w0
    r = (K0 @ full)[lp.sub.dofs]
    np.testing.assert_allclose(w1, w0 - 0.8 * r / d, rtol=0, atol=1e-17)
