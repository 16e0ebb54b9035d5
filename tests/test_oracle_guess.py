"""Pins of the oracle's learned-guess maps (oracle/guess.py) against facts outside them:
* on a field that is linear in x and y, the side samples are the field at the sample points, and
  the decoded proposal with a zero network output reproduces the field at every local unknown
  (the Coons patch is exact on bilinear data, and the correction vanishes);
* a constant k gives log k in every k feature, f enters times the load factor, and the box size is
  the ring rectangle's in mesh units;
* with k = 1 the smoothing diagonal of an interior node is 4 (the P1 stiffness on this mesh is the
  five-point stencil) and it scales with k;
* a local solution of Eq. 4 is a fixed point of the smoothing, and one sweep from another start
  is the damped Jacobi formula written out with the five-point stencil at small amplitude."""
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
