"""The learned initial guess on the GPU, through the C ABI, against the FP64 reference.

* Gradients of the training loss from the GPU kernels against reverse-mode differentiation
  in FP64 (oracle/mlp.py) on the same parameters and batch: FP32 GEMM operands within 1e-4
  relative (per parameter block), BF16 tensor-core operands within 2e-2 (BF16 keeps 8 bits of
  mantissa: each operand carries a relative rounding error up to 2^-9).
* FP32 inference against the FP64 forward pass within 1e-5 relative.
* The acceptance rule: a network with garbage weights must not change the converged solution.
* Training on pairs harvested from the method's own local solves lowers the loss, and the
  trained network reduces the local Newton iterations on held-out coefficient fields.
"""
import numpy as np
import pytest

from oracle import fem, mlp
from paper_2410_24138_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nls():
    from paper_2410_24138_gb300 import build, nls as binding
    build.build()
    return binding


def _blocks(net, flat):
    return [(W.astype(np.float64), b.astype(np.float64)) for W, b in net.split(flat)]


@pytest.mark.parametrize("kind", [0, 1], ids=["scalar", "displacement"])
@pytest.mark.parametrize("bf16,tol", [(False, 1e-4), (True, 2e-2)])
def test_gradient_matches_reference(nls, bf16, tol, kind):
    net = nls.GuessNet(h1=32, h2=48, seed=3, kind=kind)
    assert (net.n_in, net.n_out) == ((nls.GUESS_FEATURES, nls.GUESS_OUTPUTS) if kind == 0 else
                                     (nls.GUESS_FEATURES_DISP, nls.GUESS_OUTPUTS_DISP))
    rng = np.random.default_rng(0)
    B = 24
    X = rng.standard_normal((B, net.n_in)).astype(np.float32)
    T = rng.standard_normal((B, net.n_out)).astype(np.float32)
    g, L = net.gradient(X, T, bf16=bf16)
    params = _blocks(net, net.params())
    Y, cache = mlp.forward(params, X.astype(np.float64))
    ref = mlp.backward(params, cache, Y, T.astype(np.float64))
    got = net.split(g)
    assert abs(L - mlp.loss(Y, T.astype(np.float64))) <= tol * mlp.loss(Y, T.astype(np.float64))
    for (gW, gb), (rW, rb) in zip(got, ref):
        assert np.linalg.norm(gW - rW) <= tol * np.linalg.norm(rW)
        assert np.linalg.norm(gb - rb) <= tol * max(np.linalg.norm(rb), 1e-30)


@pytest.mark.parametrize("kind", [0, 1], ids=["scalar", "displacement"])
def test_inference_matches_reference(nls, kind):
    net = nls.GuessNet(h1=64, h2=32, seed=5, kind=kind)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((10, net.n_in)).astype(np.float32)
    Y = net.forward(X)
    params = _blocks(net, net.params())
    Yr, _ = mlp.forward(params, X.astype(np.float64))
    assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)


def _c4_family(seed, n=128, per=4, fscale=1.0):
    """The log-normal-coefficient diffusion family (Eq. 1 with k(x), f) at n x n cells on per x per
    brick subdomains (about 32 x 32 cells each, as in the 512 x 512 workload), f scaled by fscale."""
    g = I.gaussian_random_field(n, seed, ell=1.0 / 16.0, sigma=1.0)
    f = fscale * (0.5 + 1.5 * I.uniform01(I.splitmix64(seed ^ 0x5DEECE66D), 1)[0])
    return I.diffusion_problem(n, I.brick_partition(n, per, per, I.PARTITION_SEED), per * per, 2,
                               k_cell=np.exp(g), f_cell=np.full(n * n, f))


def test_garbage_network_does_not_change_the_solution(nls):
    p = _c4_family(1001, n=96, per=3)
    ref = nls.make_solver(p, coupling="hybrid")
    u_ref, rep_ref = ref.solve()
    s = nls.make_solver(p, coupling="hybrid")
    net = nls.GuessNet(h1=32, h2=32, seed=9)
    mean, scale, _ = net.normalisation()
    net.set_normalisation(mean, scale, 1e3)  # outputs scaled into nonsense
    nls.attach_guess(s, net, nls.GUESS_USE)
    u, rep = s.solve()
    proposed, accepted = nls.guess_counts(s)
    assert rep.status == 0 and rep.final_residual < 1e-8
    assert proposed > 0 and accepted == 0
    F = fem.global_residual(fem.Model(p), u)
    assert np.linalg.norm(F) < 1e-8
    assert np.linalg.norm(u - u_ref) <= 1e-6 * np.linalg.norm(u_ref)


def test_first_outer_policy_proposes_once_per_load_step(nls):
    """NLS_GUESS_FIRST_OUTER: proposals only at the first outer iteration of each load step; the
    solution is the method's own."""
    p = _c4_family(1001, n=96, per=3)
    ref = nls.make_solver(p, coupling="hybrid")
    u_ref, _ = ref.solve()
    s = nls.make_solver(p, coupling="hybrid")
    net = nls.GuessNet(h1=32, h2=32, seed=9)
    nls.attach_guess(s, net, nls.GUESS_USE | nls.GUESS_FIRST_OUTER)
    u, rep = s.solve()
    proposed, _ = nls.guess_counts(s)
    assert rep.status == 0 and rep.outer_iterations >= 2
    assert proposed == p.n_sub
    assert np.linalg.norm(u - u_ref) <= 1e-6 * np.linalg.norm(u_ref)


def _train(nls, seeds, fscale):
    net = nls.GuessNet(h1=256, h2=256, seed=11, capacity=20000)
    for seed in seeds:
        s = nls.make_solver(_c4_family(seed, fscale=fscale), coupling="hybrid")
        nls.attach_guess(s, net, nls.GUESS_HARVEST)
        _, rep = s.solve()
        assert rep.status == 0
        s.close()
    losses = net.train(steps=2000, batch=128, lr=1e-3, seed=5)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.1 * losses[:50].mean()
    return net


def _steps(nls, net, seeds, fscale):
    plain, guess, acc = 0, 0, 0
    for seed in seeds:
        p = _c4_family(seed, fscale=fscale)
        a = nls.make_solver(p, coupling="hybrid")
        ua, ra = a.solve()
        b = nls.make_solver(p, coupling="hybrid")
        nls.attach_guess(b, net, nls.GUESS_USE)
        ub, rb = b.solve()
        acc += nls.guess_counts(b)[1]
        assert rb.status == 0 and rb.final_residual < 1e-8
        assert np.linalg.norm(ub - ua) <= 1e-6 * np.linalg.norm(ua)
        plain += ra.subdomain_newton_steps
        guess += rb.subdomain_newton_steps
    return plain, guess, acc


def test_trained_guess_gains_local_newton_steps(nls):
    """Harvest -> train -> use on held-out coefficient fields.  With f in [0.5, 2] the local
    problems are nearly linear (u ~ 1e-2, so (1 + u^2) ~ 1) and local Newton needs one or two
    steps from any start; scaling f by 50 makes them strongly nonlinear (u ~ 0.5), the regime
    where a starting point can save steps.  Both are checked: no loss in the first, a strict
    gain in the second, the converged solutions unchanged within the FP32-path bound."""
    net = _train(nls, range(1, 25), 50.0)
    plain, guess, acc = _steps(nls, net, (1001, 1002, 1003), 50.0)
    assert acc > 0
    assert guess < plain
    net1 = _train(nls, range(1, 25), 1.0)
    plain1, guess1, _ = _steps(nls, net1, (1001, 1002), 1.0)
    assert guess1 <= plain1


@pytest.fixture(scope="module")
def guess_case(nls):
    """A 64 x 64 log-normal-k diffusion problem (held-out field seed), 16 uneven subdomains, with
    an attached network (the maps do not depend on its weights)."""
    p = I.diffusion_c4(1001, n=64, per_side=4)
    s = nls.make_solver(p, coupling="one", precision="fp32")
    net = nls.GuessNet(h1=32, h2=32, seed=2)
    nls.attach_guess(s, net, nls.GUESS_USE)
    nls.set_guess_smoothing(s, 6, 0.8)
    rng = np.random.default_rng(11)
    x = np.where(fem.free_mask(p), 0.2 * rng.random(p.n_nodes), 0.0)
    return p, s, net, x


def test_feature_map_matches_oracle(nls, guess_case):
    """Every one of the 391 raw inputs of every subdomain: FP32 storage of FP64 values whose
    interpolation weights are themselves FP32, so within 1e-6 relative (+1e-7 of the field)."""
    from oracle import decomposition as dec, guess as G
    p, s, net, x = guess_case
    F = nls.guess_features(s, x, 0.7)
    subs, _ = dec.decompose(p)
    for i, sub in enumerate(subs):
        ref = G.features(p, sub.vnodes, x, 0.7)
        np.testing.assert_allclose(F[i], ref, rtol=1e-6, atol=1e-7 * np.abs(x).max())


def test_decode_matches_oracle(nls, guess_case):
    """Coons patch of the side samples plus the bilinear 32 x 32 correction at every local unknown,
    in FP64 on both sides from the same FP32 network outputs: 1e-12 of the largest value."""
    from oracle import decomposition as dec, guess as G
    p, s, net, x = guess_case
    Y = np.random.default_rng(3).standard_normal((p.n_sub, nls.GUESS_OUTPUTS)).astype(np.float32)
    tscale = net.normalisation()[2]
    got = nls.guess_decode(s, x, Y, 0.7)
    subs, _ = dec.decompose(p)
    ref = np.concatenate([G.decode(p, sub.vnodes, x, Y[i].astype(np.float64), tscale) for i, sub in enumerate(subs)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_smoothing_matches_oracle(nls, guess_case):
    """Six damped Jacobi sweeps (omega 0.8) of the same starts on both sides, in FP64: only the
    summation order of the local residuals differs (1e-12 of the largest value)."""
    from oracle import guess as G, schwarz as S
    p, s, net, x = guess_case
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL), with_coarse=False)
    rng = np.random.default_rng(5)
    starts = [x[lp.sub.dofs] + 0.05 * rng.standard_normal(lp.sub.n) for lp in sw.locals]
    got = nls.guess_smooth(s, x, np.concatenate(starts), 0.7)
    ref = np.concatenate([G.smooth(lp, x, w0, 0.7, 6, 0.8, G.jacobi_diagonal(p, lp.sub.vnodes))
                          for lp, w0 in zip(sw.locals, starts)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.abs(got - np.concatenate(starts)).max() > 1e-3  # the sweeps did change the starts


# ---- Eq. 2: the displacement kind -------------------------------------------------------------

def _nh_case(n=32, per=3, seed=7, traction=4.0):
    """Q1 Neo-Hooke on n x n cells, per x per bricks, overlap 2 (the right column of bricks reaches
    the traction edge, the top and bottom rows the free edges: their boxes are clamped)."""
    return I.neohooke_problem(n, I.brick_partition(n, per, per, seed), per * per, 2, traction, load_steps=3)


@pytest.fixture(scope="module")
def nh_guess_case(nls):
    p = _nh_case()
    s = nls.make_solver(p, coupling="one", precision="fp32")
    net = nls.GuessNet(h1=32, h2=32, seed=2, kind=nls.GUESS_KIND_DISPLACEMENT)
    nls.attach_guess(s, net, nls.GUESS_USE)
    nls.set_guess_smoothing(s, 6, 0.8)
    # a smooth bending state (det F > 0 everywhere) plus small noise on the free dofs
    X, Y = p.xy[:, 0], p.xy[:, 1]
    x = np.zeros(2 * p.n_nodes)
    x[0::2] = 0.01 * np.sin(np.pi * X) * Y
    x[1::2] = -0.02 * X ** 2
    x += 1e-4 * np.random.default_rng(12).standard_normal(2 * p.n_nodes)
    x = np.where(fem.free_mask(p), x, 0.0)
    return p, s, net, x


def test_displacement_kind_is_checked_against_the_problem(nls):
    from paper_2410_24138_gb300.nls import NLSError
    s = nls.make_solver(_c4_family(1001, n=32, per=2), coupling="one")
    with pytest.raises(NLSError):
        nls.attach_guess(s, nls.GuessNet(h1=16, h2=16, kind=nls.GUESS_KIND_DISPLACEMENT), nls.GUESS_USE)
    t = nls.make_solver(_nh_case(n=16, per=2), coupling="one")
    with pytest.raises(NLSError):
        nls.attach_guess(t, nls.GuessNet(h1=16, h2=16), nls.GUESS_USE)


def test_displacement_feature_map_matches_oracle(nls, nh_guess_case):
    """All 267 raw inputs of every subdomain (both components' side samples, load, box) against
    the oracle: FP32 storage of FP64 values (1e-6 relative, +1e-7 of the field)."""
    from oracle import decomposition as dec, guess as G
    p, s, net, x = nh_guess_case
    F = nls.guess_features(s, x, 0.7)
    assert F.shape == (p.n_sub, nls.GUESS_FEATURES_DISP)
    subs, _ = dec.decompose(p)
    for i, sub in enumerate(subs):
        ref = G.features(p, sub.vnodes, x, 0.7)
        np.testing.assert_allclose(F[i], ref, rtol=1e-6, atol=1e-7 * np.abs(x).max())


def test_displacement_decode_matches_oracle(nls, nh_guess_case):
    """Both components' Coons patches plus their corrections at every local unknown, FP64 on
    both sides from the same FP32 outputs: 1e-12 of the largest value."""
    from oracle import decomposition as dec, guess as G
    p, s, net, x = nh_guess_case
    Y = np.random.default_rng(3).standard_normal((p.n_sub, nls.GUESS_OUTPUTS_DISP)).astype(np.float32)
    tscale = net.normalisation()[2]
    got = nls.guess_decode(s, x, Y, 0.7)
    subs, _ = dec.decompose(p)
    ref = np.concatenate([G.decode(p, sub.vnodes, x, Y[i].astype(np.float64), tscale) for i, sub in enumerate(subs)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_displacement_smoothing_matches_oracle(nls, nh_guess_case):
    """Six damped Jacobi sweeps with the elastic-stiffness diagonal on both sides, FP64: only the
    summation order of the local residuals differs (1e-12 of the largest value)."""
    from oracle import guess as G, schwarz as S
    p, s, net, x = nh_guess_case
    sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL), with_coarse=False)
    rng = np.random.default_rng(5)
    starts = [x[lp.sub.dofs] + 1e-4 * rng.standard_normal(lp.sub.n) for lp in sw.locals]
    got = nls.guess_smooth(s, x, np.concatenate(starts), 0.7)
    ref = np.concatenate([G.smooth(lp, x, w0, 0.7, 6, 0.8, G.jacobi_diagonal(p, lp.sub.vnodes))
                          for lp, w0 in zip(sw.locals, starts)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.abs(got - np.concatenate(starts)).max() > 1e-5  # the sweeps did change the starts


def test_displacement_garbage_network_does_not_change_the_solution(nls):
    p = _nh_case(n=24, per=3)
    ref = nls.make_solver(p, coupling="hybrid")
    u_ref, _ = ref.solve()
    s = nls.make_solver(p, coupling="hybrid")
    net = nls.GuessNet(h1=32, h2=32, seed=9, kind=nls.GUESS_KIND_DISPLACEMENT)
    mean, scale, _ = net.normalisation()
    net.set_normalisation(mean, scale, 1e3)
    nls.attach_guess(s, net, nls.GUESS_USE)
    u, rep = s.solve()
    proposed, accepted = nls.guess_counts(s)
    assert rep.status == 0 and rep.final_residual < 1e-8
    assert proposed > 0 and accepted == 0
    assert np.linalg.norm(u - u_ref) <= 1e-6 * np.linalg.norm(u_ref)


def test_displacement_guess_gains_full_local_newton_steps(nls):
    """Harvest along the load ramp of 24 solves on training partitions (Neo-Hooke, 256^2 Q1, 64
    bricks of ~32^2 cells, as in the 2048^2 workload), train, then propose at the first outer
    iteration of every load step on two held-out partitions in the chosen form (chord steps on
    kept factors from the second outer iteration on): most proposals are taken, the full local
    Newton steps (assembly + factorization) drop, and the converged solutions are the method's own."""
    n, per = 256, 8

    def case(seed):
        return I.neohooke_problem(n, I.brick_partition(n, per, per, seed), per * per, 2, I.NEOHOOKE_TRACTION_MAX, 5)

    net = nls.GuessNet(h1=512, h2=512, seed=11, capacity=24 * per * per * 20, kind=nls.GUESS_KIND_DISPLACEMENT)
    for seed in range(1, 25):
        s = nls.make_solver(case(seed), coupling="hybrid")
        nls.attach_guess(s, net, nls.GUESS_HARVEST)
        _, rep = s.solve()
        assert rep.status == 0
        s.close()
    losses = net.train(steps=6000, batch=256, lr=1e-3, seed=5)
    assert losses[-100:].mean() < 0.2 * losses[:20].mean()
    full_plain = full_guess = taken = offered = 0
    for seed in (101, 102):
        p = case(seed)
        a = nls.make_solver(p, coupling="hybrid")
        ua, ra = a.solve()
        b = nls.make_solver(p, coupling="hybrid")
        nls.attach_guess(b, net, nls.GUESS_USE | nls.GUESS_FIRST_OUTER)
        ub, rb = b.solve()
        pr, ac = nls.guess_counts(b)
        assert rb.status == 0 and rb.final_residual < 1e-8
        assert np.linalg.norm(ub - ua) <= 1e-6 * np.linalg.norm(ua)
        full_plain += ra.subdomain_newton_steps - ra.local_chord_steps
        full_guess += rb.subdomain_newton_steps - rb.local_chord_steps
        taken += ac
        offered += pr
    assert taken > 0.5 * offered
    assert full_guess < full_plain
