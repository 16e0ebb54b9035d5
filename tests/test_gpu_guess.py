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


@pytest.mark.parametrize("bf16,tol", [(False, 1e-4), (True, 2e-2)])
def test_gradient_matches_reference(nls, bf16, tol):
    net = nls.GuessNet(h1=32, h2=48, seed=3)
    rng = np.random.default_rng(0)
    B = 24
    X = rng.standard_normal((B, nls.GUESS_FEATURES)).astype(np.float32)
    T = rng.standard_normal((B, nls.GUESS_OUTPUTS)).astype(np.float32)
    g, L = net.gradient(X, T, bf16=bf16)
    params = _blocks(net, net.params())
    Y, cache = mlp.forward(params, X.astype(np.float64))
    ref = mlp.backward(params, cache, Y, T.astype(np.float64))
    got = net.split(g)
    assert abs(L - mlp.loss(Y, T.astype(np.float64))) <= tol * mlp.loss(Y, T.astype(np.float64))
    for (gW, gb), (rW, rb) in zip(got, ref):
        assert np.linalg.norm(gW - rW) <= tol * np.linalg.norm(rW)
        assert np.linalg.norm(gb - rb) <= tol * max(np.linalg.norm(rb), 1e-30)


def test_inference_matches_reference(nls):
    net = nls.GuessNet(h1=64, h2=32, seed=5)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((10, nls.GUESS_FEATURES)).astype(np.float32)
    Y = net.forward(X)
    params = _blocks(net, net.params())
    Yr, _ = mlp.forward(params, X.astype(np.float64))
    assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)


def _small_c4(seed, n=96, per=3):
    """The log-normal-coefficient diffusion family at 96x96 cells on 3x3 brick subdomains."""
    return I.diffusion_c4(seed, n=n, per_side=per)


def test_garbage_network_does_not_change_the_solution(nls):
    p = _small_c4(1001)
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


def test_harvest_train_and_gain(nls):
    net = nls.GuessNet(h1=128, h2=128, seed=11, capacity=4000)
    for seed in range(1, 13):
        s = nls.make_solver(_small_c4(seed), coupling="hybrid")
        nls.attach_guess(s, net, nls.GUESS_HARVEST)
        _, rep = s.solve()
        assert rep.status == 0
        s.close()
    assert net.pairs() > 100
    losses = net.train(steps=600, batch=64, lr=2e-3, seed=5)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.5 * losses[:50].mean()
    steps_plain, steps_guess, acc = 0, 0, 0
    for seed in (1001, 1002, 1003):
        p = _small_c4(seed)
        a = nls.make_solver(p, coupling="hybrid")
        _, ra = a.solve()
        b = nls.make_solver(p, coupling="hybrid")
        nls.attach_guess(b, net, nls.GUESS_USE)
        ub, rb = b.solve()
        _, accepted = nls.guess_counts(b)
        acc += accepted
        assert rb.status == 0 and rb.final_residual < 1e-8
        steps_plain += ra.subdomain_newton_steps
        steps_guess += rb.subdomain_newton_steps
    assert acc > 0
    assert steps_guess <= steps_plain
