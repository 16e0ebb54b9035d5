"""Pins of the learned-guess reference (oracle/mlp.py) against facts outside it.

* GELU against its erf definition within the accuracy of the tanh form (below 5e-4 in absolute value) and
  its derivative against central differences.
* Reverse-mode gradients against central finite differences of the loss.
* A single linear layer: the gradient has the closed form (1/B) (W X^T - T^T) X.
* One Adam step from zero moments moves every parameter by lr * sign(g) (bias-corrected).
* The Coons patch reproduces every bilinear function and matches the side data.
"""
import numpy as np
from scipy.special import erf

from oracle import mlp


def test_gelu_matches_erf_definition():
    z = np.linspace(-6, 6, 2001)
    exact = 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 5e-4
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 9, 8, 5]
    params = mlp.init_params(sizes, 1)
    X = rng.standard_normal((6, 7))
    T = rng.standard_normal((6, 5))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (arr, g) in ((W, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.loss(mlp.forward(params, X)[0], T)
                arr[idx] = old - h
                lm = mlp.loss(mlp.forward(params, X)[0], T)
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_single_linear_layer_closed_form():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((3, 4))
    b = rng.standard_normal(3)
    X = rng.standard_normal((5, 4))
    T = rng.standard_normal((5, 3))
    Y, cache = mlp.forward([(W, b)], X)
    (dW, db), = mlp.backward([(W, b)], cache, Y, T)
    R = X @ W.T + b - T
    np.testing.assert_allclose(dW, R.T @ X / 5, rtol=1e-13)
    np.testing.assert_allclose(db, R.sum(axis=0) / 5, rtol=1e-13)


def test_adam_first_step_is_signed_learning_rate():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    state = {"t": 0, "m": {}, "v": {}}
    new = mlp.adam_step(params, grads, state, lr=0.01, eps=0.0)
    np.testing.assert_allclose(new[0][0], [[1.0 - 0.01, -2.0 + 0.01]], rtol=1e-12)
    np.testing.assert_allclose(new[0][1], [0.5 - 0.01], rtol=1e-12)


def test_coons_patch_reproduces_bilinear_and_sides():
    g = lambda s, t: 0.3 + 1.2 * s - 0.7 * t + 2.5 * s * t
    sides = (lambda s: g(s, 0.0), lambda s: g(s, 1.0), lambda t: g(0.0, t), lambda t: g(1.0, t))
    for s, t in [(0.2, 0.7), (0.5, 0.5), (0.9, 0.1)]:
        assert abs(mlp.coons(*sides, s, t) - g(s, t)) < 1e-14
    h = lambda s, t: np.sin(3 * s) * np.cos(2 * t) + s * s
    hs = (lambda s: h(s, 0.0), lambda s: h(s, 1.0), lambda t: h(0.0, t), lambda t: h(1.0, t))
    for s in (0.0, 0.3, 1.0):
        assert abs(mlp.coons(*hs, s, 0.0) - h(s, 0.0)) < 1e-14
        assert abs(mlp.coons(*hs, 0.0, s) - h(0.0, s)) < 1e-14
