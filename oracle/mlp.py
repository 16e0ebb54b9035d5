"""FP64 reference of the learned initial guess (oracle, CPU; test infrastructure only).

Imported only by the tests, the smoke check and the benchmark's CPU-baseline leg.  The paper
has no learned component; this module defines, in plain numpy, what the GPU training and
inference kernels must compute, so that their gradients can be checked:

* the Coons (bilinear transfinite) patch of boundary data sampled on the four sides of the
  unit square, which the network output corrects;
* a fully connected network x -> GELU(W1 x + b1) -> GELU(W2 . + b2) -> W3 . + b3 with the tanh
  form of GELU, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
* the loss L = 1/(2 B) sum_batch ||y - t||^2 and its gradient by reverse-mode differentiation;
* one Adam step (Kingma and Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

SQRT_2_OVER_PI = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(SQRT_2_OVER_PI * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = SQRT_2_OVER_PI * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    du = SQRT_2_OVER_PI * (1.0 + 3 * 0.044715 * z ** 2)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def init_params(sizes, seed: int):
    """Weights W_l [out, in] ~ N(0, 1/in) from numpy's default generator, biases zero."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        params.append((rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in), np.zeros(fan_out)))
    return params


def forward(params, X):
    """X [B, in] -> (Y [B, out], cache of pre-activations and layer inputs)."""
    cache = []
    a = X
    for li, (W, b) in enumerate(params):
        z = a @ W.T + b
        cache.append((a, z))
        a = gelu(z) if li + 1 < len(params) else z
    return a, cache


def loss(Y, T):
    return 0.5 * np.sum((Y - T) ** 2) / Y.shape[0]


def backward(params, cache, Y, T):
    """Gradients [(dW, db)] of loss(Y, T) through the network."""
    grads = [None] * len(params)
    d = (Y - T) / Y.shape[0]
    for li in range(len(params) - 1, -1, -1):
        a, z = cache[li]
        if li + 1 < len(params):
            d = d * gelu_grad(z)
        W, _ = params[li]
        grads[li] = (d.T @ a, d.sum(axis=0))
        d = d @ W
    return grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = {"t": step count, "m": [...], "v": [...]}."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((W, b), (dW, db)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, dW), (b, db))):
            key = 2 * i + j
            m = state["m"].setdefault(key, np.zeros_like(p))
            v = state["v"].setdefault(key, np.zeros_like(p))
            m[...] = beta1 * m + (1 - beta1) * g
            v[...] = beta2 * v + (1 - beta2) * g * g
            mhat = m / (1 - beta1 ** t)
            vhat = v / (1 - beta2 ** t)
            new.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        out.append(tuple(new))
    return out


def coons(bottom, top, left, right, s, t):
    """Bilinear transfinite interpolation on [0,1]^2 of side data given as callables of one variable.

    bottom(s) = g(s, 0), top(s) = g(s, 1), left(t) = g(0, t), right(t) = g(1, t).
    """
    P00, P10, P01, P11 = bottom(0.0), bottom(1.0), top(0.0), top(1.0)
    return ((1 - t) * bottom(s) + t * top(s) + (1 - s) * left(t) + s * right(t)
            - ((1 - s) * (1 - t) * P00 + s * (1 - t) * P10 + (1 - s) * t * P01 + s * t * P11))
