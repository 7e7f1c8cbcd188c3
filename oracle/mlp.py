"""FP64 reference of the learned surrogate's network (test infrastructure only).

The surrogate is a plain multilayer perceptron: input x (the scene features), hidden layers
h_l = gelu(W_l h_{l-1} + b_l), linear output y = W_L h_{L-1} + b_L, trained on the mean squared
error against target deltas with Adam.  GELU is its tanh form (Hendrycks and Gimpel give it beside
the exact z Phi(z), from which it differs by less than 5e-4):
gelu(z) = z (1 + tanh(sqrt(2 / pi) (z + 0.044715 z^3))) / 2.  Everything here is written directly
from those definitions in float64; only the tests and the benchmark's CPU leg use it.

Parity pins (tests/test_mlp_oracle.py): gradients against central finite differences, the
one-layer case against the closed form of linear least squares, GELU against the exact z Phi(z) of
scipy's normal CDF (within the tanh form's 5e-4), its symmetry gelu(z) - gelu(-z) = z and its
limits, Adam's first step against its closed form (every parameter moves by -lr sign(g)).
"""
from __future__ import annotations

import math

import numpy as np

GELU_K, GELU_C = math.sqrt(2.0 / math.pi), 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    """d gelu / dz = (1 + t) / 2 + z (1 - t^2) k (1 + 3 c z^2) / 2, t = tanh(k (z + c z^3))."""
    t = np.tanh(GELU_K * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_C * z * z)


def init_params(sizes, seed=0):
    """He-style normal weights (std sqrt(2 / fan_in)), zero biases; float64."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        Ws.append(rng.normal(0.0, math.sqrt(2.0 / fi), (fo, fi)))
        bs.append(np.zeros(fo))
    return Ws, bs


def forward(Ws, bs, x):
    """Returns the output and the cache (inputs and pre-activations of every layer)."""
    h = np.asarray(x, np.float64)
    cache = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < len(Ws) - 1 else z
    return h, cache


def mse(y, t):
    """Mean over the batch of the squared error summed over outputs."""
    d = y - t
    return float(np.sum(d * d) / len(d))


def backward(Ws, bs, cache, y, t):
    """Gradients of mse(y, t) with respect to every W and b."""
    n = len(y)
    g = 2.0 * (y - t) / n                     # dL/dy
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        h, z = cache[l]
        if l < len(Ws) - 1:
            g = g * gelu_grad(z)
        dWs[l] = g.T @ h
        dbs[l] = g.sum(0)
        g = g @ Ws[l]
    return dWs, dbs


class Adam:
    """Adam with bias correction (Kingma & Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1 - self.b1) * g
            v *= self.b2
            v += (1 - self.b2) * g * g
            mh = m / (1 - self.b1 ** self.t)
            vh = v / (1 - self.b2 ** self.t)
            p -= self.lr * mh / (np.sqrt(vh) + self.eps)
