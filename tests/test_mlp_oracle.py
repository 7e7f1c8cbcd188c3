"""Pins of the FP64 surrogate-network oracle against things other than itself."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_tanh_form():
    """The tanh form of GELU stays within 5e-4 of the exact z Phi(z) (scipy's normal CDF) and
    meets it at the origin and in both tails; gelu(z) - gelu(-z) = z (1 + tanh is odd about 0);
    gelu'(0) = 1/2; the derivative matches central differences."""
    z = np.linspace(-8, 8, 1601)
    exact = z * norm.cdf(z)
    assert np.abs(mlp.gelu(z) - exact).max() < 5e-4
    assert np.abs(mlp.gelu(z) - exact).max() > 1e-4          # it is the tanh form, not the erf one
    assert abs(mlp.gelu(np.array(0.0))) == 0.0
    np.testing.assert_allclose(mlp.gelu(z[-100:]), z[-100:], rtol=1e-12)
    np.testing.assert_allclose(mlp.gelu(z[:100]), 0.0, atol=1e-12)
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=1e-13, atol=1e-14)
    assert mlp.gelu_grad(np.array(0.0)) == pytest.approx(0.5, abs=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h),
                               rtol=1e-7, atol=1e-9)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 9, 6, 5]
    Ws, bs = mlp.init_params(sizes, seed=1)
    bs = [rng.normal(0, 0.1, b.shape) for b in bs]
    x = rng.normal(size=(11, 7))
    t = rng.normal(size=(11, 5))
    y, cache = mlp.forward(Ws, bs, x)
    dWs, dbs = mlp.backward(Ws, bs, cache, y, t)
    h = 1e-6
    for params, grads in ((Ws, dWs), (bs, dbs)):
        for p, g in zip(params, grads):
            for idx in [tuple(rng.integers(0, s) for s in p.shape) for _ in range(6)]:
                old = p[idx]
                p[idx] = old + h
                lp = mlp.mse(mlp.forward(Ws, bs, x)[0], t)
                p[idx] = old - h
                lm = mlp.mse(mlp.forward(Ws, bs, x)[0], t)
                p[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-6 * max(1.0, abs(g[idx]))


def test_single_linear_layer_reaches_least_squares():
    """With no hidden layer the network is linear; gradient descent converges to the normal-
    equation solution of min |X W^T + b - T|^2, which numpy's lstsq computes independently."""
    rng = np.random.default_rng(2)
    X = rng.normal(size=(64, 4))
    T = X @ rng.normal(size=(4, 3)) + rng.normal(size=3) + 0.01 * rng.normal(size=(64, 3))
    Ws, bs = mlp.init_params([4, 3], seed=3)
    opt = mlp.Adam(Ws + bs, lr=0.05)
    for _ in range(3000):
        y, cache = mlp.forward(Ws, bs, X)
        dWs, dbs = mlp.backward(Ws, bs, cache, y, T)
        opt.step(Ws + bs, dWs + dbs)
    A = np.hstack([X, np.ones((64, 1))])
    sol = np.linalg.lstsq(A, T, rcond=None)[0]
    np.testing.assert_allclose(Ws[0].T, sol[:4], atol=1e-4)
    np.testing.assert_allclose(bs[0], sol[4], atol=1e-4)


def test_adam_first_step_moves_by_learning_rate():
    """After one step with bias correction, m_hat = g and v_hat = g^2, so p moves by
    -lr g / (|g| + eps)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    opt = mlp.Adam([p], lr=0.01)
    opt.step([p], [g])
    np.testing.assert_allclose(p, [1.0, -2.0, 0.5] - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
