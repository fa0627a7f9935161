"""Pins of the warm-start network oracle (oracle/mlp.py), independent of its own formulas:
finite differences, the closed-form least-squares gradient of a one-layer network, special
values and the odd-part identity of GELU, the first Adam step, and exact BF16 rounding cases."""
import numpy as np
from scipy.stats import norm

from oracle import mlp as O


def test_gelu_special_values_and_identity():
    z = np.linspace(-6, 6, 101)
    # z Phi(z) with Phi from scipy's normal distribution (another route than erf)
    assert np.allclose(O.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    # gelu(z) - gelu(-z) = z, since Phi(z) + Phi(-z) = 1
    assert np.allclose(O.gelu(z) - O.gelu(-z), z, atol=1e-14)
    assert O.gelu_grad(np.array([0.0]))[0] == 0.5
    h = 1e-6
    assert np.allclose(O.gelu_grad(z), (O.gelu(z + h) - O.gelu(z - h)) / (2 * h), atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 6, 3]
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(3))
    p = rng.normal(0, 0.5, n)
    X = rng.normal(size=(4, 5))
    T = rng.normal(size=(4, 3))
    _, _, g = O.forward_backward(dims, p, X, T)
    h = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (O.forward_backward(dims, p + e, X, T)[1] - O.forward_backward(dims, p - e, X, T)[1]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_one_layer_is_least_squares():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(6, 4))
    T = rng.normal(size=(6, 2))
    W = rng.normal(size=(4, 2))
    b = rng.normal(size=2)
    Y, loss, g = O.forward_backward([4, 2], np.concatenate([W.ravel(), b]), X, T)
    R = X @ W + b - T
    assert np.isclose(loss, np.mean(R ** 2))
    assert np.allclose(g[:8].reshape(4, 2), 2 * X.T @ R / R.size)
    assert np.allclose(g[8:], 2 * R.sum(axis=0) / R.size)


def test_first_adam_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = O.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    # t = 1: m_hat = g, v_hat = g^2, so the step is -lr g / |g|
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-9)


def test_bf16_rounding_cases():
    # exactly representable values survive; 1 + 2^-8 is a tie and rounds to even (1.0);
    # 1 + 3 * 2^-8 is a tie and rounds up to 1 + 2^-6
    vals = np.array([1.0, -2.5, 0.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7])
    out = O.bf16_round(vals)
    assert np.array_equal(out, [1.0, -2.5, 0.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7])
