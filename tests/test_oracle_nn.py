"""Pins of the oracle's network likelihoods and gradients (CPU only):
central finite differences in float64, the theta = 0 special case, independent
library routines (scipy correlate, log_softmax, numpy inverse) and brute force."""
import numpy as np
import pytest
from scipy.signal import correlate
from scipy.special import log_softmax

from oracle import nn


def _fd_check(spec, theta, X, y, coef, n_coords=None, eps=1e-6, rtol=1e-6, seed=0):
    _, g = nn.loglik_grad(spec, theta, X, y, coef)

    def f(t):
        z, _ = nn.forward(spec, t, X)
        return float(np.sum(coef * nn.per_sample_loglik(spec, z, y)))

    rng = np.random.default_rng(seed)
    idx = range(len(theta)) if n_coords is None else rng.choice(len(theta), n_coords, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (f(tp) - f(tm)) / (2 * eps)
        assert abs(fd - g[i]) <= rtol * max(1.0, abs(fd)) + 1e-7, (i, fd, g[i])


def test_fd_mlp_tanh():
    spec = nn.Spec([("dense", 5, 4), ("dense", 4, 3)], (5,), nn.TANH)
    rng = np.random.default_rng(1)
    X, y = rng.normal(size=(7, 5)), rng.integers(0, 3, 7)
    _fd_check(spec, rng.normal(size=spec.n_params), X, y, rng.uniform(0.5, 2.0, 7))


def test_fd_mlp_relu_three_layers():
    spec = nn.Spec([("dense", 6, 5), ("dense", 5, 4), ("dense", 4, 3)], (6,), nn.RELU)
    rng = np.random.default_rng(2)
    X, y = rng.normal(size=(9, 6)), rng.integers(0, 3, 9)
    _fd_check(spec, rng.normal(size=spec.n_params), X, y, np.full(9, 3.0))


def test_fd_cnn_tanh():
    spec = nn.Spec([("conv", 2, 3, 3), ("pool2",), ("conv", 3, 2, 2), ("dense", 2 * 2 * 2, 4)],
                   (2, 8, 8), nn.TANH)
    rng = np.random.default_rng(3)
    X, y = rng.uniform(size=(3, 2 * 8 * 8)), rng.integers(0, 4, 3)
    _fd_check(spec, rng.normal(size=spec.n_params), X, y, np.ones(3))


def test_fd_gaussian_linear():
    spec = nn.Spec([("dense", 3, 1)], (3,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=0.7)
    rng = np.random.default_rng(4)
    X, y = rng.normal(size=(6, 3)), rng.normal(size=6)
    _fd_check(spec, rng.normal(size=spec.n_params), X, y, np.full(6, 0.3))


def test_zero_weights_give_uniform_loglik():
    # theta = 0 makes every logit 0, so log p = -log(n_classes) exactly.
    spec = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)
    X = np.random.default_rng(5).normal(size=(11, 16))
    z, _ = nn.forward(spec, np.zeros(spec.n_params), X)
    ll = nn.per_sample_loglik(spec, z, np.arange(11) % 4)
    assert np.all(ll == -np.log(4.0))


def test_single_layer_is_logistic_regression():
    spec = nn.Spec([("dense", 4, 3)], (4,), nn.TANH)
    rng = np.random.default_rng(6)
    theta = rng.normal(size=spec.n_params)
    X, y = rng.normal(size=(8, 4)), rng.integers(0, 3, 8)
    W, b = theta[:12].reshape(3, 4), theta[12:]
    expect = log_softmax(X @ W.T + b, axis=1)[np.arange(8), y]
    z, _ = nn.forward(spec, theta, X)
    assert np.allclose(nn.per_sample_loglik(spec, z, y), expect, rtol=1e-14, atol=1e-14)


def test_conv_matches_scipy_correlate():
    spec = nn.Spec([("conv", 3, 2, 5)], (3, 9, 10), nn.TANH)
    rng = np.random.default_rng(7)
    theta = rng.normal(size=spec.n_params)
    x = rng.normal(size=(1, 3 * 9 * 10))
    z, _ = nn.forward(spec, theta, x)
    W, b = theta[:2 * 3 * 25].reshape(2, 3, 5, 5), theta[150:]
    img = x.reshape(3, 9, 10)
    for o in range(2):
        ref = correlate(img, W[o], mode="valid")[0] + b[o]
        assert np.allclose(z.reshape(2, 5, 6)[o], ref, rtol=1e-13, atol=1e-13)


def test_pool_brute_force():
    rng = np.random.default_rng(8)
    a = rng.normal(size=(2, 3, 7, 6))
    out, idx = nn._pool(a)
    assert out.shape == (2, 3, 3, 3)
    for m in range(2):
        for c in range(3):
            for i in range(3):
                for j in range(3):
                    w = [a[m, c, 2 * i, 2 * j], a[m, c, 2 * i, 2 * j + 1],
                         a[m, c, 2 * i + 1, 2 * j], a[m, c, 2 * i + 1, 2 * j + 1]]
                    assert out[m, c, i, j] == max(w)
                    assert idx[m, c, i, j] == w.index(max(w))


def test_linear_gaussian_posterior_matches_numpy_inverse():
    rng = np.random.default_rng(9)
    X, y, c = rng.normal(size=(20, 3)), rng.normal(size=20), rng.uniform(0.1, 2.0, 20)
    mu, sigma = nn.linear_gaussian_posterior(X, y, c, prior_sigma=1.5, noise_sigma=0.4)
    lam = np.eye(3) / 1.5 ** 2 + (X * c[:, None]).T @ X / 0.16
    ref_sigma = np.linalg.inv(lam)
    assert np.allclose(sigma, ref_sigma, rtol=1e-12, atol=1e-14)
    assert np.allclose(mu, ref_sigma @ ((X * c[:, None]).T @ y / 0.16), rtol=1e-12)


def test_gradient_zero_at_closed_form_mode():
    # the gradient of the log posterior vanishes at the closed-form posterior mean
    spec = nn.Spec([("dense", 3, 1)], (3,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=0.5)
    rng = np.random.default_rng(10)
    X, y = rng.normal(size=(30, 3)), rng.normal(size=30)
    mu, _ = nn.linear_gaussian_posterior(X, y, np.ones(30), 1.0, 0.5)
    theta = np.concatenate([mu, [0.0]])          # bias fixed at 0: use the W-part only
    _, g = nn.loglik_grad(spec, theta, X, y, np.ones(30))
    assert np.allclose(g[:3] - mu, 0.0, atol=1e-10)
