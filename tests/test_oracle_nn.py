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


# ---- per-channel batchnorm layer (Sec. 4's convolution-batchnorm blocks, in
# their inference form: z = gamma_c a + beta_c)

BN_SPEC = [("conv", 2, 3, 3), ("bnorm", 3), ("pool2",), ("conv", 3, 4, 2), ("bnorm", 4), ("dense", 4 * 2 * 2, 5),
           ("bnorm", 5), ("dense", 5, 3)]


def test_fd_batchnorm_cnn():
    spec = nn.Spec(BN_SPEC, (2, 8, 8), nn.TANH)
    rng = np.random.default_rng(11)
    X, y = rng.uniform(size=(4, 2 * 8 * 8)), rng.integers(0, 3, 4)
    _fd_check(spec, rng.normal(size=spec.n_params), X, y, rng.uniform(0.5, 2.0, 4))


def _fold(spec_bn, theta):
    """The same network without its bnorm layers: each bnorm folded into the
    layer before it (W' = gamma W, b' = gamma b + beta, gamma per output channel)."""
    P = spec_bn.unpack(theta)
    layers, flat = [], []
    for li, layer in enumerate(spec_bn.layers):
        if layer[0] == "bnorm":
            continue
        if layer[0] == "pool2":
            layers.append(layer)
            continue
        W, b = P[li]
        if li + 1 < len(spec_bn.layers) and spec_bn.layers[li + 1][0] == "bnorm":
            g, beta = P[li + 1]
            W = W * g.reshape((-1,) + (1,) * (W.ndim - 1))
            b = g * b + beta
        layers.append(layer)
        flat += [W.ravel(), b.ravel()]
    return layers, np.concatenate(flat)


def test_batchnorm_folds_into_the_layer_before():
    # forward: a bnorm network equals the bnorm-free network with folded parameters
    # (this pins where the activation goes: after the bnorm, not after the conv)
    spec = nn.Spec(BN_SPEC, (2, 8, 8), nn.TANH)
    rng = np.random.default_rng(12)
    X, y = rng.uniform(size=(5, 2 * 8 * 8)), rng.integers(0, 3, 5)
    theta = rng.normal(size=spec.n_params)
    layers, theta_f = _fold(spec, theta)
    spec_f = nn.Spec(layers, (2, 8, 8), nn.TANH)
    z, _ = nn.forward(spec, theta, X)
    zf, _ = nn.forward(spec_f, theta_f, X)
    np.testing.assert_allclose(z, zf, rtol=1e-12, atol=1e-12)
    # backward, by the chain rule through the fold: dL/dW = gamma dL/dW',
    # dL/db = gamma dL/db', dL/dbeta = dL/db', dL/dgamma = <dL/dW', W> + dL/db' b
    coef = rng.uniform(0.5, 2.0, 5)
    _, g = nn.loglik_grad(spec, theta, X, y, coef)
    _, gf = nn.loglik_grad(spec_f, theta_f, X, y, coef)
    Gf = spec_f.unpack(gf)
    P, G = spec.unpack(theta), spec.unpack(g)
    fi = 0
    for li, layer in enumerate(spec.layers):
        if layer[0] in ("bnorm", "pool2"):
            if layer[0] == "pool2":
                fi += 1
            continue
        dWf, dbf = Gf[fi]
        fi += 1
        W, b = P[li]
        if li + 1 < len(spec.layers) and spec.layers[li + 1][0] == "bnorm":
            gam, _ = P[li + 1]
            cshape = (-1,) + (1,) * (W.ndim - 1)
            np.testing.assert_allclose(G[li][0], gam.reshape(cshape) * dWf, rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(G[li][1], gam * dbf, rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(G[li + 1][1], dbf, rtol=1e-10, atol=1e-12)
            dgam = (dWf * W).reshape(W.shape[0], -1).sum(axis=1) + dbf * b
            np.testing.assert_allclose(G[li + 1][0], dgam, rtol=1e-10, atol=1e-12)
        else:
            np.testing.assert_allclose(G[li][0], dWf, rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(G[li][1], dbf, rtol=1e-10, atol=1e-12)


def test_unit_batchnorm_is_the_network_without_it():
    # gamma = 1, beta = 0: the layer is the identity and the activation moves past it
    spec = nn.Spec(BN_SPEC, (2, 8, 8), nn.TANH)
    layers = [l for l in BN_SPEC if l[0] != "bnorm"]
    spec_f = nn.Spec(layers, (2, 8, 8), nn.TANH)
    rng = np.random.default_rng(13)
    theta_f = rng.normal(size=spec_f.n_params)
    parts, k = [], 0
    for li, layer in enumerate(BN_SPEC):
        if layer[0] == "bnorm":
            parts += [np.ones(layer[1]), np.zeros(layer[1])]
        elif layer[0] != "pool2":
            n = sum(int(np.prod(s)) for s in spec.shapes[li])
            parts.append(theta_f[k:k + n])
            k += n
    theta = np.concatenate(parts)
    X = rng.uniform(size=(3, 2 * 8 * 8))
    np.testing.assert_array_equal(nn.forward(spec, theta, X)[0], nn.forward(spec_f, theta_f, X)[0])


def test_fashion_cnn_parameter_count():
    # Sec. 4's FashionMNIST network: two convolution-batchnorm-pool blocks, two dense
    # layers, D = 96,658 (the layout is this build's reading: 3x3 kernels, 8 and 16
    # channels, 232 hidden units)
    spec = nn.Spec([("conv", 1, 8, 3), ("bnorm", 8), ("pool2",), ("conv", 8, 16, 3), ("bnorm", 16), ("pool2",),
                    ("dense", 16 * 5 * 5, 232), ("dense", 232, 10)], (1, 28, 28), nn.TANH)
    assert spec.n_params == 96658


def test_fd_fashion_cnn_sampled_coordinates():
    # the 96,658-parameter network itself: central differences on coordinates drawn
    # from every parameter block (both batchnorm scales and shifts included)
    spec = nn.Spec([("conv", 1, 8, 3), ("bnorm", 8), ("pool2",), ("conv", 8, 16, 3), ("bnorm", 16), ("pool2",),
                    ("dense", 16 * 5 * 5, 232), ("dense", 232, 10)], (1, 28, 28), nn.TANH)
    rng = np.random.default_rng(14)
    X, y = rng.uniform(size=(3, 784)), rng.integers(0, 10, 3)
    theta = 0.3 * rng.normal(size=spec.n_params)
    _, g = nn.loglik_grad(spec, theta, X, y, np.ones(3))

    def f(t):
        z, _ = nn.forward(spec, t, X)
        return float(np.sum(nn.per_sample_loglik(spec, z, y)))

    off = 0
    for shapes in spec.shapes:
        for s in shapes:
            n = int(np.prod(s))
            for i in rng.choice(n, min(n, 2), replace=False):
                k = off + int(i)
                tp, tm = theta.copy(), theta.copy()
                tp[k] += 1e-6
                tm[k] -= 1e-6
                fd = (f(tp) - f(tm)) / 2e-6
                assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (k, fd, g[k])
            off += n
    assert off == spec.n_params
