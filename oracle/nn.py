"""Network log-likelihoods and their gradients in float64 (oracle side; test
infrastructure only).

Sec. 2: the target is pi(theta) proportional to p(y_{1:N} | theta) q_0(theta), the
likelihood of a neural network.  Sec. 4 uses 10-class image classification, so
the likelihood of one sample is categorical on the network's logits:
    log p(y_i | theta, x_i) = z_{y_i} - logsumexp(z),  z = NN(x_i; theta).
Sec. 3, eq. approx-grad scales the mini-batch sum by N / M_k; this module only
computes coefficient-weighted sums  sum_i c_i log p(y_i|theta)  and their
gradients; the coefficients are chosen by the sampler (`smc.py`).

A model is a `Spec`: a list of layers
    ("dense", n_in, n_out)      z = a W^T + b,  W [n_out, n_in]
    ("conv", c_in, c_out, k)    valid k x k cross-correlation, stride 1, W [c_out, c_in, k, k]
    ("pool2",)                  2x2 max pool, stride 2 (first maximum wins ties)
    ("bnorm", c)                per-channel scale and shift  z = gamma_c a + beta_c
                                (W = gamma [c], b = beta [c]) on a [c, h, w] map or a
                                [c] vector
An activation follows every parametric layer except the last and except a
layer whose successor is a "bnorm" layer (conv -> bnorm -> activation, the
convolution-batchnorm blocks of Sec. 4's FashionMNIST network).  The parameter
vector of one particle lists, layer by layer, W (row-major) then b.  A dense
layer after a conv/pool layer reads the feature map flattened in (c, h, w) order.

Reading of Sec. 4's batchnorm: batch normalisation in its inference form,
with fixed statistics (mean 0, variance 1), so the layer is the per-channel
affine map above and gamma, beta are parameters of the particle like any
other.  Statistics taken over the evaluated rows would make each row's
log-likelihood depend on the other rows of D_k, while eq. approx-grad scales a
subset's sum of per-row terms by N / M_k as an estimate of the full-data sum,
which needs each term to depend on its own row only.

The Gaussian likelihood log N(y; z, s^2) with one linear layer is the
linear-Gaussian model used to pin the sampler against a closed-form posterior.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

TANH, RELU, IDENTITY = "tanh", "relu", "identity"
CATEGORICAL, GAUSSIAN = "categorical", "gaussian"


@dataclass
class Spec:
    layers: list
    input_shape: tuple
    activation: str = TANH
    likelihood: str = CATEGORICAL
    noise_sigma: float = 1.0          # Gaussian likelihood only
    shapes: list = field(default_factory=list, init=False)

    def __post_init__(self):
        self.shapes = []
        shp = tuple(self.input_shape)
        for layer in self.layers:
            if layer[0] == "dense":
                assert int(np.prod(shp)) == layer[1], (shp, layer)
                self.shapes.append([(layer[2], layer[1]), (layer[2],)])
                shp = (layer[2],)
            elif layer[0] == "conv":
                _, cin, cout, k = layer
                assert shp[0] == cin, (shp, layer)
                self.shapes.append([(cout, cin, k, k), (cout,)])
                shp = (cout, shp[1] - k + 1, shp[2] - k + 1)
            elif layer[0] == "pool2":
                self.shapes.append([])
                shp = (shp[0], shp[1] // 2, shp[2] // 2)
            elif layer[0] == "bnorm":
                assert shp[0] == layer[1], (shp, layer)
                self.shapes.append([(layer[1],), (layer[1],)])
            else:
                raise ValueError(layer)
        self.out_dim = int(np.prod(shp))
        self.n_params = sum(int(np.prod(s)) for ps in self.shapes for s in ps)
        self.last_param = max(i for i, l in enumerate(self.layers) if l[0] != "pool2")

    def activation_of(self, li):
        """Activation applied to layer li's output (parametric layers only)."""
        if li == self.last_param:
            return IDENTITY
        if li + 1 < len(self.layers) and self.layers[li + 1][0] == "bnorm":
            return IDENTITY
        return self.activation

    def unpack(self, theta):
        """Views of (W, b) per layer into a flat parameter vector."""
        out, off = [], 0
        for ps in self.shapes:
            views = []
            for s in ps:
                n = int(np.prod(s))
                views.append(theta[off:off + n].reshape(s))
                off += n
            out.append(views)
        return out


def _act(name, z):
    if name == TANH:
        return np.tanh(z)
    if name == RELU:
        return np.maximum(z, 0.0)
    return z


def _act_grad(name, z):
    if name == TANH:
        return 1.0 - np.tanh(z) ** 2
    if name == RELU:
        return (z > 0.0).astype(z.dtype)
    return np.ones_like(z)


def _conv(a, W, b):
    k = W.shape[-1]
    win = sliding_window_view(a, (k, k), axis=(2, 3))          # [M, cin, Ho, Wo, k, k]
    return np.einsum("mchwij,ocij->mohw", win, W) + b[None, :, None, None]


def _conv_backward(a, W, dz):
    k = W.shape[-1]
    win = sliding_window_view(a, (k, k), axis=(2, 3))
    dW = np.einsum("mohw,mchwij->ocij", dz, win)
    db = dz.sum(axis=(0, 2, 3))
    padded = np.pad(dz, ((0, 0), (0, 0), (k - 1, k - 1), (k - 1, k - 1)))
    dwin = sliding_window_view(padded, (k, k), axis=(2, 3))    # [M, cout, H, W, k, k]
    da = np.einsum("mohwij,ocij->mchw", dwin, W[:, :, ::-1, ::-1])
    return da, dW, db


def _pool(a):
    M, C, H, W = a.shape
    Ho, Wo = H // 2, W // 2
    win = a[:, :, :2 * Ho, :2 * Wo].reshape(M, C, Ho, 2, Wo, 2).transpose(0, 1, 2, 4, 3, 5)
    win = win.reshape(M, C, Ho, Wo, 4)                           # window order: (0,0),(0,1),(1,0),(1,1)
    idx = np.argmax(win, axis=-1)                                # first maximum wins
    return np.take_along_axis(win, idx[..., None], -1)[..., 0], idx


def _pool_backward(dout, idx, in_shape):
    M, C, H, W = in_shape
    Ho, Wo = dout.shape[2], dout.shape[3]
    win = np.zeros((M, C, Ho, Wo, 4))
    np.put_along_axis(win, idx[..., None], dout[..., None], -1)
    win = win.reshape(M, C, Ho, Wo, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(M, C, 2 * Ho, 2 * Wo)
    da = np.zeros(in_shape)
    da[:, :, :2 * Ho, :2 * Wo] = win
    return da


def forward(spec: Spec, theta, X):
    """Logits z[M, out] of one particle and the cache needed by `backward`."""
    theta = np.asarray(theta, dtype=np.float64)
    params = spec.unpack(theta)
    M = X.shape[0]
    a = np.asarray(X, dtype=np.float64).reshape((M,) + tuple(spec.input_shape))
    cache = []
    for li, layer in enumerate(spec.layers):
        if layer[0] == "dense":
            a_in = a.reshape(M, -1)
            W, b = params[li]
            z = a_in @ W.T + b
        elif layer[0] == "conv":
            a_in = a
            W, b = params[li]
            z = _conv(a_in, W, b)
        elif layer[0] == "bnorm":
            a_in = a
            g, b = params[li]
            shape = (1, -1) + (1,) * (a_in.ndim - 2)
            z = g.reshape(shape) * a_in + b.reshape(shape)
        else:
            a_in = a
            z, idx = _pool(a_in)
            cache.append(("pool2", a_in.shape, idx))
            a = z
            continue
        act = spec.activation_of(li)
        cache.append((layer[0], a_in, z, act))
        a = _act(act, z)
    return a.reshape(M, -1), cache


def per_sample_loglik(spec: Spec, z, y):
    """log p(y_i | theta) per sample from the logits."""
    if spec.likelihood == CATEGORICAL:
        zmax = z.max(axis=1, keepdims=True)
        lse = zmax[:, 0] + np.log(np.exp(z - zmax).sum(axis=1))
        return z[np.arange(z.shape[0]), np.asarray(y, dtype=np.int64)] - lse
    s2 = spec.noise_sigma ** 2
    r = np.asarray(y, dtype=np.float64) - z[:, 0]
    return -0.5 * r * r / s2 - 0.5 * np.log(2.0 * np.pi * s2)


def loglik_grad(spec: Spec, theta, X, y, coef):
    """Per-sample log-likelihoods l_i (unweighted) and the gradient of
    sum_i coef_i l_i with respect to theta (one particle).  Backpropagation:
    dl/dz = onehot(y) - softmax(z) (categorical) or (y - z)/s^2 (Gaussian)."""
    z, cache = forward(spec, theta, X)
    ll = per_sample_loglik(spec, z, y)
    coef = np.broadcast_to(np.asarray(coef, dtype=np.float64), ll.shape)
    M = z.shape[0]
    if spec.likelihood == CATEGORICAL:
        p = np.exp(z - z.max(axis=1, keepdims=True))
        p /= p.sum(axis=1, keepdims=True)
        dz = -p
        dz[np.arange(M), np.asarray(y, dtype=np.int64)] += 1.0
    else:
        dz = ((np.asarray(y, dtype=np.float64) - z[:, 0]) / spec.noise_sigma ** 2)[:, None]
    dz = dz * coef[:, None]
    grads = [None] * len(spec.layers)
    da = dz
    for li in range(len(spec.layers) - 1, -1, -1):
        entry = cache[li]
        if entry[0] == "pool2":
            _, in_shape, idx = entry
            da = _pool_backward(da.reshape((M,) + in_shape[1:2] + idx.shape[2:]), idx, in_shape)
            continue
        kind, a_in, z_l, act = entry
        dzl = da.reshape(z_l.shape) * _act_grad(act, z_l)
        W = spec.unpack(np.asarray(theta, dtype=np.float64))[li][0]
        if kind == "dense":
            grads[li] = (dzl.T @ a_in, dzl.sum(axis=0))
            da = dzl @ W
        elif kind == "bnorm":
            axes = (0,) + tuple(range(2, dzl.ndim))
            grads[li] = ((dzl * a_in).sum(axis=axes), dzl.sum(axis=axes))
            da = dzl * W.reshape((1, -1) + (1,) * (dzl.ndim - 2))
        else:
            da, dW, db = _conv_backward(a_in, W, dzl)
            grads[li] = (dW, db)
    flat = np.concatenate([g.ravel() for gl in grads if gl is not None for g in gl])
    return ll, flat


def predictive_probs(spec: Spec, theta, X):
    """softmax(NN(x; theta)) per row (categorical models)."""
    z, _ = forward(spec, theta, X)
    p = np.exp(z - z.max(axis=1, keepdims=True))
    return p / p.sum(axis=1, keepdims=True)


def linear_gaussian_posterior(X, y, coef, prior_sigma: float, noise_sigma: float):
    """Closed-form Gaussian posterior of w for y_i ~ N(x_i . w, s_n^2) with
    prior N(0, s_p^2 I) and per-sample likelihood exponents coef_i (a tempered
    or rescaled likelihood is still Gaussian):
        Lambda = I / s_p^2 + sum_i c_i x_i x_i^T / s_n^2,
        mu = Lambda^{-1} sum_i c_i x_i y_i / s_n^2.
    Returns (mu, Sigma = Lambda^{-1})."""
    X = np.asarray(X, dtype=np.float64)
    c = np.broadcast_to(np.asarray(coef, dtype=np.float64), (X.shape[0],))
    d = X.shape[1]
    lam = np.eye(d) / prior_sigma ** 2 + (X * c[:, None]).T @ X / noise_sigma ** 2
    rhs = (X * c[:, None]).T @ np.asarray(y, dtype=np.float64) / noise_sigma ** 2
    # Cholesky solve written out (no LAPACK call), d is tiny.
    L = np.zeros((d, d))
    for i in range(d):
        for j in range(i + 1):
            s = lam[i, j] - L[i, :j] @ L[j, :j]
            L[i, j] = np.sqrt(s) if i == j else s / L[j, j]
    Linv = np.zeros((d, d))
    for i in range(d):
        Linv[i, i] = 1.0 / L[i, i]
        for j in range(i):
            Linv[i, j] = -(L[i, j:i] @ Linv[j:i, j]) / L[i, i]
    sigma = Linv.T @ Linv
    return sigma @ rhs, sigma
