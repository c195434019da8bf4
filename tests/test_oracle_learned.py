"""Pins of the learned-proposal oracle (CPU only): central finite differences
of the network's loss gradient, the zero-output-layer network reducing to the
plain proposal, the features of an identical particle set, and Adam reducing
the loss on a fixed regression problem."""
import math

import numpy as np

from oracle import learned as L


def test_param_count():
    assert L.N_PARAMS == 64 * 8 + 64 + 2 * 64 + 2 == 706


def test_loss_gradient_matches_central_differences():
    r = np.random.default_rng(0)
    p = r.normal(scale=0.3, size=L.N_PARAMS)
    F, T = r.normal(size=(13, 8)), r.normal(size=(13, 2))
    loss, g = L.loss_grad(p, F, T)
    idx = r.choice(L.N_PARAMS, 60, replace=False)
    for i in list(idx) + [L.N_PARAMS - 1, L.N_PARAMS - 3]:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (L.loss_grad(p + e, F, T)[0] - L.loss_grad(p - e, F, T)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), i


def test_zero_output_layer_is_plain_proposal():
    p = np.random.default_rng(1).normal(size=L.N_PARAMS)
    W1, b1, W2, b2 = L.unpack(p)
    p[64 * 8 + 64:] = 0.0
    out, _ = L.forward(p, np.random.default_rng(2).normal(size=(4, 8)))
    inv_mass, h = L.proposal(out, 0.002)
    assert np.all(inv_mass == 1.0) and h == 0.002
    inv_mass, h = L.proposal(np.array([[np.nan, 0.0]]), 0.002)
    assert inv_mass[0] == 1.0 and h == 0.002


def test_features_of_identical_particles():
    J, sizes, isb = 5, [6, 2], [0, 1]
    theta = np.tile(np.array([1.0, 2.0, 2.0, 1.0, 0.0, 3.0, 0.5, 0.5]), (J, 1))
    grad = np.full((J, 8), 2.0)
    wn = np.full(J, 1.0 / J)
    f = L.features(theta, grad, wn, sizes, isb, ess=J, rows_frac=0.25, beta=1.0)
    assert np.allclose(f[0], [math.log(4.0), math.log(19.0 / 6.0), math.log(1e-30), math.log(6) / 10, 0,
                              0.0, 0.25, 1.0], atol=1e-9)
    assert np.allclose(f[1][:2], [math.log(4.0), math.log(0.25)])
    assert f[1][4] == 1.0


def test_adam_reduces_loss():
    r = np.random.default_rng(3)
    F = r.normal(size=(64, 8))
    T = np.stack([np.tanh(F[:, 0]) - 0.5 * F[:, 2], 0.3 * F[:, 1]], axis=1)
    p0 = r.normal(scale=0.2, size=L.N_PARAMS)
    l0, _ = L.loss_grad(p0, F, T)
    p1, l1 = L.adam(p0, F, T, 300, 0.01)
    assert l1 < 0.1 * l0


def test_group_scores():
    th0 = np.zeros((4, 3))
    th1 = np.array([[1.0, 0, 0], [1.0, 1.0, 0], [0, 0, 2.0], [0, 0, 0]])
    wn = np.array([0.25, 0.25, 0.5, 0.0])
    s = L.group_scores(th0, th1, wn, [[0, 1], [2, 3]])
    assert np.allclose(s, [1.5 * (0.25 / 0.125) / 2, 2.0 * (0.25 / 0.25) / 2])


def test_adam_first_two_steps_by_hand():
    """Adam (Kingma & Ba 2015) on a network whose first layer and output
    weights are zero: the hidden units are tanh(0) = 0, the output is b2 and the
    loss gradient is g = b2 - mean(T) for b2 and exactly 0 elsewhere.  With
    mean(T) = (1, -2), b2 = 0, lr = 0.5, beta1 = 0.9, beta2 = 0.999:
      step 1: m = 0.1 g, v = 0.001 g^2, bias-corrected m^ = g, v^ = g^2, so
              b2 = -lr g / (|g| + eps) = (0.5, -0.5) up to eps;
      step 2: g = (-0.5, 1.5), m = 0.09 (-1, 2) + 0.1 g = (-0.14, 0.33),
              v = 0.000999 (1, 4) + 0.001 g^2 = (0.001249, 0.006246),
              m^ = m / 0.19, v^ = v / 0.001999, b2 -= lr m^ / (sqrt(v^) + eps):
              b2 = (0.5 + 0.4660898..., -0.5 - 0.4912875...).
    Every other parameter keeps its (zero) gradient and does not move."""
    F = np.random.default_rng(4).normal(size=(6, 8))
    T = np.tile(np.array([1.0, -2.0]), (6, 1)) + np.array([[0.3, -0.1]]) * np.array([[1], [-1], [1], [-1], [1],
                                                                                      [-1]])
    p0 = np.zeros(L.N_PARAMS)
    p1, _ = L.adam(p0, F, T, 1, 0.5)
    b2 = p1[-2:]
    assert np.allclose(b2, [0.5, -0.5], rtol=1e-7) and np.all(p1[:-2] == 0.0)
    p2, _ = L.adam(p0, F, T, 2, 0.5)
    step2 = np.array([0.46608981940570154, 0.4912875407292165])
    assert np.allclose(p2[-2:], [0.5 + step2[0], -0.5 - step2[1]], rtol=1e-7, atol=1e-12)
    assert np.all(p2[:-2] == 0.0)
