"""Learned proposal for the leapfrog kernel, float64 (oracle side; test
infrastructure only).

Not in the paper: this generalises the kernel of Sec. 2.1 from M = I to a
diagonal mass that is constant on each parameter segment (the W or b of one
layer), M = diag(1 / inv_mass_s), and scales the step h.  Both are fixed before
the momenta of an iteration are drawn, so the reversed-momentum L-kernel
weight (eq. weight_update_fp with N(.; 0, M)) stays exact.

Per segment s the network sees 8 features
    f = [log mean g^2, log mean theta^2, log mean_e Var_w(theta_e), log(size_s)/10,
         is_bias, log(ESS/J), M_k/N, beta]
where g = grad log pi_k at the current particles, the means run over all
particles and elements of the segment, and Var_w is the weighted
across-particle variance of each element (E_w[theta^2] - E_w[theta]^2, its mean
clipped at 0 before the log).  An 8-64-2 tanh MLP maps f to
(a_s, b_s); the proposal is
    inv_mass_s = exp(clip(a_s, -4, 4)),  h = h_plain * exp(clip(mean_s b_s, -3, 3)).
With a zero output layer the proposal is the plain one (M = I, h = h_plain).

Training data are made by the sampler itself: within one iteration the
particles are split into G groups, group g moving with candidate
(a + sigma eps_g, b + sigma eps'_g) (group 0 unperturbed); each group's score is
its mean squared jump times its weight health ESS_g / n_g, and the best
candidate becomes the regression target of the iteration's features.  The
network is fit by full-batch Adam on the mean squared error.
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT, N_HID, N_OUT = 8, 64, 2
N_PARAMS = N_HID * N_FEAT + N_HID + N_OUT * N_HID + N_OUT
A_CLIP, B_CLIP = 4.0, 3.0
EPS = 1e-30


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_HID * N_FEAT].reshape(N_HID, N_FEAT); o += N_HID * N_FEAT
    b1 = p[o:o + N_HID]; o += N_HID
    W2 = p[o:o + N_OUT * N_HID].reshape(N_OUT, N_HID); o += N_OUT * N_HID
    b2 = p[o:o + N_OUT]
    return W1, b1, W2, b2


def features(theta, grad_logpi, wn, seg_sizes, seg_is_bias, ess, rows_frac, beta):
    """Per-segment features; theta / grad_logpi are [J, D] in canonical order
    (segments consecutive: W then b of each parametric layer)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(grad_logpi, dtype=np.float64)
    wn = np.asarray(wn, dtype=np.float64)
    J = theta.shape[0]
    out = np.zeros((len(seg_sizes), N_FEAT))
    off = 0
    for s, (size, isb) in enumerate(zip(seg_sizes, seg_is_bias)):
        th = theta[:, off:off + size]
        gg = g[:, off:off + size]
        mu = wn @ th
        var = wn @ (th * th) - mu * mu
        out[s] = [math.log(float(np.mean(gg * gg)) + EPS), math.log(float(np.mean(th * th)) + EPS),
                  math.log(max(float(np.mean(var)), 0.0) + EPS), math.log(size) / 10.0, float(isb),
                  math.log(ess / J), rows_frac, beta]
        off += size
    return out


def forward(params, F):
    """Network output [n, 2] and the hidden activations."""
    W1, b1, W2, b2 = unpack(params)
    Hd = np.tanh(np.asarray(F, dtype=np.float64) @ W1.T + b1)
    return Hd @ W2.T + b2, Hd


def loss_grad(params, F, T):
    """Mean squared error L = (1/n) sum_i 0.5 |out_i - T_i|^2 and dL/dparams."""
    F = np.asarray(F, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    W1, b1, W2, b2 = unpack(params)
    out, Hd = forward(params, F)
    n = F.shape[0]
    r = (out - T) / n
    loss = 0.5 * float(np.sum((out - T) ** 2)) / n
    gW2 = r.T @ Hd
    gb2 = r.sum(axis=0)
    dH = (r @ W2) * (1.0 - Hd * Hd)
    gW1 = dH.T @ F
    gb1 = dH.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def proposal(out, h_plain):
    """(inv_mass per segment, h) from the network output (non-finite -> plain)."""
    out = np.asarray(out, dtype=np.float64)
    if not np.all(np.isfinite(out)):
        return np.ones(out.shape[0]), h_plain
    a = np.clip(out[:, 0], -A_CLIP, A_CLIP)
    b = float(np.clip(np.mean(out[:, 1]), -B_CLIP, B_CLIP))
    return np.exp(a), h_plain * math.exp(b)


def adam(params, F, T, epochs, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam on the mean squared error; returns (params, last loss)."""
    p = np.array(params, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    loss = None
    for t in range(1, epochs + 1):
        loss, g = loss_grad(p, F, T)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, loss


def group_scores(theta_old, theta_new, wn, groups):
    """Score of each candidate group: mean squared jump of its particles times
    its weight health ESS_g / n_g with ESS_g = (sum w)^2 / sum w^2."""
    d2 = np.sum((np.asarray(theta_new, np.float64) - np.asarray(theta_old, np.float64)) ** 2, axis=1)
    wn = np.asarray(wn, dtype=np.float64)
    out = []
    for idx in groups:
        w = wn[idx]
        ess_g = (w.sum() ** 2) / max(float(np.sum(w * w)), 1e-300)
        out.append(float(np.mean(d2[idx])) * ess_g / len(idx))
    return np.array(out)
