"""GPU tests of the torch.autograd.Function around the library's adjoint
(`paper_2601_21983_gb300.autograd.log_target`): its value and gradient
against smc_eval and the FP64 oracle (FP32 engine 1e-5, BF16 engine 2e-2),
the chain rule through an upstream weighting, central finite differences of
the function's own forward pass, and the 784-400-400-10 network at J = 1024
(the scale configuration) on sampled particles."""
import numpy as np
import pytest

import synthetic
from oracle import nn

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from paper_2601_21983_gb300.autograd import log_target  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)
MLP1 = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.RELU)
MLP4 = nn.Spec([("dense", 784, 400), ("dense", 400, 400), ("dense", 400, 10)], (784,), nn.RELU)


def _grad(ctx, th0, weights=None):
    theta = torch.from_numpy(th0).cuda().requires_grad_(True)
    lp = log_target(ctx, theta)
    loss = lp.sum() if weights is None else (lp * torch.from_numpy(weights).cuda()).sum()
    (g,) = torch.autograd.grad(loss, theta)
    torch.cuda.synchronize()
    return lp.detach().cpu().numpy(), g.cpu().numpy()


def test_fp32_log_target_matches_eval_and_oracle():
    X, y = synthetic.gaussian_mixture(512, d=16, n_classes=4, seed=51)
    J = 8
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=51)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 51, std=0.3)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 200, 200, 10))
        orc.set_schedule("linear", 200, 200, 10, th0)
        lp, g = _grad(ctx, th0)
        elp, egll, _, _ = S.smc_eval(ctx, J, MLP0.n_params)
        assert np.array_equal(lp, elp)
        assert np.allclose(g, egll - th0, rtol=1e-6, atol=1e-6)
        rlp, rg, _, _ = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=1e-5)
        for j in range(J):
            assert rel_err(g[j], rg[j] - th0[j]) < 1e-5, j
    finally:
        S.smc_destroy(ctx)


def test_chain_rule_and_finite_differences():
    """d/dtheta sum_j w_j log pi(theta_j) = w_j grad log pi(theta_j); central
    differences of the function's forward pass agree with its gradient."""
    X, y = synthetic.gaussian_mixture(256, d=16, n_classes=4, seed=52)
    J = 4
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=52)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 52, std=0.3)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", 256, 256, 5))
        w = np.array([0.5, -1.0, 2.0, 0.0])
        _, g1 = _grad(ctx, th0)
        _, gw = _grad(ctx, th0, w)
        assert np.allclose(gw, w[:, None] * g1, rtol=1e-6, atol=1e-6)
        r = np.random.default_rng(52)
        eps = 1e-2
        errs = []
        for _ in range(24):
            i = int(r.integers(MLP0.n_params))
            vals = []
            for sgn in (1.0, -1.0):
                th = th0.copy()
                th[:, i] += sgn * eps          # every particle at the same coordinate
                with torch.no_grad():
                    vals.append(log_target(ctx, torch.from_numpy(th).cuda()).cpu().numpy())
            fd = (vals[0] - vals[1]) / (2 * eps)
            errs.extend(np.abs(fd - g1[:, i]) / np.maximum(1.0, np.abs(fd)))
        assert np.median(errs) < 2e-3 and np.max(errs) < 2e-2
    finally:
        S.smc_destroy(ctx)


def test_bf16_log_target_against_oracle():
    X, y = synthetic.template_images(700, seed=53)
    J = 4
    ctx, orc, _ = make_pair(MLP1, X, y, J, seed=53, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, MLP1.n_params, 53, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 256, 256, 10))
        orc.set_schedule("linear", 256, 256, 10, th0)
        lp, g = _grad(ctx, th0)
        rlp, rg, _, _ = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=2e-2)
        for j in range(J):
            assert rel_err(g[j], rg[j] - th0[j]) < 2e-2, j
    finally:
        S.smc_destroy(ctx)


def test_scale_config_J1024_sampled_particles():
    """MLP 784-400-400-10 ReLU (D = 478,410) with J = 1024 particles on 1024
    rows of the MNIST-shaped data (FP32 engine, sample chunks of 256 rows):
    the gradient of log pi through the autograd function against the FP64
    oracle on three sampled particles, and central differences on 64 random
    coordinates of each of those particles."""
    N, J = 1024, 1024
    X, y = synthetic.template_images(N, seed=54)
    ctx, orc, _ = make_pair(MLP4, X, y, J, seed=54, chunk=256)
    try:
        D = MLP4.n_params
        th0 = synthetic.particles(J, D, 54, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        lp, g = _grad(ctx, th0)
        assert np.all(np.isfinite(lp)) and np.all(np.isfinite(g))
        picks = [0, 517, J - 1]
        for j in picks:
            ll, gg = nn.loglik_grad(MLP4, th0[j].astype(np.float64), orc.X, orc.y, 1.0)
            rlp = ll.sum() - 0.5 * float(th0[j].astype(np.float64) @ th0[j])
            assert abs(lp[j] - rlp) <= 1e-5 * abs(rlp), j
            assert rel_err(g[j], gg - th0[j]) < 1e-5, j
        r = np.random.default_rng(54)
        eps = 1e-2
        coords = {j: r.choice(D, 64, replace=False) for j in picks}
        errs = []
        for t in range(64):
            vals = []
            for sgn in (1.0, -1.0):
                th = th0.copy()
                for j in picks:
                    th[j, coords[j][t]] += sgn * eps
                with torch.no_grad():
                    vals.append(log_target(ctx, torch.from_numpy(th).cuda()).cpu().numpy())
            for j in picks:
                fd = (vals[0][j] - vals[1][j]) / (2 * eps)
                errs.append(abs(fd - g[j, coords[j][t]]) / max(1.0, abs(fd)))
        # a ReLU kink inside +-eps spoils single coordinates: bound the quantiles
        assert np.median(errs) < 1e-2 and np.percentile(errs, 90) < 0.05
    finally:
        S.smc_destroy(ctx)
