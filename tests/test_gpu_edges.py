"""GPU edge cases of the sampler through the C ABI against the FP64 oracle:
one particle, the maximum of 4096 particles, a one-row subset, a data set
shorter than one 128-row tile, and the particle-count bounds."""
import numpy as np
import pytest

import synthetic
from oracle import nn

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)
MLP1 = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.RELU)


def _eval_parity(ctx, orc, J, D, tol, picks=None):
    lp, g, la, lb = S.smc_eval(ctx, J, D)
    if picks is None:
        rlp, rg, rla, _ = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=tol) and np.allclose(la, rla, rtol=tol)
        for j in range(J):
            assert rel_err(g[j], rg[j]) < tol, j
        return
    for j in picks:
        rlp, rgg, rla, _ = orc.target(orc.theta[j])
        assert abs(lp[j] - rlp) <= tol * abs(rlp), j
        assert abs(la[j] - rla) <= tol * abs(rla), j
        assert rel_err(g[j], rgg + orc.theta[j] / orc.sigma ** 2) < tol, j


@pytest.mark.parametrize("precision", [S.PREC_FP32, S.PREC_BF16])
def test_single_particle_steps(precision):
    """J = 1: the weight is always 1 (ESS = 1 is not below J / 2), so there is
    no resampling; evaluation and a teacher-forced move against the oracle."""
    if precision == S.PREC_FP32:
        spec, (X, y), h, tol = MLP0, synthetic.gaussian_mixture(300, d=16, n_classes=4, seed=71), 0.02, 1e-5
    else:
        spec, (X, y), h, tol = MLP1, synthetic.template_images(300, seed=71), 0.002, 2e-2
    ctx, orc, _ = make_pair(spec, X, y, 1, seed=71, precision=precision)
    try:
        th0 = synthetic.particles(1, spec.n_params, 71, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 100, 100, 5))
        orc.set_schedule("linear", 100, 100, 5, th0)
        _eval_parity(ctx, orc, 1, spec.n_params, tol)
        for k in range(1, 3):
            S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert not S.smc_resample(ctx)
            z = synthetic.normals((1, spec.n_params), 710 + k)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, h, 2)
            orc.step(h, 2, z)
            assert st["ess"] == 1.0
        th, lw, lp = S.smc_get_state(ctx, 1, spec.n_params)
        assert rel_err(th[0], orc.theta[0]) < tol
        assert abs(lp[0] - orc.logpi[0]) <= tol * abs(orc.logpi[0])
    finally:
        S.smc_destroy(ctx)


def test_maximum_particle_count_bf16():
    """J = 4096 (the library's maximum): 2048 particle pairs in the fused
    kernel; evaluation on sampled particles against the oracle, then one move
    with finite weights and an ESS in [1, J]."""
    J = 4096
    X, y = synthetic.template_images(300, seed=72)
    ctx, orc, _ = make_pair(MLP1, X, y, J, seed=72, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, MLP1.n_params, 72, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", 300, 300, 5))
        orc.set_schedule("fb", 300, 300, 5, th0)
        _eval_parity(ctx, orc, J, MLP1.n_params, 2e-2, picks=[0, 1, 2047, 2048, J - 1])
        S.smc_anneal_next(ctx)
        st = S.smc_step(ctx, 0.002, 2)
        _, lw, _ = S.smc_get_state(ctx, J, MLP1.n_params, theta=False)
        assert np.all(np.isfinite(lw)) and 1.0 <= st["ess"] <= J
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("precision", [S.PREC_FP32, S.PREC_BF16])
def test_one_row_subset(precision):
    """Constant schedule with C = 1: the target holds one row (coefficient N)."""
    spec, (X, y) = (MLP0, synthetic.gaussian_mixture(64, d=16, n_classes=4, seed=73)) if precision == S.PREC_FP32 \
        else (MLP1, synthetic.template_images(64, seed=73))
    J = 3
    ctx, orc, _ = make_pair(spec, X, y, J, seed=73, precision=precision)
    try:
        th0 = synthetic.particles(J, spec.n_params, 73, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant", 1, 1, 5))
        orc.set_schedule("constant", 1, 1, 5, th0)
        assert orc.subset_rows == 1
        _eval_parity(ctx, orc, J, spec.n_params, 1e-5 if precision == S.PREC_FP32 else 2e-2)
    finally:
        S.smc_destroy(ctx)


def test_data_shorter_than_one_tile_bf16():
    """N = 37 rows (less than one 128-row tile, odd) on the BF16 engine, J = 5
    (an unpaired last particle): full-batch evaluation against the oracle,
    every parameter block.  The hidden layer is tanh: with ReLU and so few
    rows, one pre-activation within BF16 rounding of zero flips its mask and
    moves a whole row's share (1/37) of that unit's gradient, which tests the
    kink rather than the kernels."""
    spec = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.TANH)
    X, y = synthetic.template_images(37, seed=74)
    J = 5
    ctx, orc, _ = make_pair(spec, X, y, J, seed=74, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, spec.n_params, 74, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", 37, 37, 5))
        orc.set_schedule("fb", 37, 37, 5, th0)
        _eval_parity(ctx, orc, J, spec.n_params, 2e-2)
        _, g, _, _ = S.smc_eval(ctx, J, spec.n_params)
        _, rg, _, _ = oracle_eval(orc)
        for j in range(J):
            off = 0
            for n in (100 * 784, 100, 10 * 100, 10):
                assert rel_err(g[j, off:off + n], rg[j, off:off + n]) < 2e-2, (j, n)
                off += n
    finally:
        S.smc_destroy(ctx)


def test_particle_count_bounds():
    X, y = synthetic.gaussian_mixture(64, d=16, n_classes=4, seed=75)
    for J in (0, 4097):
        with pytest.raises(S.SMCError) as e:
            make_pair(MLP0, X, y, J, seed=75)
        assert e.value.status == 1
