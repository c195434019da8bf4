"""GPU parity of the batchnorm layer (Sec. 4's convolution-batchnorm blocks,
read in inference form: a per-channel scale and shift with fixed statistics)
on the FP32 engine, through the C ABI, against the FP64 oracle at the FP32
bar of 1e-5 relative (norm-wise per particle for gradients and parameters)."""
import numpy as np
import pytest

import synthetic
from oracle import nn

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

# Sec. 4's FashionMNIST network (D = 96,658): 3x3 convolutions with 8 and 16
# channels, each followed by batchnorm, the activation and 2x2 max pooling, then
# dense 400 -> 232 -> 10
FASHION = [("conv", 1, 8, 3), ("bnorm", 8), ("pool2",), ("conv", 8, 16, 3), ("bnorm", 16), ("pool2",),
           ("dense", 400, 232), ("dense", 232, 10)]
# small network with a batchnorm after each kind of layer it may follow
SMALL = [("conv", 3, 4, 3), ("bnorm", 4), ("pool2",), ("conv", 4, 6, 3), ("bnorm", 6), ("dense", 24, 8),
         ("bnorm", 8), ("dense", 8, 5)]


def _per_particle_rel(a, b):
    return max(rel_err(a[j], b[j]) for j in range(a.shape[0]))


def _particles(spec, J, seed):
    """Prior-scale draws with the batchnorm scales moved near 1 (gamma = 1 + 0.3 z),
    so every block passes a signal of the usual size."""
    th = synthetic.particles(J, spec.n_params, seed, std=0.1)
    off = 0
    for layer, shapes in zip(spec.layers, spec.shapes):
        n = [int(np.prod(s)) for s in shapes]
        if layer[0] == "bnorm":
            th[:, off:off + n[0]] = 1.0 + 3.0 * th[:, off:off + n[0]]
        off += sum(n)
    return th


@pytest.mark.parametrize("act", [nn.TANH, nn.RELU])
def test_fashion_cnn_eval_parity(act):
    """The 96,658-parameter network on 28x28 10-class images, rows in three
    chunks (the last one ragged): log-likelihood sums, log pi and whole
    gradients against the oracle."""
    spec = nn.Spec(FASHION, (1, 28, 28), act)
    assert spec.n_params == 96658
    N, J = 48, 2
    X, y = synthetic.template_images(N, seed=31)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=31, chunk=20)
    try:
        th0 = _particles(spec, J, 31)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=1e-5)
        assert np.allclose(lp, rlp, rtol=1e-5)
        assert _per_particle_rel(g, rg) < 1e-5
    finally:
        S.smc_destroy(ctx)


def test_bnorm_blocks_of_the_gradient():
    """Each parameter block of a small network with batchnorm after a
    convolution and after a dense layer (gamma and beta blocks included)
    against the oracle, over two chunks."""
    spec = nn.Spec(SMALL, (3, 10, 10), nn.TANH)
    N, J = 40, 4
    X, y = synthetic.smooth_field_images(N, seed=32, side=10, n_classes=5)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=32, chunk=24)
    try:
        th0 = _particles(spec, J, 32)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=1e-5)
        off = 0
        for layer, shapes in zip(spec.layers, spec.shapes):
            for s in shapes:
                n = int(np.prod(s))
                blk = slice(off, off + n)
                assert _per_particle_rel(g[:, blk], rg[:, blk]) < 1e-5, (layer, s)
                off += n
    finally:
        S.smc_destroy(ctx)


def test_bnorm_network_sda_trajectory():
    """Three SDA iterations (anneal, resample, teacher-forced HMC move) of the
    small batchnorm network against the oracle sampler: subset sizes exact,
    temperatures to the FP32 rounding of their increment, particles, log pi
    and log-weights to 1e-5."""
    spec = nn.Spec(SMALL, (3, 10, 10), nn.TANH)
    N, J = 96, 4
    X, y = synthetic.smooth_field_images(N, seed=33, side=10, n_classes=5)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=33, chunk=40)
    try:
        th0 = _particles(spec, J, 33)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("sda", 32, 32, 20, delta_s=20.0))
        orc.set_schedule("sda", 32, 32, 20, th0, delta_s=20.0)
        for k in range(1, 4):
            beta_prev = orc.sda.beta
            info = S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert info["rows"] == orc.subset_rows
            assert abs(info["beta"] - orc.sda.beta) <= 1e-3 * abs(orc.sda.beta - beta_prev) + 1e-12
            S.smc_set_uniforms(ctx, [0.3])
            S.smc_resample(ctx)
            orc.resample(u=0.3)
            z = synthetic.normals((J, spec.n_params), 330 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.005, 3)
            orc.step(0.005, 3, z)
            th, lw, lp = S.smc_get_state(ctx, J, spec.n_params)
            assert _per_particle_rel(th, orc.theta) < 1e-5, k
            assert np.allclose(lp, orc.logpi, rtol=1e-5), k
            assert np.max(np.abs(lw - orc.logw)) <= 1e-5 * np.abs(orc.logpi).max() + 1e-6, k
    finally:
        S.smc_destroy(ctx)


def test_bnorm_model_rules():
    """A batchnorm model is refused by the BF16 engines (SMC_EUNSUPPORTED) and a
    batchnorm that does not follow a dense or conv layer is refused at init
    (SMC_EINVAL)."""
    X, y = synthetic.template_images(16, seed=34)
    model = S.make_model(FASHION, (1, 28, 28), S.ACT_TANH)
    with pytest.raises(S.SMCError) as e:
        S.smc_init(model, X, y_class=y, cfg=S.make_config(2, 1, S.PREC_BF16, stream=torch.cuda.current_stream()))
    assert e.value.status == 7
    bad = S.make_model([("conv", 1, 8, 3), ("pool2",), ("bnorm", 8), ("dense", 8 * 13 * 13, 10)], (1, 28, 28),
                       S.ACT_TANH)
    with pytest.raises(S.SMCError) as e:
        S.smc_init(bad, X, y_class=y, cfg=S.make_config(2, 1, stream=torch.cuda.current_stream()))
    assert e.value.status == 1
