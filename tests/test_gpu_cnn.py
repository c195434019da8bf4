"""GPU parity of the BF16 tensor-core engine for the CIFAR-shaped CNN (conv5x5
3->16, tanh, pool, conv5x5 16->32, tanh, pool, fc 800->10; the convolutions
and weight gradients on tcgen05) against the FP64 oracle, through the C ABI, on
the same seeded inputs.  Tolerance 2e-2 relative on log-likelihoods and on
whole gradients (norm-wise per particle), and on the dense layer's blocks,
which no pooling separates from the logits.  The convolution blocks sit behind
max-pool kinks: on these smooth images neighbouring conv outputs are often
within BF16 rounding of each other, so the kernel's BF16 argmax and the
oracle's FP64 argmax can pick different positions and route a window's
gradient through a different input patch (as a ReLU mask flips at BF16
rounding of 0 in the dense tests); and their weight gradients are sums over
hundreds of positions per image whose terms largely cancel, which magnifies
the BF16 rounding of dZ and of the inputs (2-3% on the conv-1 weights here,
about 3% on white-noise images, where argmax decisions rarely differ).  Those
blocks are bounded at 5e-2.  The
whole gradient's bound follows from the blocks' bounds: with e_b <= t_b for
every block b, the norm-wise error of the whole is at most
sqrt(sum_b t_b^2 |g_b|^2) / |g|, which is 2e-2 when the dense blocks carry the
norm and approaches 5e-2 when the convolution blocks do (1-channel images).

The engine rounds images and particles to BF16 on entry; about a third of
the convolution blocks' error above is that rounding.  The evaluation check
of the configuration's network therefore also runs on images and particles
that are BF16 values already (the same arrays for both sides), and there
every block, the convolution blocks included, is held to 2e-2 (measured
1.2-1.6%).  With one input channel or a handful of images the cancellation
alone leaves the convolution blocks at 2-3% even then, so those checks keep
the bounds above."""
import numpy as np
import pytest

import synthetic
from oracle import nn, smc as osmc

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-2
CNN2 = nn.Spec([("conv", 3, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 800, 10)], (3, 32, 32),
               nn.TANH)
BLOCKS = [(16, 3, 5, 5), (16,), (32, 16, 5, 5), (32,), (10, 800), (10,)]
# a second shape for the implicit conv-2 kernels: 1x28x28 images, a 12 x 12
# pooled grid (tap shifts ky 12 + kx up to 52), 4 x 4 x 32 = 512 features
CNN28 = nn.Spec([("conv", 1, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 512, 10)], (1, 28, 28),
                nn.TANH)
BLOCKS28 = [(16, 1, 5, 5), (16,), (32, 16, 5, 5), (32,), (10, 512), (10,)]


def _bf16(a):
    """a rounded to the nearest BF16 value (ties to even), kept in float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def _per_particle_rel(a, b):
    return max(rel_err(a[j], b[j]) for j in range(a.shape[0]))


BLOCK_TOL = [5e-2, 5e-2, 5e-2, 5e-2, TOL, TOL]   # conv W1, b1, W2, b2 (behind pooling), dense W, b


def _whole_bound(rg, blocks):
    """Per particle: sqrt(sum_b t_b^2 |g_b|^2) / |g| over the oracle's blocks."""
    out = []
    for j in range(rg.shape[0]):
        off, acc = 0, 0.0
        for shp, t in zip(blocks, BLOCK_TOL):
            n = int(np.prod(shp))
            acc += t * t * float(np.sum(rg[j, off:off + n] ** 2))
            off += n
        out.append(np.sqrt(acc / float(np.sum(rg[j] ** 2))))
    return np.array(out)


def _check_eval(ctx, orc, J, spec=CNN2, blocks=BLOCKS, exact_inputs=False):
    lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
    rlp, rg, rla, rlb = oracle_eval(orc)
    scale = np.abs(rla) + np.abs(rlb)
    assert np.all(np.abs(la - rla) <= TOL * scale + 1e-6)
    assert np.all(np.abs(lb - rlb) <= TOL * scale + 1e-6)
    assert np.allclose(lp, rlp, rtol=TOL)
    off, errs = 0, []
    for shp in blocks:
        n = int(np.prod(shp))
        errs.append(_per_particle_rel(g[:, off:off + n], rg[:, off:off + n]))
        off += n
    bound = np.full(J, TOL) if exact_inputs else np.maximum(_whole_bound(rg, blocks), TOL)
    whole = np.array([rel_err(g[j], rg[j]) for j in range(J)])
    print("block errors", [f"{e:.2e}" for e in errs], "whole", f"{whole.max():.2e}", "bound", f"{bound.min():.2e}")
    for shp, e, tol in zip(blocks, errs, [TOL] * len(blocks) if exact_inputs else BLOCK_TOL):
        assert e < tol, (shp, e)
    assert np.all(whole < bound), (whole, bound)
    return lp, g


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("chunk", [0, 40])
def test_bf16_cnn_eval_parity(chunk, exact):
    """log pi, region sums and the gradient of every parameter block at prior-
    scale particles, whole subset and in chunks of 40 images (ragged tail);
    exact: images and particles that are BF16 values."""
    N, J = 96, 4
    X, y = synthetic.smooth_field_images(N, seed=71)
    X = _bf16(X) if exact else X
    ctx, orc, _ = make_pair(CNN2, X, y, J, seed=71, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, CNN2.n_params, 71, std=0.1)
        th0 = _bf16(th0) if exact else th0
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 48, 48, 10))
        orc.set_schedule("linear", 48, 48, 10, th0)
        _check_eval(ctx, orc, J, exact_inputs=exact)
        S.smc_anneal_next(ctx)
        orc.anneal_next()
        _check_eval(ctx, orc, J, exact_inputs=exact)
    finally:
        S.smc_destroy(ctx)


def test_bf16_cnn_second_shape_parity():
    """The same engine on 1x28x28 images (a 12 x 12 pooled grid instead of
    14 x 14, so other tap shifts, window sizes and tile-to-image alignments in
    the implicit conv-2 kernels; 512 features into the head), 5 particles,
    chunks of 36 images (a ragged tail of 8), before and after one tempering
    step."""
    N, J = 80, 5
    X, y = synthetic.smooth_field_images(N, seed=74, side=28, channels=1)
    ctx, orc, _ = make_pair(CNN28, X, y, J, seed=74, precision=S.PREC_BF16, chunk=36)
    try:
        th0 = synthetic.particles(J, CNN28.n_params, 74, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 40, 40, 10))
        orc.set_schedule("linear", 40, 40, 10, th0)
        _check_eval(ctx, orc, J, CNN28, BLOCKS28)
        S.smc_anneal_next(ctx)
        orc.anneal_next()
        _check_eval(ctx, orc, J, CNN28, BLOCKS28)
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("J,N,chunk", [(1, 3, 2), (2, 1, 0), (7, 5, 1)])
def test_bf16_cnn_tiny_edges(J, N, chunk):
    """Edges of the engine's work split: one particle (J = 1: conv 1's N = 16
    columns, one split unit per tile run), a single image (196 grid rows: two
    128-row tiles, the second mostly past the data), chunks of one image, and
    J = 7 (splits that do not divide the grid evenly)."""
    X, y = synthetic.smooth_field_images(N, seed=76)
    ctx, orc, _ = make_pair(CNN2, X, y, J, seed=76, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, CNN2.n_params, 76, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant", N, N, 10))
        orc.set_schedule("constant", N, N, 10, th0)
        _check_eval(ctx, orc, J)
    finally:
        S.smc_destroy(ctx)


def test_bf16_cnn_sda_parity():
    """SDA (Sec. 3.1) on the CNN: both row regions, teacher-forced from the GPU's
    particles and weights each iteration; region sums, log pi and gradients
    within 2e-2, the temperature update from the GPU's own sums against the
    oracle's rule, subset sizes bit-exact; then the posterior predictive."""
    N, J = 64, 3
    D = CNN2.n_params
    X, y = synthetic.smooth_field_images(N, seed=72)
    ctx, orc, _ = make_pair(CNN2, X, y, J, seed=72, precision=S.PREC_BF16, chunk=24)
    try:
        th0 = synthetic.particles(J, D, 72, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("sda", 16, 16, 20, delta_s=20.0))
        orc.set_schedule("sda", 16, 16, 20, th0, delta_s=20.0)
        both = 0
        for k in range(1, 5):
            th, lw, lp = S.smc_get_state(ctx, J, D)
            wn = S.smc_get_weights(ctx, J)
            orc.theta = th.astype(np.float64)
            _, _, ela, elb = S.smc_eval(ctx, J, D)
            _check_eval(ctx, orc, J)
            both += int(orc.sda.m_full > 0 and orc.sda.block > 0)
            orc.logpi, orc.la, orc.lb = lp.astype(np.float64), ela.astype(np.float64), elb.astype(np.float64)
            orc.logw, orc.wn = lw.astype(np.float64), wn.astype(np.float64)
            orc.ess = osmc.ess(orc.wn)
            info = S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert info["rows"] == orc.subset_rows and info["rows_full"] == orc.sda.m_full, k
            assert info["beta"] == pytest.approx(orc.sda.beta, rel=1e-9, abs=1e-12), k
            S.smc_set_uniforms(ctx, [0.3])
            S.smc_resample(ctx, force=True)
            orc.resample(u=0.3, force=True)
            z = synthetic.normals((J, D), 900 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.005, 1)
            orc.step(0.005, 1, z)
            th2, _, lp2 = S.smc_get_state(ctx, J, D)
            assert _per_particle_rel(th2, orc.theta) < TOL and np.allclose(lp2, orc.logpi, rtol=TOL), k
        assert both >= 1
        Xt, _ = synthetic.smooth_field_images(50, seed=72, test=True)
        probs = np.empty((50, 10), np.float32)
        orc.theta = S.smc_get_state(ctx, J, D)[0].astype(np.float64)
        orc.wn = S.smc_get_weights(ctx, J).astype(np.float64)
        S.smc_posterior_predict(ctx, np.ascontiguousarray(Xt, np.float32), probs)
        ref = orc.predict(Xt.astype(np.float64))
        assert np.max(np.abs(probs - ref)) < TOL
        assert np.allclose(probs.sum(axis=1), 1.0, atol=1e-5)
    finally:
        S.smc_destroy(ctx)


def test_bf16_cnn_full_data_sampled_particles():
    """The configuration's full sizes in the engine's own chunking: J = 128
    particles and all 50000 images resident; a 1000-image subset (two
    mini-batches of 500) evaluated for every particle, checked against the FP64
    oracle on sampled particles (the oracle's convolutions take tens of ms per
    image, so it cannot sum all 50000 rows)."""
    N, J, M = 50000, 128, 1000
    D = CNN2.n_params
    X, y = synthetic.smooth_field_images(N, seed=73)
    ctx, orc, _ = make_pair(CNN2, X, y, J, seed=73, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, D, 73, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant", M, M, 10))
        lp, g, la, lb = S.smc_eval(ctx, J, D)
        assert np.all(np.isfinite(g)) and np.all(lb == 0.0)
        # Constant keeps the first M rows of the annealed order, c_i = N / M
        for j in [0, 127]:
            ll, gg = nn.loglik_grad(CNN2, th0[j].astype(np.float64), orc.X[:M], orc.y[:M], N / M)
            assert abs(la[j] - ll.sum()) <= TOL * abs(ll.sum()), j
            assert rel_err(g[j], gg) < TOL, j
    finally:
        S.smc_destroy(ctx)
