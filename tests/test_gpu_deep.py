"""GPU parity of the BF16 tensor-core engine for networks with two or more
hidden layers (forward layers and weight gradients on tcgen05 CTA pairs, the
head on mma.sync) against the FP64 oracle, through the C ABI, on the same
seeded inputs.  Tolerance: 2e-2 relative on log-likelihoods and on whole
gradients (norm-wise per particle; per parameter block as well for tanh
networks, whose gradients have no ReLU kinks that BF16 rounding can flip)."""
import numpy as np
import pytest

import synthetic
from oracle import nn, rng, smc as osmc

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-2


def _mlp4(act):
    return nn.Spec([("dense", 784, 400), ("dense", 400, 400), ("dense", 400, 10)], (784,), act)


def _mlp3(act):
    return nn.Spec([("dense", 64, 48), ("dense", 48, 32), ("dense", 32, 16), ("dense", 16, 4)], (64,), act)


def _data(spec, N, seed):
    if spec.input_shape == (784,):
        return synthetic.template_images(N, seed=seed)
    return synthetic.gaussian_mixture(N, d=64, n_classes=4, seed=seed)


def _blocks(spec):
    shapes = []
    for kind, nin, nout in spec.layers:
        shapes += [(nout, nin), (nout,)]
    return shapes


def _per_particle_rel(a, b):
    return max(rel_err(a[j], b[j]) for j in range(a.shape[0]))


def _check_eval(ctx, orc, spec, J, smooth):
    lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
    rlp, rg, rla, rlb = oracle_eval(orc)
    scale = np.abs(rla) + np.abs(rlb)
    assert np.all(np.abs(la - rla) <= TOL * scale + 1e-6)
    assert np.all(np.abs(lb - rlb) <= TOL * scale + 1e-6)
    assert np.allclose(lp, rlp, rtol=TOL)
    assert _per_particle_rel(g, rg) < TOL
    if smooth:
        off = 0
        for shp in _blocks(spec):
            n = int(np.prod(shp))
            assert _per_particle_rel(g[:, off:off + n], rg[:, off:off + n]) < TOL, shp
            off += n
    return lp, g


@pytest.mark.parametrize("which,N,J,chunk,act", [("mlp4", 700, 4, 0, nn.TANH), ("mlp4", 700, 3, 256, nn.RELU),
                                                 ("mlp3", 500, 5, 0, nn.TANH), ("mlp3", 500, 5, 128, nn.RELU)])
def test_bf16_deep_eval_parity(which, N, J, chunk, act):
    """log pi, the two region sums and the log-likelihood gradient of every
    particle, for 784-400-400-10 and a three-hidden-layer 64-48-32-16-4
    network, whole-subset and chunked (ragged last chunk)."""
    spec = _mlp4(act) if which == "mlp4" else _mlp3(act)
    X, y = _data(spec, N, 61)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=61, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, spec.n_params, 61, std=0.05 if which == "mlp4" else 0.3)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 300, 300, 10))
        orc.set_schedule("linear", 300, 300, 10, th0)
        _check_eval(ctx, orc, spec, J, act == nn.TANH)
        # the next target (600 rows, a different coefficient) on the same particles
        S.smc_anneal_next(ctx)
        orc.anneal_next()
        _check_eval(ctx, orc, spec, J, act == nn.TANH)
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("chunk", [0, 128])
def test_bf16_deep_fresh_windows_off_the_8_row_grid(chunk):
    """Fresh mini-batches of 100 rows start at rows 100 k mod N, mostly off the
    8-row boundaries the first-layer weight gradient reads from: the rows
    before the window inside its first chunk must contribute nothing."""
    spec = _mlp4(nn.TANH)
    N, J = 700, 3
    X, y = _data(spec, N, 62)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=62, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, spec.n_params, 62, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant_fresh", 100, 100, 20))
        orc.set_schedule("constant_fresh", 100, 100, 20, th0)
        for k in range(1, 8):
            S.smc_anneal_next(ctx)
            orc.anneal_next()
            if k in (1, 3, 6):        # windows at rows 100, 300 and 600..699 + 0..0
                _check_eval(ctx, orc, spec, J, True)
    finally:
        S.smc_destroy(ctx)


def test_bf16_deep_step_parity_teacher_forced():
    """One HMC move (h = 0.002, S = 3) with injected momenta: particles, log pi
    after the move and log-weights against the oracle."""
    spec = _mlp4(nn.RELU)
    N, J = 640, 4
    X, y = _data(spec, N, 63)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=63, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, spec.n_params, 63, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 128, 128, 10))
        orc.set_schedule("linear", 128, 128, 10, th0)
        S.smc_anneal_next(ctx)
        orc.anneal_next()
        z = synthetic.normals((J, spec.n_params), 64)
        S.smc_set_noise(ctx, z)
        st = S.smc_step(ctx, 0.002, 3)
        orc.step(0.002, 3, z)
        th, lw, lp = S.smc_get_state(ctx, J, spec.n_params)
        assert st["grad_evals"] == 4 and st["rows"] == 256
        assert _per_particle_rel(th, orc.theta) < TOL
        assert np.allclose(lp, orc.logpi, rtol=TOL)
        assert np.max(np.abs(lw - orc.logw)) <= TOL * np.abs(orc.logpi).max()
    finally:
        S.smc_destroy(ctx)


def test_bf16_deep_sda_parity():
    """Smooth data annealing (Sec. 3.1) on 784-400-400-10: both row regions in
    use (coefficient 1 and beta), teacher-forced from the GPU's particles and
    weights each iteration; the region sums, log pi and gradient within 2e-2,
    the temperature update from the GPU's own sums against the oracle's rule."""
    spec = _mlp4(nn.TANH)
    N, J, D = 1024, 4, None
    X, y = _data(spec, N, 65)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=65, precision=S.PREC_BF16)
    D = spec.n_params
    try:
        th0 = synthetic.particles(J, D, 65, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("sda", 256, 256, 40, delta_s=4.0))
        orc.set_schedule("sda", 256, 256, 40, th0, delta_s=4.0)
        both = 0
        for k in range(1, 11):
            th, lw, lp = S.smc_get_state(ctx, J, D)
            wn = S.smc_get_weights(ctx, J)
            orc.theta = th.astype(np.float64)
            _, _, ela, elb = S.smc_eval(ctx, J, D)
            _check_eval(ctx, orc, spec, J, True)
            both += int(orc.sda.m_full > 0 and orc.sda.block > 0)
            orc.logpi, orc.la, orc.lb = lp.astype(np.float64), ela.astype(np.float64), elb.astype(np.float64)
            orc.logw, orc.wn = lw.astype(np.float64), wn.astype(np.float64)
            orc.ess = osmc.ess(orc.wn)
            info = S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert info["rows"] == orc.subset_rows and info["rows_full"] == orc.sda.m_full, k
            assert info["beta"] == pytest.approx(orc.sda.beta, rel=1e-9, abs=1e-12), k
            S.smc_set_uniforms(ctx, [0.5])
            S.smc_resample(ctx, force=True)
            orc.resample(u=0.5, force=True)
            z = synthetic.normals((J, D), 800 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.002, 1)
            orc.step(0.002, 1, z)
        assert both >= 2
    finally:
        S.smc_destroy(ctx)


def test_bf16_deep_predictive_parity():
    spec = _mlp4(nn.RELU)
    N, J = 512, 4
    X, y = _data(spec, N, 66)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=66, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, spec.n_params, 66, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        Xt, _ = synthetic.template_images(300, seed=66, test=True)
        probs = np.empty((300, 10), np.float32)
        S.smc_posterior_predict(ctx, np.ascontiguousarray(Xt), probs)
        ref = orc.predict(Xt.astype(np.float64))
        assert np.max(np.abs(probs - ref)) < TOL
        assert np.allclose(probs.sum(axis=1), 1.0, atol=1e-5)
    finally:
        S.smc_destroy(ctx)


def test_bf16_deep_adjoint_against_finite_differences():
    """The BF16 adjoint against central differences of the exact (FP64) log pi
    on 64 random coordinates per particle (784-400-400-10 ReLU, 2000 rows);
    a ReLU kink inside +-eps spoils single coordinates, so quantiles are bounded."""
    spec = _mlp4(nn.RELU)
    N, J = 2000, 2
    X, y = _data(spec, N, 67)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=67, precision=S.PREC_BF16)
    try:
        D = spec.n_params
        th0 = synthetic.particles(J, D, 67, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        _, g, _, _ = S.smc_eval(ctx, J, D)

        def logpi(theta):
            z, _ = nn.forward(spec, theta, orc.X)
            return float(nn.per_sample_loglik(spec, z, orc.y).sum()) - 0.5 * float(theta @ theta)

        r = np.random.default_rng(67)
        eps = 1e-3
        errs = []
        for j in range(J):
            base = th0[j].astype(np.float64)
            for i in r.choice(D, 64, replace=False):
                tp, tm = base.copy(), base.copy()
                tp[i] += eps
                tm[i] -= eps
                fd = (logpi(tp) - logpi(tm)) / (2 * eps)
                errs.append(abs(fd - (g[j, i] - base[i])) / max(1.0, abs(fd)))
        assert np.median(errs) < TOL and np.percentile(errs, 90) < 0.1, (np.median(errs), np.percentile(errs, 90))
    finally:
        S.smc_destroy(ctx)


def test_bf16_deep_scale_config_full_size_sampled_particles():
    """The scale configuration at full size in the engine's own chunking: MLP
    784-400-400-10 ReLU (D = 478,410), J = 1024 particles, all 60000 rows of
    the MNIST-shaped stand-in; log-likelihood and whole gradient of sampled
    particles against the FP64 oracle evaluated one particle at a time."""
    spec = _mlp4(nn.RELU)
    N, J = 60000, 1024
    X, y = _data(spec, N, 68)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=68, precision=S.PREC_BF16)
    try:
        D = spec.n_params
        th0 = synthetic.particles(J, D, 68, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 10))
        lp, g, la, lb = S.smc_eval(ctx, J, D)
        assert np.all(lb == 0.0) and np.all(np.isfinite(g))
        for j in [0, 1, 511, 1023]:
            ll, gg = nn.loglik_grad(spec, th0[j].astype(np.float64), orc.X, orc.y, 1.0)
            assert abs(la[j] - ll.sum()) <= TOL * abs(ll.sum()), j
            assert rel_err(g[j], gg) < TOL, j
    finally:
        S.smc_destroy(ctx)
