"""GPU parity of the sampler against the FP64 oracle, through the C ABI, on the
same seeded inputs.

Tolerances (stated by the build's target): FP32 paths 1e-5 relative; BF16
contractions 2e-2 relative for log-likelihoods and gradients; schedules,
mini-batch order and resampling indices bit-exact (resampling compared on
weights that agree to rounding, with near-ties reported instead of failed).
Gradient and parameter errors are norm-wise per particle."""
import math

import numpy as np
import pytest

import synthetic
from oracle import nn, rng, schedules, smc as osmc

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, oracle_eval, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)          # 16-32-4 tanh
MLP1 = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.RELU)     # 784-100-10 ReLU
CNN = nn.Spec([("conv", 3, 4, 3), ("pool2",), ("conv", 4, 3, 3), ("dense", 12, 5)], (3, 10, 10), nn.TANH)


def _mixture(N, seed):
    return synthetic.gaussian_mixture(N, d=16, n_classes=4, seed=seed)


def _images(N, seed):
    return synthetic.template_images(N, seed=seed)


def _per_particle_rel(a, b):
    return max(rel_err(a[j], b[j]) for j in range(a.shape[0]))


# ------------------------------------------------------------------ layout
def test_permutation_bitexact():
    X, y = _mixture(1000, 4)
    ctx, orc, _ = make_pair(MLP0, X, y, 4, seed=12345)
    try:
        assert np.array_equal(S.smc_get_permutation(ctx, 1000), rng.fisher_yates_permutation(1000, 12345))
    finally:
        S.smc_destroy(ctx)


def test_prior_draw_matches_oracle_philox():
    X, y = _mixture(64, 1)
    J, seed = 3, 77
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=seed, prior_sigma=0.5)
    try:
        th, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
        ref = 0.5 * rng.philox_normals(seed, 1, 0, J * MLP0.n_params).reshape(J, -1)
        assert np.max(np.abs(th - ref)) < 2e-5
    finally:
        S.smc_destroy(ctx)


# ------------------------------------------------------- evaluation parity
@pytest.mark.parametrize("chunk", [0, 100])
def test_fp32_mlp_eval_parity(chunk):
    X, y = _mixture(512, 3)
    J = 8
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=3, chunk=chunk)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 3)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 200, 200, 10))
        orc.set_schedule("linear", 200, 200, 10, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, MLP0.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=1e-5)
        assert np.allclose(la, rla, rtol=1e-5) and np.all(lb == 0.0)
        assert _per_particle_rel(g, rg) < 1e-5
    finally:
        S.smc_destroy(ctx)


# (hidden layers, rows, chunk rows): together they run every tile shape of the
# FP32 dense GEMM.  37-150-131-3 on 203 rows in chunks of 141 leaves every tile
# ragged (K = 37, 150, 131 off the 8-deep K step, a 3-column last tile,
# weight-gradient rows of 150 / 131 floats whose starts alternate between
# 16-byte aligned and not, so both epilogue store paths run) on 80 x 200
# tiles; 224-128 in chunks of 256 and of 200 runs 128 x 112, 128 x 128,
# 200 x 112 and 200 x 128 tiles; 400 in chunks of 256 runs 128 x 200 tiles.
DENSE_TILE_CASES = {
    "ragged_80x200": ((150, 131), 203, 141),
    "128x112_128x128": ((224, 128), 600, 256),
    "200x112_200x128": ((224, 128), 456, 200),
    "128x200": ((400,), 300, 256),
}


@pytest.mark.parametrize("case", sorted(DENSE_TILE_CASES))
def test_fp32_dense_tile_shapes_parity(case):
    hidden, N, chunk = DENSE_TILE_CASES[case]
    dims = (37,) + hidden + (3,)
    spec = nn.Spec([("dense", a, b) for a, b in zip(dims[:-1], dims[1:])], (37,), nn.TANH)
    J = 3
    X, y = synthetic.gaussian_mixture(N, d=37, n_classes=3, seed=21)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=21, chunk=chunk)
    try:
        th0 = synthetic.particles(J, spec.n_params, 21, std=0.2)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=1e-5)
        assert np.allclose(lp, rlp, rtol=1e-5)
        assert _per_particle_rel(g, rg) < 1e-5
        # every parameter segment separately (a wrong tile edge shows up in one)
        off = 0
        for L in spec.layers:
            nw, nb = L[1] * L[2], L[2]
            for seg in (slice(off, off + nw), slice(off + nw, off + nw + nb)):
                assert _per_particle_rel(g[:, seg], rg[:, seg]) < 1e-5
            off += nw + nb
        assert off == spec.n_params
    finally:
        S.smc_destroy(ctx)


def test_fp32_cnn_eval_parity():
    N, J = 70, 3
    X = synthetic.smooth_field_images(N, seed=2, side=10, channels=3)[0]
    y = (np.arange(N) % 5).astype(np.int32)
    ctx, orc, _ = make_pair(CNN, X, y, J, seed=8, chunk=25)
    try:
        th0 = synthetic.particles(J, CNN.n_params, 9, std=0.5)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, CNN.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=1e-5)
        assert np.allclose(lp, rlp, rtol=1e-5)
        assert _per_particle_rel(g, rg) < 1e-5
    finally:
        S.smc_destroy(ctx)


def test_fp32_gaussian_eval_parity():
    spec = nn.Spec([("dense", 3, 1)], (3,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=0.5)
    X, yv, _ = synthetic.linear_gaussian(150, 3, seed=5, noise_std=0.5)
    J = 4
    ctx, orc, _ = make_pair(spec, X, yv, J, seed=5)
    try:
        th0 = synthetic.particles(J, spec.n_params, 5)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("automated", 30, 30, 8))
        orc.set_schedule("automated", 30, 30, 8, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=1e-5) and np.allclose(la, rla, rtol=1e-5)
        assert _per_particle_rel(g, rg) < 1e-5
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("spec_dims,N,J,chunk,act", [((784, 100, 10), 700, 8, 0, nn.RELU),
                                                     ((784, 100, 10), 700, 8, 256, nn.TANH),
                                                     ((784, 100, 10), 1000, 3, 0, nn.TANH),
                                                     ((64, 48, 4), 300, 5, 0, nn.RELU)])
def test_bf16_eval_parity(spec_dims, N, J, chunk, act):
    """BF16 tensor-core evaluation against the FP64 oracle: whole gradient per
    particle within 2e-2 (norm-wise), log-likelihoods within 2e-2.  Each
    parameter block is also checked for the smooth (tanh) network; with ReLU a
    first-layer pre-activation within BF16 rounding of 0 can flip its mask,
    which moves single bias-gradient entries by a whole row's contribution, so
    per-block checks there would test the kink, not the kernels."""
    din, H, Cc = spec_dims
    spec = nn.Spec([("dense", din, H), ("dense", H, Cc)], (din,), act)
    if din == 784:
        X, y = _images(N, 6)
    else:
        X, y = synthetic.gaussian_mixture(N, d=din, n_classes=Cc, seed=6)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=6, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, spec.n_params, 6, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 256, 256, 10))
        orc.set_schedule("linear", 256, 256, 10, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=2e-2)
        assert np.allclose(lp, rlp, rtol=2e-2)
        assert _per_particle_rel(g, rg) < 2e-2
        if act == nn.TANH:
            off = 0
            for shp in [(H, din), (H,), (Cc, H), (Cc,)]:
                n = int(np.prod(shp))
                assert _per_particle_rel(g[:, off:off + n], rg[:, off:off + n]) < 2e-2, shp
                off += n
    finally:
        S.smc_destroy(ctx)


# --------------------------------------------------------------- one move
@pytest.mark.parametrize("precision", [S.PREC_FP32, S.PREC_BF16])
def test_step_parity_teacher_forced(precision):
    if precision == S.PREC_FP32:
        spec, (X, y), J, h, tol = MLP0, _mixture(512, 7), 8, 0.05, 1e-5
    else:
        spec, (X, y), J, h, tol = MLP1, _images(640, 7), 8, 0.002, 2e-2
    ctx, orc, _ = make_pair(spec, X, y, J, seed=7, precision=precision)
    try:
        th0 = synthetic.particles(J, spec.n_params, 70, std=0.3 if precision == S.PREC_FP32 else 0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 128, 128, 10))
        orc.set_schedule("linear", 128, 128, 10, th0)
        S.smc_anneal_next(ctx)
        orc.anneal_next()
        z = synthetic.normals((J, spec.n_params), 71)
        S.smc_set_noise(ctx, z)
        st = S.smc_step(ctx, h, 3)
        orc.step(h, 3, z)
        th, lw, lp = S.smc_get_state(ctx, J, spec.n_params)
        assert st["grad_evals"] == 4 and st["rows"] == 256
        assert _per_particle_rel(th, orc.theta) < tol
        assert np.allclose(lp, orc.logpi, rtol=tol)
        # log-weight increments (FP32: tight; BF16: relative to the log pi scale)
        inc_scale = np.abs(orc.logpi).max()
        assert np.max(np.abs(lw - orc.logw)) <= tol * inc_scale + 1e-6
        if precision == S.PREC_FP32:
            assert abs(st["ess"] - orc.ess) <= max(1e-3, tol) * J
        else:
            _check_weights_follow_logweights(ctx, J, lw, orc, st["ess"])
            # A pure annealing reweight (h = 0, special case p5): the move is the
            # identity and the kinetic terms cancel exactly, so the increment is
            # log pi_k(theta) - log pi_{k-1}(theta) and each log-weight's error can
            # grow by at most the two log pi errors of its particle.
            err_prev = np.abs(lw - orc.logw)
            S.smc_anneal_next(ctx)
            orc.anneal_next()
            d_start = np.abs(S.smc_get_state(ctx, J, None, theta=False)[2] - orc.logpi)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, 0.0, 3)
            orc.step(0.0, 3, z)
            assert st["rows"] == 384
            _, lw, lp = S.smc_get_state(ctx, J, spec.n_params)
            d_end = np.abs(lp - orc.logpi)
            assert np.all(d_end <= tol * np.abs(orc.logpi))
            err = np.abs(lw - orc.logw)
            allowed = err_prev + d_start + d_end + 1e-9 * (np.abs(orc.logpi) + np.abs(orc.logw))
            assert np.all(err <= allowed), (err, allowed)
            _check_weights_follow_logweights(ctx, J, lw, orc, st["ess"])
    finally:
        S.smc_destroy(ctx)


def _check_weights_follow_logweights(ctx, J, lw, orc, ess):
    """BF16 normalised weights and ESS, bounded by what the normalisation
    arithmetic allows (eqs. normalise, jeff): if every log-weight is within E
    of the oracle's, the log-sum-exp is within E too, so each normalised
    weight is within a factor e^{+-2E} and sum w~^2 within e^{+-4E}:
    |w~/w~_ref - 1| <= e^{2E} - 1 and |ESS/ESS_ref - 1| <= e^{4E} - 1."""
    E = float(np.max(np.abs(lw - orc.logw))) + 1e-12
    wn = S.smc_get_weights(ctx, J)
    assert np.all(np.abs(wn / orc.wn - 1.0) <= math.expm1(2 * E) * (1 + 1e-9) + 1e-12), (wn, orc.wn, E)
    assert abs(ess / orc.ess - 1.0) <= math.expm1(4 * E) * (1 + 1e-9) + 1e-12, (ess, orc.ess, E)


# ------------------------------------------------------- full trajectories
def test_config0_trajectory_parity():
    """2048 samples of a 16-d 4-class mixture, MLP 16-32-4 tanh, N(0,1) prior,
    J = 32, 8 mini-batches of 256, Linear schedule, 30 iterations, h = 0.002,
    S = 3, with injected momenta and resampling uniforms."""
    N, J, K, h, S_ = 2048, 32, 30, 0.002, 3
    X, y = _mixture(N, 0)
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=0)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 100)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 256, 256, K))
        orc.set_schedule("linear", 256, 256, K, th0)
        g = rng.SplitMix64(99)
        for k in range(1, K):
            info = S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert info["rows"] == orc.subset_rows == schedules.subset_size("linear", k, N, 256, 256, K)
            u = g.next_double()
            S.smc_set_uniforms(ctx, [u])
            near_tie = abs(orc.ess - J / 2) < 1e-6 * J
            did = S.smc_resample(ctx)
            odid = orc.resample(u=u)
            if near_tie:
                pytest.skip(f"ESS within 1e-6 J of J/2 at k={k}")
            assert did == odid, k
            if did:
                assert np.array_equal(S.smc_get_ancestors(ctx, J), orc.ancestors), k
            z = synthetic.normals((J, MLP0.n_params), 1000 + k)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, h, S_, )
            orc.step(h, S_, z)
            assert abs(st["ess"] - orc.ess) <= 1e-4 * J, (k, st["ess"], orc.ess)
        th, lw, lp = S.smc_get_state(ctx, J, MLP0.n_params)
        assert _per_particle_rel(th, orc.theta) < 1e-4
        assert np.allclose(lp, orc.logpi, rtol=1e-4)
        Xt, yt = synthetic.gaussian_mixture(1024, seed=0, test=True)
        probs = np.empty((1024, 4), np.float32)
        S.smc_posterior_predict(ctx, np.ascontiguousarray(Xt), probs)
        ref = orc.predict(Xt.astype(np.float64))
        assert np.max(np.abs(probs - ref)) < 1e-4
        acc, _ = osmc.accuracy_nll(probs, yt)
        racc, _ = osmc.accuracy_nll(ref, yt)
        assert abs(acc - racc) <= 2.0 / 1024
    finally:
        S.smc_destroy(ctx)


def test_sda_parity():
    N, J = 768, 16
    X, y = _mixture(N, 11)
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=11)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 11, std=0.3)
        S.smc_set_state(ctx, th0)
        # Delta S = 50 makes beta reach 1 within a few iterations so appends occur
        S.smc_set_schedule(ctx, S.make_schedule("sda", 128, 128, 40, delta_s=50.0))
        orc.set_schedule("sda", 128, 128, 40, th0, delta_s=50.0)
        appended = 0
        for k in range(1, 12):
            beta_prev = orc.sda.beta
            info = S.smc_anneal_next(ctx)
            oapp = orc.anneal_next()
            assert info["rows"] == orc.subset_rows and info["rows_full"] == orc.sda.m_full
            # beta' - beta = dS / |Var + Cov| with Var = E[X^2] - E[X]^2 of block log-likelihoods
            # of order 1e2: FP32 rounding of the sums is amplified by the cancellation, so the
            # increment is compared to 1e-3 relative.
            inc = abs(orc.sda.beta - beta_prev)
            assert abs(info["beta"] - orc.sda.beta) <= 1e-3 * inc + 1e-12, k
            appended += int(oapp)
            u = 0.25 + 0.5 * ((k * 0.618) % 1.0)
            S.smc_set_uniforms(ctx, [u])
            S.smc_resample(ctx)
            orc.resample(u=u)
            z = synthetic.normals((J, MLP0.n_params), 500 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.01, 2)
            orc.step(0.01, 2, z)
            th, _, lp = S.smc_get_state(ctx, J, MLP0.n_params)
            assert np.allclose(lp, orc.logpi, rtol=1e-4), k
        assert appended >= 1
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("act", [nn.TANH, nn.RELU])
def test_bf16_sda_parity(act):
    """The BF16 engine under smooth data annealing (Sec. 3.1): both row regions
    in use (fully included rows at coefficient 1, the tempered block at beta),
    so the fused kernel's two log-likelihood sums, its beta-weighted dlogits
    and the SDA moments all take part.  Each iteration, at the GPU's particles:
    La, Lb and log pi against the oracle within 2e-2, the whole log-likelihood
    gradient per particle within 2e-2 (per parameter block too for tanh);
    then the temperature update from the GPU's own weights and sums against
    the oracle's rule (FP64 moments on both sides, 1e-9), the subset sizes
    bit-exact, and one teacher-forced move within 2e-2."""
    N, J, D = 1024, 8, MLP1.n_params
    spec = nn.Spec(MLP1.layers, MLP1.input_shape, act)
    X, y = _images(N, 31)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=31, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, D, 31, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("sda", 256, 256, 40, delta_s=4.0))
        orc.set_schedule("sda", 256, 256, 40, th0, delta_s=4.0)
        appended, both_regions, tempered = 0, 0, 0
        for k in range(1, 17):
            th, lw, lp = S.smc_get_state(ctx, J, D)
            wn = S.smc_get_weights(ctx, J)
            elp, eg, ela, elb = S.smc_eval(ctx, J, D)
            # the oracle at the GPU's particles, target and weights (teacher forcing)
            orc.theta = th.astype(np.float64)
            rlp, rg, rla, rlb = oracle_eval(orc)
            scale = np.abs(rla) + np.abs(rlb)
            assert np.all(np.abs(ela - rla) <= 2e-2 * scale + 1e-6), k
            assert np.all(np.abs(elb - rlb) <= 2e-2 * scale + 1e-6), k
            assert np.allclose(elp, rlp, rtol=2e-2), k
            assert _per_particle_rel(eg, rg) < 2e-2, k
            if act == nn.TANH:
                off = 0
                for shp in [(100, 784), (100,), (10, 100), (10,)]:
                    n = int(np.prod(shp))
                    assert _per_particle_rel(eg[:, off:off + n], rg[:, off:off + n]) < 2e-2, (k, shp)
                    off += n
            both_regions += int(orc.sda.m_full > 0 and orc.sda.block > 0)
            tempered += int(orc.sda.block > 0 and orc.sda.beta < 1.0)
            orc.logpi, orc.la, orc.lb = lp.astype(np.float64), ela.astype(np.float64), elb.astype(np.float64)
            orc.logw, orc.wn = lw.astype(np.float64), wn.astype(np.float64)
            orc.ess = osmc.ess(orc.wn)
            info = S.smc_anneal_next(ctx)
            appended += int(orc.anneal_next())
            assert info["rows"] == orc.subset_rows and info["rows_full"] == orc.sda.m_full, k
            assert info["beta"] == pytest.approx(orc.sda.beta, rel=1e-9, abs=1e-12), (k, info["beta"], orc.sda.beta)
            u = 0.25 + 0.5 * ((k * 0.618) % 1.0)
            near_tie = abs(orc.ess - J / 2) < 1e-6 * J
            S.smc_set_uniforms(ctx, [u])
            did = S.smc_resample(ctx)
            odid = orc.resample(u=u)
            if not near_tie:
                assert did == odid, k
                if did:
                    assert np.array_equal(S.smc_get_ancestors(ctx, J), orc.ancestors), k
            if did != odid:      # a near-tie decided differently: continue from the GPU's particles
                th, _, _ = S.smc_get_state(ctx, J, D)
                orc.theta = th.astype(np.float64)
            z = synthetic.normals((J, D), 700 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.002, 2)
            orc.step(0.002, 2, z)
            th2, _, lp2 = S.smc_get_state(ctx, J, D)
            assert _per_particle_rel(th2, orc.theta) < 2e-2, k
            assert np.allclose(lp2, orc.logpi, rtol=2e-2), k
        assert appended >= 2 and both_regions >= 4 and tempered >= 5, (appended, both_regions, tempered)
    finally:
        S.smc_destroy(ctx)


def test_bf16_predictive_parity():
    N, J = 512, 6
    X, y = _images(N, 21)
    ctx, orc, _ = make_pair(MLP1, X, y, J, seed=21, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, MLP1.n_params, 21, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        Xt, _ = synthetic.template_images(300, seed=21, test=True)
        probs = np.empty((300, 10), np.float32)
        S.smc_posterior_predict(ctx, np.ascontiguousarray(Xt), probs)
        ref = orc.predict(Xt.astype(np.float64))
        assert np.max(np.abs(probs - ref)) < 2e-2
        assert np.allclose(probs.sum(axis=1), 1.0, atol=1e-5)
    finally:
        S.smc_destroy(ctx)


# ------------------------------------------------------------ properties
def test_runs_are_bitwise_deterministic():
    X, y = _mixture(600, 2)
    outs = []
    for _ in range(2):
        ctx, _, _ = make_pair(MLP0, X, y, 16, seed=42)
        try:
            S.smc_set_schedule(ctx, S.make_schedule("linear", 150, 150, 10))
            for _k in range(4):
                S.smc_anneal_next(ctx)
                S.smc_resample(ctx)
                S.smc_step(ctx, 0.01, 3)
            outs.append(S.smc_get_state(ctx, 16, MLP0.n_params))
        finally:
            S.smc_destroy(ctx)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_weights_invariants_after_steps():
    X, y = _mixture(512, 9)
    J = 64
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=9)
    try:
        S.smc_set_schedule(ctx, S.make_schedule("linear", 128, 128, 8))
        for _ in range(3):
            S.smc_anneal_next(ctx)
            st = S.smc_step(ctx, 0.01, 2)
            w = S.smc_get_weights(ctx, J)
            assert abs(w.sum() - 1.0) < 1e-12
            assert 1.0 - 1e-9 <= st["ess"] <= J + 1e-9
            assert abs(st["ess"] - 1.0 / np.sum(w * w)) < 1e-9 * J
            S.smc_resample(ctx, force=True)
            assert np.allclose(S.smc_get_weights(ctx, J), 1.0 / J)
    finally:
        S.smc_destroy(ctx)


def test_error_statuses():
    X, y = _mixture(64, 1)
    with pytest.raises(S.SMCError) as e:
        make_pair(MLP0, X, y, 0, seed=1)
    assert e.value.status == 1
    Xc = np.zeros((16, 300), np.float32)
    with pytest.raises(S.SMCError) as e:
        make_pair(CNN, Xc, np.zeros(16, np.int32), 2, seed=1, precision=S.PREC_BF16)
    assert e.value.status == 7
    ctx, _, _ = make_pair(MLP0, X, y, 2, seed=1)
    try:
        with pytest.raises(S.SMCError) as e:
            S.smc_step(ctx, 0.01, 1)
        assert e.value.status == 4          # step before set_schedule
        S.smc_set_schedule(ctx, S.make_schedule("fb", 64, 64, 3))
        with pytest.raises(S.SMCError) as e:
            S.smc_step(ctx, -1.0, 1)
        assert e.value.status == 1
        with pytest.raises(S.SMCError):
            S.smc_set_uniforms(ctx, [1.5])
    finally:
        S.smc_destroy(ctx)


# ------------------------------------------------- configuration-shaped cases
CNN2 = nn.Spec([("conv", 3, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 800, 10)],
               (3, 32, 32), nn.TANH)
MLP4 = nn.Spec([("dense", 784, 400), ("dense", 400, 400), ("dense", 400, 10)], (784,), nn.RELU)


def test_cnn_config_sda_parity():
    """3x32x32 10-class smooth-field images, CNN conv5x5 3->16, pool, conv5x5
    16->32, pool, fc 800->10 (tanh), SDA schedule: FP32 engine against the
    oracle over three iterations (anneal, resample, move)."""
    N, J = 96, 4
    X, y = synthetic.smooth_field_images(N, seed=12)
    ctx, orc, _ = make_pair(CNN2, X, y, J, seed=12, chunk=40)
    try:
        th0 = synthetic.particles(J, CNN2.n_params, 12, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("sda", 32, 32, 20, delta_s=20.0))
        orc.set_schedule("sda", 32, 32, 20, th0, delta_s=20.0)
        lp, g, la, lb = S.smc_eval(ctx, J, CNN2.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(lb, rlb, rtol=1e-5) and _per_particle_rel(g, rg) < 1e-5
        for k in range(1, 4):
            beta_prev = orc.sda.beta
            info = S.smc_anneal_next(ctx)
            orc.anneal_next()
            assert info["rows"] == orc.subset_rows
            assert abs(info["beta"] - orc.sda.beta) <= 1e-3 * abs(orc.sda.beta - beta_prev) + 1e-12
            S.smc_set_uniforms(ctx, [0.3])
            S.smc_resample(ctx)
            orc.resample(u=0.3)
            z = synthetic.normals((J, CNN2.n_params), 40 + k)
            S.smc_set_noise(ctx, z)
            S.smc_step(ctx, 0.005, 2)
            orc.step(0.005, 2, z)
            th, _, lp = S.smc_get_state(ctx, J, CNN2.n_params)
            assert _per_particle_rel(th, orc.theta) < 1e-5 and np.allclose(lp, orc.logpi, rtol=1e-5)
        # posterior predictive over a separate test draw (weights from the last move)
        Xt, _ = synthetic.smooth_field_images(50, seed=12, test=True)
        probs = np.empty((50, 10), np.float32)
        S.smc_posterior_predict(ctx, np.ascontiguousarray(Xt, np.float32), probs)
        ref = orc.predict(Xt.astype(np.float64))
        assert np.max(np.abs(probs - ref)) < 1e-5
    finally:
        S.smc_destroy(ctx)


def test_two_hidden_layer_config_parity_and_fd():
    """MLP 784-400-400-10 ReLU on the MNIST-shaped data: gradient against the
    oracle and a finite-difference check of the library's own adjoint on 64
    random coordinates per particle (log pi evaluated by the library)."""
    N, J = 200, 2
    X, y = _images(N, 13)
    ctx, orc, _ = make_pair(MLP4, X, y, J, seed=13)
    try:
        th0 = synthetic.particles(J, MLP4.n_params, 13, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, MLP4.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(lp, rlp, rtol=1e-5) and _per_particle_rel(g, rg) < 1e-5
        r = np.random.default_rng(13)
        eps = 1e-2
        fd_err = []
        for j in range(J):
            idx = r.choice(MLP4.n_params, 64, replace=False)
            for i in idx:
                vals = []
                for sgn in (1.0, -1.0):
                    th = th0.copy()
                    th[j, i] += sgn * eps
                    S.smc_set_state(ctx, th)
                    vals.append(S.smc_eval(ctx, J, MLP4.n_params)[0][j])
                fd = (vals[0] - vals[1]) / (2 * eps)
                # gradient of log pi includes the prior term -theta / sigma^2
                fd_err.append(abs(fd - (g[j, i] - th0[j, i])) / max(1.0, abs(fd)))
        # a ReLU kink inside +-eps spoils single coordinates, so the bound is on quantiles
        assert np.median(fd_err) < 1e-2 and np.percentile(fd_err, 90) < 0.05
    finally:
        S.smc_destroy(ctx)


def test_bf16_full_size_sampled_particles():
    """The bench workload's shape (MLP 784-100-10 ReLU, J = 256 particles, all
    60000 rows in one pass, the launch configuration the bench times): log
    likelihood and whole gradient of sampled particles - both members of the
    first and last particle pairs and some in between - against the FP64 oracle
    evaluated one particle at a time."""
    N, J = 60000, 256
    X, y = _images(N, 17)
    ctx, orc, _ = make_pair(MLP1, X, y, J, seed=17, precision=S.PREC_BF16)
    try:
        th0 = synthetic.particles(J, MLP1.n_params, 17, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 10))      # |D_0| = N, c_i = 1
        lp, g, la, lb = S.smc_eval(ctx, J, MLP1.n_params)
        assert np.all(lb == 0.0)
        for j in [0, 1, 2, 77, 128, 129, 254, 255]:
            ll, gg = nn.loglik_grad(MLP1, th0[j], orc.X, orc.y, 1.0)
            assert abs(la[j] - ll.sum()) <= 2e-2 * abs(ll.sum()), j
            assert rel_err(g[j], gg) < 2e-2, j
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("J,N,chunk", [(8, 700, 0), (5, 1000, 256)])
def test_bf16_fused_and_unfused_heads_agree(monkeypatch, J, N, chunk):
    """The forward GEMM with the head in its epilogue against the separate
    forward GEMM + head kernels on the same particles: same log-likelihoods and
    gradients up to BF16 rounding of dZ1 in db1 and the summation order."""
    spec = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.TANH)
    X, y = _images(N, 19)
    th0 = synthetic.particles(J, spec.n_params, 19, std=0.1)
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("SMC_FUSED_HEAD", fused)
        ctx, _, _ = make_pair(spec, X, y, J, seed=19, precision=S.PREC_BF16, chunk=chunk)
        try:
            S.smc_set_state(ctx, th0)
            S.smc_set_schedule(ctx, S.make_schedule("linear", 256, 256, 10))
            out[fused] = S.smc_eval(ctx, J, spec.n_params)
        finally:
            S.smc_destroy(ctx)
    (lp1, g1, la1, lb1), (lp0, g0, la0, lb0) = out["1"], out["0"]
    assert np.allclose(la1, la0, rtol=1e-5) and np.allclose(lb1, lb0, rtol=1e-5, atol=1e-6)
    assert np.allclose(lp1, lp0, rtol=1e-5)
    assert _per_particle_rel(g1, g0) < 2e-3


LENET5 = [("conv", 1, 6, 5), ("pool2",), ("conv", 6, 16, 5), ("pool2",), ("dense", 400, 120), ("dense", 120, 84),
          ("dense", 84, 10)]


@pytest.mark.parametrize("act", [nn.TANH, nn.RELU])
def test_lenet5_eval_parity(act):
    """LeNet-5 (Sec. 4's model family; D = 61,706) as a model description:
    28x28 images zero-padded to 32x32 (the first convolution's padding of 2),
    two 5x5 valid convolutions with 2x2 max pooling, dense 400-120-84-10;
    log-likelihoods and whole gradients against the FP64 oracle."""
    spec = nn.Spec(LENET5, (1, 32, 32), act)
    assert spec.n_params == 61706
    N, J = 48, 2
    X, y = _images(N, 23)
    X = np.pad(X.reshape(N, 1, 28, 28), ((0, 0), (0, 0), (2, 2), (2, 2))).reshape(N, 1024)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=23, chunk=20)
    try:
        th0 = synthetic.particles(J, spec.n_params, 23, std=0.1)
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


def test_bf16_split_k_across_chunks():
    """Subsets long enough for the weight-gradient GEMM to split K (here eight
    slices, summed inside the CTA-pair kernel) and processed in two chunks
    whose gradients accumulate: whole gradients and log-likelihoods against
    the FP64 oracle."""
    N, J, chunk = 20000, 8, 10000
    X, y = _images(N, 29)
    ctx, orc, _ = make_pair(MLP1, X, y, J, seed=29, precision=S.PREC_BF16, chunk=chunk)
    try:
        th0 = synthetic.particles(J, MLP1.n_params, 29, std=0.1)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        lp, g, la, lb = S.smc_eval(ctx, J, MLP1.n_params)
        for j in range(J):
            ll, gg = nn.loglik_grad(MLP1, th0[j], orc.X, orc.y, 1.0)
            assert abs(la[j] - ll.sum()) <= 2e-2 * abs(ll.sum()), j
            assert rel_err(g[j], gg) < 2e-2, j
    finally:
        S.smc_destroy(ctx)


# ------------------------------------------------ fresh mini-batch schedules
def _fresh_window_eval(spec, X, y, J, seed, precision, kind, C, K, n_iter, chunk, tol, std):
    """Anneal through n_iter targets of a fresh-mini-batch schedule and compare
    each target's evaluation (log pi, L_a, whole gradient) with the oracle."""
    N = X.shape[0]
    ctx, orc, _ = make_pair(spec, X, y, J, seed=seed, precision=precision, chunk=chunk)
    wrapped = False
    try:
        th0 = synthetic.particles(J, spec.n_params, seed, std=std)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule(kind, C, C, K))
        orc.set_schedule(kind, C, C, K, th0)
        for k in range(n_iter):
            if k:
                info = S.smc_anneal_next(ctx)
                orc.anneal_next()
                assert info["rows"] == orc.subset_rows
            rows = orc.rows()
            wrapped = wrapped or bool(rows[0] > rows[-1])
            lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
            rlp, rg, rla, rlb = oracle_eval(orc)
            assert np.allclose(la, rla, rtol=tol), k
            assert np.allclose(lp, rlp, rtol=tol), k
            assert np.all(lb == 0.0)
            assert _per_particle_rel(g, rg) < tol, k
    finally:
        S.smc_destroy(ctx)
    return wrapped


@pytest.mark.parametrize("kind,chunk", [("constant_fresh", 0), ("constant_fresh", 64), ("ctr_fresh", 0)])
def test_fp32_fresh_minibatch_eval_parity(kind, chunk):
    """N = 500 rows, C = 160: the window starts at 0, 160, 320, 480 (wrapping
    to rows 0..139), 140, ...; CTR's late switch (k >= 0.9 K) takes all rows."""
    X, y = _mixture(500, 37)
    assert _fresh_window_eval(MLP0, X, y, 8, 37, S.PREC_FP32, kind, 160, 10, 10 if kind == "ctr_fresh" else 6,
                              chunk, 1e-5, 0.3)


@pytest.mark.parametrize("chunk", [0, 128])
def test_bf16_fresh_minibatch_eval_parity(chunk):
    """BF16 engine, N = 1000, C = 256: the fourth window runs from row 768 to
    999 and wraps to rows 0..23, so the weight-gradient GEMM's first chunk is
    not the chunk of row 0."""
    X, y = _images(1000, 38)
    assert _fresh_window_eval(MLP1, X, y, 8, 38, S.PREC_BF16, "constant_fresh", 256, 10, 5, chunk, 2e-2, 0.1)


def test_fresh_minibatch_trajectory_parity():
    """Constant with a fresh mini-batch every iteration, J = 16, 12 moves with
    injected momenta and resampling uniforms: ESS, ancestors, particles and
    log pi against the oracle."""
    N, J, K, C, h, S_ = 600, 16, 12, 128, 0.01, 2
    X, y = _mixture(N, 39)
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=39)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 39)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant_fresh", C, C, K))
        orc.set_schedule("constant_fresh", C, C, K, th0)
        g = rng.SplitMix64(39)
        for k in range(1, K):
            S.smc_anneal_next(ctx)
            orc.anneal_next()
            u = g.next_double()
            S.smc_set_uniforms(ctx, [u])
            near_tie = abs(orc.ess - J / 2) < 1e-6 * J
            did = S.smc_resample(ctx)
            odid = orc.resample(u=u)
            if near_tie:
                pytest.skip(f"ESS within 1e-6 J of J/2 at k={k}")
            assert did == odid, k
            if did:
                assert np.array_equal(S.smc_get_ancestors(ctx, J), orc.ancestors), k
            z = synthetic.normals((J, MLP0.n_params), 3900 + k)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, h, S_)
            orc.step(h, S_, z)
            assert st["rows"] == C
            assert abs(st["ess"] - orc.ess) <= 1e-4 * J, (k, st["ess"], orc.ess)
        th, lw, lp = S.smc_get_state(ctx, J, MLP0.n_params)
        assert _per_particle_rel(th, orc.theta) < 1e-4
        assert np.allclose(lp, orc.logpi, rtol=1e-4)
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("fused", [True, False])
def test_bf16_fresh_minibatch_unaligned_windows(monkeypatch, fused):
    """BF16 engine, N = 1000, C = 300, chunks of 128 rows: windows start at
    rows 0, 300, 600 and 900 (wrapping to 0..199), two of them off the 8-row
    boundary the weight-gradient GEMM's TMA source needs, so their first
    chunk begins up to 7 rows early with those rows masked out; fused and
    separate head kernels."""
    if not fused:
        monkeypatch.setenv("SMC_FUSED_HEAD", "0")
    X, y = _images(1000, 40)
    assert _fresh_window_eval(MLP1, X, y, 4, 40, S.PREC_BF16, "constant_fresh", 300, 10, 4, 128, 2e-2, 0.1)


def test_multinomial_unscaled_trajectory_parity():
    """The paper-faithful variants as configuration: multinomial resampling
    (J injected uniforms) and c_i = 1 instead of N / M_k, on a Constant
    schedule (M_k < N, so the scale matters), 10 moves with injected momenta
    and resampling forced every third iteration: ancestors, ESS, particles
    and log pi against the oracle."""
    N, J, K, h, S_ = 600, 16, 10, 0.01, 2
    X, y = _mixture(N, 55)
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=55, scaled=False, resampler=S.RESAMPLE_MULTINOMIAL)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 55)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("constant", 128, 128, K))
        orc.set_schedule("constant", 128, 128, K, th0)
        rlp0 = oracle_eval(orc)[0]
        lp0 = S.smc_eval(ctx, J, MLP0.n_params)[0]
        assert np.allclose(lp0, rlp0, rtol=1e-5)
        g = rng.SplitMix64(55)
        resampled = 0
        for k in range(1, K):
            S.smc_anneal_next(ctx)
            orc.anneal_next()
            u = [g.next_double() for _ in range(J)]
            force = k % 3 == 0
            S.smc_set_uniforms(ctx, u)
            near_tie = not force and abs(orc.ess - J / 2) < 1e-6 * J
            did = S.smc_resample(ctx, force=force)
            odid = orc.resample(uniforms=np.array(u), kind="multinomial", force=force)
            if near_tie:
                pytest.skip(f"ESS within 1e-6 J of J/2 at k={k}")
            assert did == odid, k
            if did:
                resampled += 1
                assert np.array_equal(S.smc_get_ancestors(ctx, J), orc.ancestors), k
            z = synthetic.normals((J, MLP0.n_params), 5500 + k)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, h, S_)
            orc.step(h, S_, z)
            assert abs(st["ess"] - orc.ess) <= 1e-4 * J, (k, st["ess"], orc.ess)
        assert resampled >= 3
        th, lw, lp = S.smc_get_state(ctx, J, MLP0.n_params)
        assert _per_particle_rel(th, orc.theta) < 1e-4
        assert np.allclose(lp, orc.logpi, rtol=1e-4)
    finally:
        S.smc_destroy(ctx)


@pytest.mark.parametrize("precision", [S.PREC_FP32, S.PREC_BF16])
def test_fused_momentum_draw_matches_philox_stream(precision):
    """The first leapfrog pass draws P^0 itself; a twin context given the same
    (seed, momentum stream, step) Philox normals as injected noise must follow
    the same trajectory bit for bit."""
    if precision == S.PREC_FP32:
        spec, (X, y), h = MLP0, _mixture(512, 56), 0.01
    else:
        spec, (X, y), h = MLP1, _images(512, 56), 0.002
    J, D, seed = 8, spec.n_params, 56
    a, _, _ = make_pair(spec, X, y, J, seed=seed, precision=precision)
    b, _, _ = make_pair(spec, X, y, J, seed=seed, precision=precision)
    try:
        th0 = synthetic.particles(J, D, 56, std=0.1)
        for ctx in (a, b):
            S.smc_set_state(ctx, th0)
            S.smc_set_schedule(ctx, S.make_schedule("linear", 128, 128, 10))
        for step in range(3):
            for ctx in (a, b):
                S.smc_anneal_next(ctx)
            z = torch.empty(J * D, dtype=torch.float32, device="cuda")
            S.smc_k_philox_normals(seed, 2, step, 0, z)
            torch.cuda.synchronize()
            S.smc_set_noise(b, z.cpu().numpy().reshape(J, D))
            sa = S.smc_step(a, h, 2)
            sb = S.smc_step(b, h, 2)
            assert sa["ess"] == sb["ess"], step
            for u, v in zip(S.smc_get_state(a, J, D), S.smc_get_state(b, J, D)):
                assert np.array_equal(u, v), step
    finally:
        S.smc_destroy(a)
        S.smc_destroy(b)


def test_fp32_conv_fallback_parity():
    """A 64 -> 64 channel 5x5 convolution needs more shared memory than a block
    has (1600 taps x 64 channels of weights), so that layer runs on the direct
    kernels while the first (3 -> 64) runs on the tiled ones: evaluation
    against the oracle, whole gradient per particle."""
    spec = nn.Spec([("conv", 3, 64, 5), ("conv", 64, 64, 5), ("dense", 64 * 8 * 8, 10)], (3, 16, 16), nn.TANH)
    N, J = 8, 2
    X, y = synthetic.smooth_field_images(N, seed=57, side=16)
    ctx, orc, _ = make_pair(spec, X, y, J, seed=57)
    try:
        th0 = synthetic.particles(J, spec.n_params, 57, std=0.05)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 5))
        orc.set_schedule("fb", N, N, 5, th0)
        lp, g, la, lb = S.smc_eval(ctx, J, spec.n_params)
        rlp, rg, rla, rlb = oracle_eval(orc)
        assert np.allclose(la, rla, rtol=1e-5) and np.allclose(lp, rlp, rtol=1e-5)
        assert _per_particle_rel(g, rg) < 1e-5
    finally:
        S.smc_destroy(ctx)
