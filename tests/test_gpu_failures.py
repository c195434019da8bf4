"""Failure detection without a GPU fault: every failure is made on the host or
by a bounded device wait that is left to run out.

* the library's bounded device-side wait (the one the tensor-core kernels use)
  gives up after its limit on an mbarrier nothing completes, reports
  SMC_ETIMEOUT, and the GPU context keeps working;
* a particle whose parameters are NaN gets log-weight -inf and weight 0, is
  counted as non-finite, and resampling never picks it;
* all particles non-finite: SMC_ENUMERIC (from the initial weights on, at
  every call that normalises them);
* a model too large for device memory: SMC_ENOMEM from smc_init, and the next
  context works."""
import time

import numpy as np
import pytest

import synthetic
from oracle import nn

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)


def _mixture(n, seed):
    return synthetic.gaussian_mixture(n, d=16, n_classes=4, seed=seed)


def _sampler_works(seed):
    X, y = _mixture(128, seed)
    ctx, _, _ = make_pair(MLP0, X, y, 4, seed=seed)
    try:
        S.smc_set_schedule(ctx, S.make_schedule("fb", 128, 128, 3))
        S.smc_anneal_next(ctx)
        st = S.smc_step(ctx, 0.01, 2)
        assert np.isfinite(st["ess"]) and 1.0 <= st["ess"] <= 4.0
    finally:
        S.smc_destroy(ctx)


def test_bounded_wait_gives_up_and_context_stays_usable():
    t0 = time.perf_counter()
    with pytest.raises(S.SMCError) as e:
        S.smc_k_wait_probe(50.0, arrive=False)
    assert e.value.status == 6                      # SMC_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    S.smc_k_wait_probe(50.0, arrive=True)           # a completed phase is seen at once
    with pytest.raises(S.SMCError) as e:
        S.smc_k_wait_probe(0.0, arrive=True)
    assert e.value.status == 1
    _sampler_works(81)


def test_nan_particle_gets_zero_weight_and_is_not_resampled():
    X, y = _mixture(256, 82)
    J = 8
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=82)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 82, std=0.3)
        th0[3] = np.nan
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("fb", 256, 256, 5))
        _, lw, _ = S.smc_get_state(ctx, J, MLP0.n_params, theta=False)
        wn = S.smc_get_weights(ctx, J)
        assert lw[3] == -np.inf and wn[3] == 0.0
        assert np.all(np.isfinite(lw[np.arange(J) != 3]))
        assert abs(wn.sum() - 1.0) < 1e-12
        S.smc_anneal_next(ctx)
        st = S.smc_step(ctx, 0.01, 2)
        assert st["n_nonfinite"] >= 1
        assert S.smc_resample(ctx, force=True)
        anc = S.smc_get_ancestors(ctx, J)
        assert 3 not in anc
        th, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
        assert np.all(np.isfinite(th))
    finally:
        S.smc_destroy(ctx)


def test_all_particles_non_finite_is_an_error():
    X, y = _mixture(64, 83)
    J = 4
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=83)
    try:
        S.smc_set_state(ctx, np.full((J, MLP0.n_params), np.nan, np.float32))
        with pytest.raises(S.SMCError) as e:        # the initial weights (eq. init_weight)
            S.smc_set_schedule(ctx, S.make_schedule("fb", 64, 64, 5))
        assert e.value.status == 5                  # SMC_ENUMERIC
        with pytest.raises(S.SMCError) as e:        # a data condition, not a CUDA failure:
            S.smc_step(ctx, 0.01, 1)                # the next move reports it again
        assert e.value.status == 5
    finally:
        S.smc_destroy(ctx)


def test_allocation_failure_reports_enomem():
    """D = 1.0e9 parameters per particle x 512 particles (2 TB of FP32 per
    particle array) cannot be allocated on the device."""
    model = S.make_model([("dense", 50000, 20000), ("dense", 20000, 10)], (50000,), S.ACT_TANH)
    X = np.zeros((4, 50000), np.float32)
    y = np.zeros(4, np.int32)
    cfg = S.make_config(512, 84, S.PREC_FP32, stream=torch.cuda.current_stream())
    with pytest.raises(S.SMCError) as e:
        S.smc_init(model, X, y_class=y, cfg=cfg)
    assert e.value.status == 2                      # SMC_ENOMEM
    _sampler_works(84)
