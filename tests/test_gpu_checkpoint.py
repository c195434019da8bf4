"""GPU tests of smc_checkpoint / smc_restore through the C ABI: a run continued
from a restored checkpoint reproduces the original continuation bit for bit
(particles, log-weights, log pi, ESS, ancestors) for the FP32 and BF16 engines,
a fixed schedule, SDA and the learned proposal; a checkpoint is refused by a
context with another J, seed or precision, and a malformed file is refused."""
import numpy as np
import pytest

import synthetic
from oracle import nn

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)
MLP1 = nn.Spec([("dense", 784, 100), ("dense", 100, 10)], (784,), nn.RELU)


def _continue(ctx, J, D, n, proposal=S.PROPOSAL_PLAIN, h=0.01):
    out = []
    for _ in range(n):
        S.smc_anneal_next(ctx)
        did = S.smc_resample(ctx)
        st = S.smc_step(ctx, h, 2, proposal)
        th, lw, lp = S.smc_get_state(ctx, J, D)
        out.append((th, lw, lp, st["ess"], did, S.smc_get_ancestors(ctx, J)))
    return out


def _same(a, b):
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(np.asarray(u), np.asarray(v))


def _roundtrip(tmp_path, spec, X, y, J, seed, sched, n_before, n_after, precision=S.PREC_FP32, proposal=None,
               prepare=None):
    path = str(tmp_path / "state.ckpt")
    D = spec.n_params
    ctx, _, _ = make_pair(spec, X, y, J, seed=seed, precision=precision)
    try:
        S.smc_set_schedule(ctx, sched)
        if prepare:
            prepare(ctx)
        _continue(ctx, J, D, n_before, proposal or S.PROPOSAL_PLAIN)
        S.smc_checkpoint(ctx, path)
        ref = _continue(ctx, J, D, n_after, proposal or S.PROPOSAL_PLAIN)
    finally:
        S.smc_destroy(ctx)
    ctx2, _, _ = make_pair(spec, X, y, J, seed=seed, precision=precision)
    try:
        S.smc_restore(ctx2, path)
        got = _continue(ctx2, J, D, n_after, proposal or S.PROPOSAL_PLAIN)
    finally:
        S.smc_destroy(ctx2)
    _same(ref, got)
    return path


def test_fp32_fixed_schedule_roundtrip(tmp_path):
    X, y = synthetic.gaussian_mixture(512, seed=31)
    _roundtrip(tmp_path, MLP0, X, y, 16, 31, S.make_schedule("linear", 128, 128, 10), 3, 4)


def test_fp32_sda_roundtrip(tmp_path):
    X, y = synthetic.gaussian_mixture(512, seed=32)
    _roundtrip(tmp_path, MLP0, X, y, 16, 32, S.make_schedule("sda", 128, 128, 10, delta_s=50.0), 4, 5)


def test_bf16_roundtrip(tmp_path):
    X, y = synthetic.template_images(700, seed=33)
    _roundtrip(tmp_path, MLP1, X, y, 8, 33, S.make_schedule("linear", 256, 256, 10), 2, 3, precision=S.PREC_BF16)


def test_learned_proposal_roundtrip(tmp_path):
    X, y = synthetic.gaussian_mixture(512, seed=34)

    def prepare(ctx):
        for _ in range(4):
            S.smc_step(ctx, 0.01, 2, S.PROPOSAL_EXPLORE, groups=4, explore_sigma=0.5)
        S.smc_learned_train(ctx, 20, 0.01)

    _roundtrip(tmp_path, MLP0, X, y, 16, 34, S.make_schedule("fb", 512, 512, 10), 2, 3,
               proposal=S.PROPOSAL_LEARNED, prepare=prepare)


def test_restore_refuses_other_runs(tmp_path):
    X, y = synthetic.gaussian_mixture(256, seed=35)
    path = str(tmp_path / "a.ckpt")
    ctx, _, _ = make_pair(MLP0, X, y, 8, seed=35)
    try:
        S.smc_set_schedule(ctx, S.make_schedule("fb", 256, 256, 5))
        S.smc_checkpoint(ctx, path)
    finally:
        S.smc_destroy(ctx)
    for J, seed in [(16, 35), (8, 36)]:
        other, _, _ = make_pair(MLP0, X, y, J, seed=seed)
        try:
            with pytest.raises(S.SMCError) as e:
                S.smc_restore(other, path)
            assert e.value.status == 1
        finally:
            S.smc_destroy(other)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 8)
    ctx, _, _ = make_pair(MLP0, X, y, 8, seed=35)
    try:
        with pytest.raises(S.SMCError) as e:
            S.smc_restore(ctx, str(bad))
        assert e.value.status == 1
        with open(path, "rb") as f:          # truncated: header intact, arrays cut short
            head = f.read(400)
        trunc = tmp_path / "trunc.ckpt"
        trunc.write_bytes(head)
        with pytest.raises(S.SMCError) as e:
            S.smc_restore(ctx, str(trunc))
        assert e.value.status == 1
    finally:
        S.smc_destroy(ctx)


def test_fresh_minibatch_roundtrip(tmp_path):
    """The window start of a fresh-mini-batch schedule follows from k, which
    the checkpoint restores (N = 500, C = 160: the restored run wraps)."""
    X, y = synthetic.gaussian_mixture(500, seed=36)
    _roundtrip(tmp_path, MLP0, X, y, 16, 36, S.make_schedule("constant_fresh", 160, 160, 10), 2, 4)
