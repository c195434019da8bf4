"""GPU tests of the row-upload calls: rows staged by smc_upload_rows_async
take effect at the next smc_set_schedule / smc_anneal_next and give exactly
the evaluation of the same rows uploaded synchronously (FP32 and BF16
engines), two staged uploads apply in call order, and an upload issued while
an iteration computes is not seen by that iteration."""
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


def _case(precision):
    if precision == S.PREC_FP32:
        X, y = synthetic.gaussian_mixture(512, d=16, n_classes=4, seed=61)
        return MLP0, X, y
    X, y = synthetic.template_images(512, seed=61)
    return MLP1, X, y


def _eval(ctx, J, D):
    lp, g, la, lb = S.smc_eval(ctx, J, D)
    return lp, g


@pytest.mark.parametrize("precision", [S.PREC_FP32, S.PREC_BF16])
def test_async_upload_matches_sync_upload(precision):
    spec, X, y = _case(precision)
    J, D = 4, spec.n_params
    r = np.random.default_rng(61)
    new_x = np.ascontiguousarray(X[r.permutation(len(X))[:200]], np.float32)
    new_y = np.ascontiguousarray(r.integers(0, spec.out_dim, 200), np.int32)
    th0 = synthetic.particles(J, D, 61, std=0.1)
    out = []
    for mode in ("sync", "async"):
        ctx, _, _ = make_pair(spec, X, y, J, seed=61, precision=precision)
        try:
            S.smc_set_state(ctx, th0)
            S.smc_set_schedule(ctx, S.make_schedule("fb", 512, 512, 5))
            if mode == "sync":
                S.smc_upload_rows(ctx, 96, new_x, new_y)
            else:
                hx = torch.from_numpy(new_x).pin_memory()
                hy = torch.from_numpy(new_y).pin_memory()
                S.smc_upload_rows_async(ctx, 96, hx.numpy(), hy.numpy())
            S.smc_anneal_next(ctx)
            out.append(_eval(ctx, J, D))
        finally:
            S.smc_destroy(ctx)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_async_uploads_apply_in_order_and_at_set_schedule():
    spec, X, y = _case(S.PREC_FP32)
    J, D = 4, spec.n_params
    r = np.random.default_rng(62)
    a_x = np.ascontiguousarray(r.normal(size=(100, 16)), np.float32)
    b_x = np.ascontiguousarray(r.normal(size=(100, 16)), np.float32)
    lab = np.ascontiguousarray(r.integers(0, 4, 100), np.int32)
    th0 = synthetic.particles(J, D, 62, std=0.3)
    # reference: rows [0, 100) <- a, then rows [50, 150) <- b, uploaded synchronously
    ref, _, _ = make_pair(spec, X, y, J, seed=62)
    got, _, _ = make_pair(spec, X, y, J, seed=62)
    try:
        S.smc_set_state(ref, th0)
        S.smc_upload_rows(ref, 0, a_x, lab)
        S.smc_upload_rows(ref, 50, b_x, lab)
        S.smc_set_schedule(ref, S.make_schedule("fb", 512, 512, 5))
        S.smc_set_state(got, th0)
        S.smc_upload_rows_async(got, 0, a_x, lab)
        S.smc_upload_rows_async(got, 50, b_x, lab)
        S.smc_set_schedule(got, S.make_schedule("fb", 512, 512, 5))   # applies both, in order
        for u, v in zip(_eval(ref, J, D), _eval(got, J, D)):
            assert np.array_equal(u, v)
    finally:
        S.smc_destroy(ref)
        S.smc_destroy(got)


def test_prefetched_upload_is_not_seen_by_the_running_iteration():
    """The bench's pattern: step k's rows applied at its anneal, step k+1's rows
    uploaded before step k runs.  Step k must still see its own rows."""
    spec, X, y = _case(S.PREC_BF16)
    J, D = 4, spec.n_params
    th0 = synthetic.particles(J, D, 63, std=0.1)
    zeros = np.zeros((512, 784), np.float32)
    lab = np.zeros(512, np.int32)
    res = []
    for prefetch in (False, True):
        ctx, _, _ = make_pair(spec, X, y, J, seed=63, precision=S.PREC_BF16)
        try:
            S.smc_set_state(ctx, th0)
            S.smc_set_schedule(ctx, S.make_schedule("fb", 512, 512, 5))
            S.smc_anneal_next(ctx)
            if prefetch:
                S.smc_upload_rows_async(ctx, 0, zeros, lab)   # for the next iteration
            z = synthetic.normals((J, D), 63)
            S.smc_set_noise(ctx, z)
            st = S.smc_step(ctx, 0.002, 2)
            th, lw, lp = S.smc_get_state(ctx, J, D)
            res.append((th, lw, lp, st["ess"]))
        finally:
            S.smc_destroy(ctx)
    for u, v in zip(res[0], res[1]):
        assert np.array_equal(np.asarray(u), np.asarray(v))


def test_async_then_sync_upload_keep_call_order():
    """Rows staged asynchronously and then overwritten synchronously: the later
    (synchronous) rows win, as if both had been synchronous."""
    spec, X, y = _case(S.PREC_FP32)
    J, D = 4, spec.n_params
    r = np.random.default_rng(64)
    a_x = np.ascontiguousarray(r.normal(size=(100, 16)), np.float32)
    b_x = np.ascontiguousarray(r.normal(size=(100, 16)), np.float32)
    lab = np.ascontiguousarray(r.integers(0, 4, 100), np.int32)
    th0 = synthetic.particles(J, D, 64, std=0.3)
    ref, _, _ = make_pair(spec, X, y, J, seed=64)
    got, _, _ = make_pair(spec, X, y, J, seed=64)
    try:
        for ctx, mode in ((ref, "sync"), (got, "mixed")):
            S.smc_set_state(ctx, th0)
            if mode == "sync":
                S.smc_upload_rows(ctx, 0, a_x, lab)
            else:
                S.smc_upload_rows_async(ctx, 0, a_x, lab)
            S.smc_upload_rows(ctx, 50, b_x, lab)
            S.smc_set_schedule(ctx, S.make_schedule("fb", 512, 512, 5))
        for u, v in zip(_eval(ref, J, D), _eval(got, J, D)):
            assert np.array_equal(u, v)
    finally:
        S.smc_destroy(ref)
        S.smc_destroy(got)
