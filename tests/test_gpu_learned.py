"""GPU tests of the learned proposal (the build's own addition, not in the
paper), through the C ABI, against the FP64 oracle (oracle/learned.py):
network gradient and Adam training, features, BF16 inference, exactness of a
learned move (per-particle kernels in the weights), the untrained network
reducing to the plain proposal, candidate scoring, and the gain of a trained
network over the plain proposal on the same problem."""
import numpy as np
import pytest

import synthetic
from oracle import learned as OL, nn, rng, smc as osmc

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402
from tests._gpu import make_pair, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

MLP0 = nn.Spec([("dense", 16, 32), ("dense", 32, 4)], (16,), nn.TANH)


def _bf16(x):
    t = torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def _seg_layout(spec):
    sizes, isb = [], []
    for shp in spec.shapes:
        for k, s in enumerate(shp):
            sizes.append(int(np.prod(s)))
            isb.append(k == 1)
    return sizes, isb


def test_network_gradient_matches_oracle():
    S.load()
    r = np.random.default_rng(0)
    p = r.normal(scale=0.3, size=OL.N_PARAMS)
    F, T = r.normal(size=(300, 8)), r.normal(size=(300, 2))
    loss, g = S.smc_k_learned_loss_grad(F, T, p)
    rl, rg = OL.loss_grad(p.astype(np.float32).astype(np.float64), F.astype(np.float32), T.astype(np.float32))
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    assert rel_err(g, rg) < 1e-5


def test_adam_training_matches_oracle():
    X, y = synthetic.gaussian_mixture(64, seed=1)
    ctx, _, _ = make_pair(MLP0, X, y, 4, seed=1)
    try:
        r = np.random.default_rng(2)
        F = r.normal(size=(500, 8)).astype(np.float32)
        T = np.stack([np.tanh(F[:, 0]) - 0.3 * F[:, 3], 0.2 * F[:, 5]], axis=1).astype(np.float32)
        p0 = (0.3 * r.normal(size=OL.N_PARAMS)).astype(np.float32)
        S.smc_learned_params(ctx, p0)
        S.smc_learned_load_data(ctx, F, T)
        loss = S.smc_learned_train(ctx, 25, 0.01)
        p1 = S.smc_learned_params(ctx)
        rp, rloss = OL.adam(p0.astype(np.float64), F, T, 25, 0.01)
        assert rel_err(p1 - p0, rp - p0) < 1e-3
        assert abs(loss - rloss) <= 1e-3 * rloss
    finally:
        S.smc_destroy(ctx)


def test_untrained_network_is_the_plain_proposal_bitwise():
    X, y = synthetic.gaussian_mixture(256, seed=3)
    outs = []
    for prop in [S.PROPOSAL_PLAIN, S.PROPOSAL_LEARNED]:
        ctx, _, _ = make_pair(MLP0, X, y, 8, seed=3)
        try:
            S.smc_set_schedule(ctx, S.make_schedule("fb", 256, 256, 5))
            S.smc_set_noise(ctx, synthetic.normals((8, MLP0.n_params), 4))
            st = S.smc_step(ctx, 0.01, 3, prop)
            assert st["proposal_used"] == prop and st["h_used"] == 0.01
            outs.append(S.smc_get_state(ctx, 8, MLP0.n_params))
        finally:
            S.smc_destroy(ctx)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_learned_move_matches_oracle():
    """Features (FP32 stats) and BF16 inference against the FP64 oracle, then
    the move with that proposal: each particle's weight uses the kernel it
    moved with (eq. weight_update_fp with N(.; 0, M))."""
    N, J = 512, 16
    X, y = synthetic.gaussian_mixture(N, seed=5)
    ctx, orc, _ = make_pair(MLP0, X, y, J, seed=5)
    try:
        th0 = synthetic.particles(J, MLP0.n_params, 5, std=0.5)
        S.smc_set_state(ctx, th0)
        S.smc_set_schedule(ctx, S.make_schedule("linear", 128, 128, 10))
        orc.set_schedule("linear", 128, 128, 10, th0)
        r = np.random.default_rng(6)
        params = _bf16(0.3 * r.normal(size=OL.N_PARAMS))        # exactly representable in BF16
        S.smc_learned_params(ctx, params)
        z = synthetic.normals((J, MLP0.n_params), 7)
        S.smc_set_noise(ctx, z)
        h = 0.01
        st = S.smc_step(ctx, h, 2, S.PROPOSAL_LEARNED)
        feats, cand, _ = S.smc_learned_last(ctx)
        # oracle features at the starting particles
        sizes, isb = _seg_layout(MLP0)
        grad = np.stack([orc.target(orc.theta[j])[1] for j in range(J)])
        rf = OL.features(orc.theta, grad, orc.wn, sizes, isb, orc.ess, orc.subset_rows / orc.N, 1.0)
        assert np.allclose(feats, rf, rtol=1e-4, atol=1e-4)
        out, _ = OL.forward(params, rf)
        inv_mass, h_l = OL.proposal(out, h)
        assert np.allclose(np.exp(cand[0, :-1]), inv_mass, rtol=2e-2)
        assert abs(st["h_used"] - h_l) <= 2e-2 * h_l
        # the move under the oracle's own proposal
        im = np.concatenate([np.full(sz, m) for sz, m in zip(sizes, inv_mass)])
        orc.step(h_l, 2, z, inv_mass=im)
        th, lw, lp = S.smc_get_state(ctx, J, MLP0.n_params)
        disp = [rel_err(th[j] - th0[j], orc.theta[j] - th0[j]) for j in range(J)]
        assert max(disp) < 5e-2
        assert np.allclose(lp, orc.logpi, rtol=1e-3)
    finally:
        S.smc_destroy(ctx)


def test_exploration_scores_and_rows():
    N, J, G = 512, 32, 4
    X, y = synthetic.gaussian_mixture(N, seed=8)
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=8)
    try:
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 10))
        th0, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
        st = S.smc_step(ctx, 0.01, 2, S.PROPOSAL_EXPLORE, groups=G, explore_sigma=0.5)
        assert st["proposal_used"] == S.PROPOSAL_EXPLORE
        th1, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
        wn = S.smc_get_weights(ctx, J)
        F, cand, scores = S.smc_learned_last(ctx, G)
        groups = [list(range((g * J + G - 1) // G, ((g + 1) * J + G - 1) // G)) for g in range(G)]
        ref = OL.group_scores(th0, th1, wn, groups)
        assert np.allclose(scores[:G], ref, rtol=1e-4)
        best = int(scores[G])
        assert best == int(np.argmax(ref))
        Fd, Td = S.smc_learned_data(ctx)
        ns = S.smc_num_segments(ctx)
        assert Fd.shape == (ns, 8)
        assert np.allclose(Fd, F) and np.allclose(Td[:, 0], cand[best, :ns]) and np.allclose(Td[:, 1], cand[best, ns])
    finally:
        S.smc_destroy(ctx)


def test_trained_network_gains_over_plain():
    """Train on the sampler's own exploratory iterations, then compare the
    learned and plain proposals from the same state over the same iterations:
    the learned one must move the particles further (mean squared jump) while
    keeping the ESS at least half of the plain one."""
    N, J, h = 1024, 64, 0.002
    X, y = synthetic.gaussian_mixture(N, seed=9)
    ctx, _, _ = make_pair(MLP0, X, y, J, seed=9)
    try:
        S.smc_set_schedule(ctx, S.make_schedule("fb", N, N, 100))
        for rnd in range(3):
            for _ in range(12):
                S.smc_step(ctx, h, 2, S.PROPOSAL_EXPLORE, groups=8, explore_sigma=0.6)
                S.smc_resample(ctx)
            S.smc_learned_train(ctx, 200, 0.01)
        start = S.smc_get_state(ctx, J, MLP0.n_params)
        res = {}
        for prop in [S.PROPOSAL_PLAIN, S.PROPOSAL_LEARNED]:
            S.smc_set_state(ctx, *start)
            jumps, esses = [], []
            for k in range(6):
                before, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
                S.smc_set_noise(ctx, synthetic.normals((J, MLP0.n_params), 300 + k))
                st = S.smc_step(ctx, h, 2, prop)
                after, _, _ = S.smc_get_state(ctx, J, MLP0.n_params)
                jumps.append(np.mean(np.sum((after - before) ** 2, axis=1)))
                esses.append(st["ess"])
            res[prop] = (np.mean(jumps), np.mean(esses))
        (jp, ep), (jl, el) = res[S.PROPOSAL_PLAIN], res[S.PROPOSAL_LEARNED]
        assert jl > 2.0 * jp, res
        assert el > 0.5 * ep, res
    finally:
        S.smc_destroy(ctx)
