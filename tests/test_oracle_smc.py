"""Pins of the oracle sampler (CPU only): invariants of normalisation, ESS and
resampling, exact rational brute force for systematic resampling, the
harmonic-oscillator closed form and reversibility of the leapfrog, the h = 0
data-annealing reweight, and convergence to the closed-form posterior of a
linear-Gaussian model."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic
from oracle import nn, rng, schedules, smc


# ------------------------------------------------------------- normalise / ESS
def test_normalise_and_ess_invariants():
    r = np.random.default_rng(0)
    for J in [1, 2, 7, 256]:
        logw = r.normal(scale=20.0, size=J)
        wn = smc.normalise(logw)
        assert abs(wn.sum() - 1.0) <= 1e-15 * J + 1e-15
        e = smc.ess(wn)
        assert 1.0 - 1e-12 <= e <= J * (1 + 1e-12)
        assert np.allclose(smc.normalise(logw + 123.4), wn, rtol=1e-12)  # shift invariance
    assert abs(smc.ess(smc.normalise(np.zeros(64))) - 64.0) < 1e-12
    one_hot = np.full(10, -np.inf)
    one_hot[3] = 0.0
    assert smc.ess(smc.normalise(one_hot)) == 1.0
    with pytest.raises(FloatingPointError):
        smc.normalise(np.full(4, -np.inf))


# ----------------------------------------------------------------- resampling
def test_systematic_counts_floor_ceil():
    for seed in range(20):
        J = [3, 16, 100, 1024][seed % 4]
        wn = synthetic.normalised_weights(J, seed)
        u = synthetic.uniforms(1, seed)[0]
        a = smc.systematic_ancestors(wn, u)
        assert len(a) == J and np.all(np.diff(a) >= 0)
        n = np.bincount(a, minlength=J)
        assert np.all(n >= np.floor(J * wn) - 0) and np.all(n <= np.ceil(J * wn))


def test_systematic_exact_rational_bruteforce():
    # For J <= 6 compute each ancestor from the definition in exact rationals.
    for seed in range(30):
        J = 2 + seed % 5
        wn = synthetic.normalised_weights(J, 100 + seed, spread=1.0)
        u = synthetic.uniforms(1, 200 + seed)[0]
        q = [int(np.rint(w * 2.0 ** 52)) for w in wn]
        C = np.cumsum(q).tolist()
        T = C[-1]
        got = smc.systematic_ancestors(wn, u).tolist()
        for i in range(J):
            t = Fraction(((float(i) + u) / float(J)) * float(T))   # the float64 threshold
            exact = next((j for j in range(J) if Fraction(C[j]) > t), J - 1)
            assert got[i] == exact


def test_systematic_unbiased_over_u_grid():
    J = 8
    wn = synthetic.normalised_weights(J, 5)
    grid = (np.arange(20000) + 0.5) / 20000
    mean_counts = np.zeros(J)
    for u in grid:
        mean_counts += np.bincount(smc.systematic_ancestors(wn, u), minlength=J)
    mean_counts /= len(grid)
    assert np.allclose(mean_counts, J * wn, atol=2e-3)


def test_multinomial_chi_square():
    J = 6
    wn = synthetic.normalised_weights(J, 9, spread=0.7)
    counts = np.zeros(J)
    draws = 0
    for rep in range(2000):
        a = smc.multinomial_ancestors(wn, synthetic.uniforms(J, 1000 + rep))
        assert np.all(np.diff(a) >= 0)
        counts += np.bincount(a, minlength=J)
        draws += J
    expect = draws * wn
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 30.0      # 5 dof


# ------------------------------------------------------------------- leapfrog
def _gaussian_target(lam, mu):
    def target(theta):
        d = theta - mu
        return -0.5 * float(d @ (lam * d)), -lam * d
    return target


def test_leapfrog_converges_to_harmonic_flow():
    # 1-d Gaussian target N(mu, 1/lam): Hamiltonian flow is a rotation with
    # angular frequency sqrt(lam); leapfrog error at fixed time t = S h is O(h^2).
    lam, mu, th0, p0, t = np.array([2.5]), np.array([0.3]), np.array([1.1]), np.array([-0.4]), 0.6
    w = math.sqrt(lam[0])
    exact = mu[0] + (th0[0] - mu[0]) * math.cos(w * t) + p0[0] / w * math.sin(w * t)
    errs = []
    for S in [6, 12, 24, 48]:
        th, _, _ = smc.leapfrog(_gaussian_target(lam, mu), th0, p0, t / S, S, np.ones(1))
        errs.append(abs(th[0] - exact))
    slopes = [math.log(errs[i] / errs[i + 1], 2) for i in range(3)]
    assert all(1.9 < s < 2.1 for s in slopes), slopes


def test_leapfrog_reversible_and_energy_error_order():
    r = np.random.default_rng(3)
    lam, mu = r.uniform(0.5, 3.0, 5), r.normal(size=5)
    th0, p0 = r.normal(size=5), r.normal(size=5)
    inv_mass = r.uniform(0.5, 2.0, 5)
    tgt = _gaussian_target(lam, mu)
    th1, p1, _ = smc.leapfrog(tgt, th0, p0, 0.05, 7, inv_mass)
    th2, p2, _ = smc.leapfrog(tgt, th1, -p1, 0.05, 7, inv_mass)
    assert np.allclose(th2, th0, atol=1e-12) and np.allclose(-p2, p0, atol=1e-12)

    def dH(h):
        th, p, out = smc.leapfrog(tgt, th0, p0, h, int(round(0.4 / h)), inv_mass)
        H0 = -tgt(th0)[0] + 0.5 * p0 @ (inv_mass * p0)
        return abs(-out[0] + 0.5 * p @ (inv_mass * p) - H0)
    e = [dH(h) for h in (0.04, 0.02, 0.01)]
    assert 3.0 < e[0] / e[1] < 5.0 and 3.0 < e[1] / e[2] < 5.0


# ----------------------------------------------------------- sampler (MLP)
def _small_problem(J=5, N=64, seed=0):
    X, y = synthetic.gaussian_mixture(N, d=4, n_classes=3, seed=seed)
    spec = nn.Spec([("dense", 4, 6), ("dense", 6, 3)], (4,), nn.TANH)
    perm = rng.fisher_yates_permutation(N, seed)
    theta0 = synthetic.particles(J, spec.n_params, seed)
    return spec, X, y, perm, theta0


def test_initial_weights_are_scaled_loglik():
    spec, X, y, perm, theta0 = _small_problem()
    s = smc.Sampler(spec, X, y, 5, perm)
    s.set_schedule("linear", 16, 16, 10, theta0)
    Xp, yp = X[perm].astype(np.float64), y[perm]
    for j in range(5):
        z, _ = nn.forward(spec, theta0[j].astype(np.float64), Xp[:16])
        ll = nn.per_sample_loglik(spec, z, yp[:16])
        assert abs(s.logw[j] - (64 / 16) * ll.sum()) < 1e-9


def test_zero_step_is_pure_annealing_reweight():
    # h = 0: the move is the identity and the kinetic terms cancel, so the
    # increment is log pi_k(theta) - log pi_{k-1}(theta) (special case p5).
    spec, X, y, perm, theta0 = _small_problem()
    s = smc.Sampler(spec, X, y, 5, perm)
    s.set_schedule("linear", 16, 16, 10, theta0)
    logw0 = s.logw.copy()
    s.anneal_next()
    s.step(0.0, 3, synthetic.normals((5, spec.n_params), 1))
    Xp, yp = X[perm].astype(np.float64), y[perm]
    for j in range(5):
        z, _ = nn.forward(spec, theta0[j].astype(np.float64), Xp[:32])
        ll = nn.per_sample_loglik(spec, z, yp[:32])
        expect = (64 / 32) * ll[:32].sum() - (64 / 16) * ll[:16].sum()
        assert abs((s.logw[j] - logw0[j]) - expect) < 1e-9
    assert np.array_equal(s.theta, theta0.astype(np.float64))


def test_resample_resets_weights_and_keeps_count():
    spec, X, y, perm, theta0 = _small_problem(J=8)
    s = smc.Sampler(spec, X, y, 8, perm)
    s.set_schedule("fb", 16, 16, 10, theta0)
    did = s.resample(u=0.37, force=True)
    assert did and s.theta.shape == (8, spec.n_params)
    assert np.allclose(s.logw, -math.log(8)) and abs(s.ess - 8) < 1e-9
    for i, a in enumerate(s.ancestors):
        assert np.array_equal(s.theta[i], theta0[a].astype(np.float64))


def test_predictive_identical_particles_is_softmax():
    spec, X, y, perm, theta0 = _small_problem(J=4)
    same = np.repeat(theta0[:1], 4, axis=0)
    s = smc.Sampler(spec, X, y, 4, perm)
    s.set_schedule("fb", 16, 16, 10, same)
    probs = s.predict(X[:10].astype(np.float64))
    assert np.allclose(probs, nn.predictive_probs(spec, same[0].astype(np.float64), X[:10]), rtol=1e-12)
    assert np.allclose(probs.sum(axis=1), 1.0)


# ---------------------------------------------- closed-form posterior (p1)
@pytest.mark.parametrize("seed", [0, 1])
def test_linear_gaussian_smc_matches_closed_form(seed):
    d, N, J, sn = 2, 40, 400, 0.5
    X, yv, _ = synthetic.linear_gaussian(N, d, seed=seed, noise_std=sn)
    spec = nn.Spec([("dense", d, 1)], (d,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=sn)
    perm = rng.fisher_yates_permutation(N, seed)
    theta0 = synthetic.particles(J, spec.n_params, 50 + seed)
    s = smc.Sampler(spec, X, yv, J, perm, prior_sigma=1.0)
    K = 10
    s.set_schedule("linear", 5, 5, K, theta0)
    g = rng.SplitMix64(seed)
    for k in range(1, K):
        s.anneal_next()
        s.resample(u=g.next_double())
        s.step(0.05, 3, synthetic.normals((J, spec.n_params), 1000 * seed + k))
    assert s.subset_rows == N
    # posterior over (w, b): append a constant input column for the bias
    Xb = np.concatenate([X[perm].astype(np.float64), np.ones((N, 1))], axis=1)
    mu, Sig = nn.linear_gaussian_posterior(Xb, yv[perm], np.ones(N), 1.0, sn)
    m = s.wn @ s.theta
    se = np.sqrt(np.diag(Sig) / s.ess) * 3.0       # MC error with generous inflation
    assert np.all(np.abs(m - mu) < 4.0 * se + 1e-3), (m, mu, se)
    cov = (s.theta - m).T @ (s.wn[:, None] * (s.theta - m))
    assert np.allclose(np.diag(cov), np.diag(Sig), rtol=0.5)


def test_weight_increment_is_energy_error_under_fixed_target():
    # With a fixed target (full batch), eq. weight_update_fp gives
    # log w_k - log w_{k-1} = -(H_k - H_{k-1}), H = -log pi + P^T M^-1 P / 2,
    # which leapfrog keeps O(h^2) at fixed integration time; a dropped or
    # sign-flipped kinetic term would leave an O(1) or O(h) increment.
    d, N, sn = 2, 30, 0.5
    X, yv, _ = synthetic.linear_gaussian(N, d, seed=4, noise_std=sn)
    spec = nn.Spec([("dense", d, 1)], (d,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=sn)
    perm = rng.fisher_yates_permutation(N, 4)
    theta0 = synthetic.particles(3, spec.n_params, 7)
    z = synthetic.normals((3, spec.n_params), 8)
    incs = []
    for h in (0.02, 0.01, 0.005):
        s = smc.Sampler(spec, X, yv, 3, perm)
        s.set_schedule("fb", N, N, 5, theta0)
        before = s.logw.copy()
        s.step(h, int(round(0.2 / h)), z)
        incs.append(np.max(np.abs(s.logw - before)))
    assert 3.0 < incs[0] / incs[1] < 5.0 and 3.0 < incs[1] / incs[2] < 5.0, incs


def test_fresh_batch_target_is_the_prefix_target_of_rotated_data():
    """The fresh-batch target at iteration k equals the ordinary prefix target on
    the same data rotated so that the batch starts at row 0 (the window is the
    only difference between the two readings of Constant)."""
    spec = nn.Spec([("dense", 4, 3), ("dense", 3, 2)], (4,), nn.TANH)
    X, y = synthetic.gaussian_mixture(37, d=4, n_classes=2, seed=3)
    perm = np.arange(37)
    th = synthetic.particles(1, spec.n_params, 3, std=0.5)
    fresh = smc.Sampler(spec, X, y, 1, perm)
    fresh.set_schedule("constant_fresh", 10, 10, 20, th)
    for _ in range(4):
        fresh.anneal_next()                      # k = 4: rows 40..49 mod 37 = 3..12
    start = 40 % 37
    plain = smc.Sampler(spec, np.roll(X, -start, axis=0), np.roll(y, -start), 1, perm)
    plain.set_schedule("constant", 10, 10, 20, th)
    a, b = fresh.target(th[0]), plain.target(th[0])
    assert np.isclose(a[0], b[0], rtol=1e-13) and np.allclose(a[1], b[1], rtol=1e-12, atol=1e-14)
    assert list(fresh.rows()) == list(range(3, 13))


# ------------------------------------------- SDA wiring of the sampler (p1, p7)
def _gauss_nll(Xb, yp, theta, lo, hi, sn):
    """-sum_{i in [lo, hi)} log N(y_i; x_i . theta, sn^2), written out here
    (not through the oracle's network code)."""
    r = yp[lo:hi] - Xb[lo:hi] @ theta
    return float(0.5 * np.sum(r * r) / sn ** 2 + (hi - lo) * math.log(math.sqrt(2.0 * math.pi) * sn))


def _tempered_check(s, Xb, yp, coef, sn):
    """Weighted mean of the particles against the closed-form posterior whose
    likelihood exponents are `coef` (per row), within Monte Carlo error."""
    mu, Sig = nn.linear_gaussian_posterior(Xb, yp, coef, 1.0, sn)
    m = s.wn @ s.theta
    se = np.sqrt(np.diag(Sig) / s.ess) * 3.0
    return bool(np.all(np.abs(m - mu) < 4.0 * se + 1e-3))


@pytest.mark.parametrize("seed", [2, 3])
def test_sda_sampler_tracks_tempered_posteriors_and_beta_rule(seed):
    """SDA inside the sampler (Sec. 3.1, eq. sda_initial_target and the
    annealed target after it) on a linear-Gaussian model, where every target is
    Gaussian.  (i) Before each temperature update the next beta is recomputed
    from the pre-resampling weights with Omega (fully included rows) and
    Omega_hat (tempered block) evaluated here from scratch: beta moves by
    dS / |Var(Omega_hat) + Cov(Omega, Omega_hat)|, clipped to 1.  A swap of
    Omega and Omega_hat, a sign slip or stale moments in the sampler's wiring
    changes that value.  (ii) After each move the weighted particle mean
    matches the closed-form posterior with exponent 1 on the fully included
    rows, beta on the block and 0 elsewhere.  A planted mistake in (ii) (the
    block at exponent 1 while beta < 1) must be rejected somewhere along the run."""
    d, N, J, sn, K = 2, 40, 400, 0.5, 40
    X, yv, _ = synthetic.linear_gaussian(N, d, seed=seed, noise_std=sn)
    spec = nn.Spec([("dense", d, 1)], (d,), nn.IDENTITY, nn.GAUSSIAN, noise_sigma=sn)
    perm = rng.fisher_yates_permutation(N, seed)
    s = smc.Sampler(spec, X, yv, J, perm, prior_sigma=1.0)
    s.set_schedule("sda", 5, 5, K, synthetic.particles(J, spec.n_params, 60 + seed))
    Xb = np.concatenate([X[perm].astype(np.float64), np.ones((N, 1))], axis=1)
    yp = yv[perm].astype(np.float64)
    g = rng.SplitMix64(seed)
    n_beta, n_append, n_planted_rejected = 0, 0, 0
    for k in range(1, K):
        full, block, beta = s.sda.m_full, s.sda.block, s.sda.beta
        w = s.wn.copy()
        om = np.array([_gauss_nll(Xb, yp, th, 0, full, sn) for th in s.theta])
        oh = np.array([_gauss_nll(Xb, yp, th, full, full + block, sn) for th in s.theta])
        appended = s.anneal_next()
        if beta < 1.0:
            e = lambda a: float(np.dot(w, a))
            den = (e(oh * oh) - e(oh) ** 2) + (e(om * oh) - e(om) * e(oh))
            expect = min(beta + 1.0 / abs(den), 1.0)
            assert not appended and s.sda.beta == pytest.approx(expect, rel=1e-9), (k, s.sda.beta, expect)
            n_beta += 1
        elif full + block < N:
            assert appended and s.sda.m_full == full + block and s.sda.beta == 0.1
            n_append += 1
        s.resample(u=g.next_double())
        s.step(0.05, 3, synthetic.normals((J, spec.n_params), 500 * seed + k))
        full, block, beta = s.sda.m_full, s.sda.block, s.sda.beta
        coef = np.concatenate([np.ones(full), np.full(block, beta), np.zeros(N - full - block)])
        assert _tempered_check(s, Xb, yp, coef, sn), (k, full, block, beta)
        if block and beta < 0.5:
            wrong = np.concatenate([np.ones(full + block), np.zeros(N - full - block)])
            n_planted_rejected += not _tempered_check(s, Xb, yp, wrong, sn)
    assert n_beta >= 8 and n_append == 7 and s.subset_rows == N
    assert n_planted_rejected >= 1
