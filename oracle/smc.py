"""The data-annealed SMC sampler in float64 (oracle side; test infrastructure only).

Order of the calls (reading r9, the paper is silent): after `set_schedule`
(iteration 0, eq. init_weight) each iteration k runs
    anneal_next (target k; SDA moments from the previous step's weights)
    -> resample (if J_eff < J/2) -> step (move + reweight + normalise + ESS).  The target of iteration k is
    log pi_k(theta) = -|theta|^2 / (2 sigma^2) + sum_{i in D_k} c_i log p(y_i | theta)
with prior N(0, sigma^2 I) (reading r4) and per-row coefficients
    fixed schedules: c_i = N / M_k on D_k = rows [0, M_k)  (eq. approx-grad; reading r1
                     applies the same scale to the log-likelihood), or c_i = 1 when
                     the unscaled variant is selected;
    SDA:             c_i = 1 on the fully included rows, beta on the tempered block
                     (eq. sda_initial_target and the annealed target after it; reading r2).
Rows are taken in the order of one Fisher-Yates permutation drawn once (reading r3).
"""
from __future__ import annotations

import math

import numpy as np

from . import nn, schedules


# --------------------------------------------------------------------- weights
def normalise(logw):
    """Eq. normalise in log space: m = max log w, s = sum_j exp(log w_j - m)
    (summed left to right), w~_j = exp(log w_j - m) / s."""
    logw = np.asarray(logw, dtype=np.float64)
    m = max(logw)
    if not math.isfinite(m):
        raise FloatingPointError("every log-weight is -inf or nan")
    e = [math.exp(v - m) if math.isfinite(v) else 0.0 for v in logw]
    s = 0.0
    for v in e:
        s += v
    return np.array([v / s for v in e])


def ess(wn):
    """Eq. jeff: J_eff = 1 / sum_j w~_j^2."""
    return 1.0 / float(sum(w * w for w in wn))


# ------------------------------------------------------------------ resampling
def fixed_point_cumsum(wn):
    """Reading r11: normalised weights are quantised to q_j = round(w~_j 2^52)
    (round half to even) and summed exactly in 64-bit integers, so the
    cumulative weights C_j do not depend on summation order."""
    q = np.rint(np.asarray(wn, dtype=np.float64) * 2.0 ** 52).astype(np.uint64)
    return np.cumsum(q, dtype=np.uint64)


def _search(C, thresholds):
    Cf = C.astype(np.float64)            # exact: C_j < 2^53
    J = len(C)
    return np.minimum(np.searchsorted(Cf, np.asarray(thresholds), side="right"), J - 1).astype(np.int32)


def systematic_ancestors(wn, u: float):
    """Systematic resampling (Douc et al. 2005, cited in Sec. 2): one u in [0, 1),
    U_i = ((i + u) / J) * C_{J-1} in correctly rounded float64 steps, and
    a_i = min{j : C_j > U_i}, clamped to J - 1."""
    C = fixed_point_cumsum(wn)
    J = len(C)
    T = float(C[-1])
    t = [((float(i) + u) / float(J)) * T for i in range(J)]
    return _search(C, t)


def multinomial_ancestors(wn, uniforms):
    """Multinomial resampling (Sec. 2, "we use multinomial resampling"): J
    independent uniforms, sorted ascending, U_i = u_(i) * C_{J-1}, same search."""
    C = fixed_point_cumsum(wn)
    T = float(C[-1])
    t = [float(v) * T for v in np.sort(np.asarray(uniforms, dtype=np.float64))]
    return _search(C, t)


# -------------------------------------------------------------------- leapfrog
def leapfrog(target, theta, P, h: float, S: int, inv_mass):
    """S leapfrog steps (Sec. 2.1, eqs. mom_first, pos_update, mom_second) with
    mass matrix M = diag(1 / inv_mass):
        P <- P + h/2 grad log pi(theta);  theta <- theta + h M^-1 P;
        P <- P + h/2 grad log pi(theta).
    `target(theta)` returns (log pi, grad log pi, ...).  Returns the final
    (theta, P) and the target's output at the final theta."""
    theta = np.array(theta, dtype=np.float64)
    P = np.array(P, dtype=np.float64)
    out = target(theta)
    for _ in range(S):
        P = P + 0.5 * h * out[1]
        theta = theta + h * inv_mass * P
        out = target(theta)
        P = P + 0.5 * h * out[1]
    return theta, P, out


# --------------------------------------------------------------------- sampler
class Sampler:
    """FP64 SMC sampler over J networks.  Randomness is injected: initial
    particles, standard-normal momentum draws and resampling uniforms are
    arguments, so the CUDA path can be driven with the same draws."""

    def __init__(self, spec: nn.Spec, X, y, J: int, perm, prior_sigma: float = 1.0,
                 scaled: bool = True):
        perm = np.asarray(perm, dtype=np.int64)
        self.spec = spec
        self.X = np.asarray(X, dtype=np.float64)[perm]
        self.y = np.asarray(y)[perm]
        self.N = self.X.shape[0]
        self.J = J
        self.D = spec.n_params
        self.sigma = prior_sigma
        self.scaled = scaled

    # ---------------------------------------------------------------- target
    def regions(self):
        """(rows_a, coef_a, rows_b, coef_b): rows [0, rows_a) carry coef_a, the
        next rows_b rows carry coef_b."""
        if self.kind == schedules.SDA:
            s = self.sda
            return s.m_full, 1.0, s.block, s.beta
        M = self.M
        return M, (self.N / M if self.scaled else 1.0), 0, 0.0

    def rows(self):
        """Indices (annealed order) of the current subset: a prefix, or for the
        fresh schedules M consecutive rows from `schedules.subset_start`,
        wrapping past N."""
        ra, _, rb, _ = self.regions()
        n = ra + rb
        start = 0 if self.kind == schedules.SDA else schedules.subset_start(self.kind, self.k, self.N, n)
        return (start + np.arange(n)) % self.N

    def target(self, theta):
        """log pi_k(theta), its gradient, and the unweighted log-likelihood sums
        over the two row regions (L_a, L_b)."""
        ra, ca, rb, cb = self.regions()
        n = ra + rb
        coef = np.concatenate([np.full(ra, ca), np.full(rb, cb)])
        idx = self.rows()
        ll, g = nn.loglik_grad(self.spec, theta, self.X[idx], self.y[idx], coef)
        la, lb = float(ll[:ra].sum()), float(ll[ra:n].sum())
        logpi = -0.5 * float(theta @ theta) / self.sigma ** 2 + ca * la + cb * lb
        return logpi, g - theta / self.sigma ** 2, la, lb

    # ------------------------------------------------------------ iteration 0
    def set_schedule(self, kind: str, C: int, kappa: int, K: int, theta0,
                     beta0: float = 0.1, beta_reinit: float = 0.1, delta_s: float = 1.0):
        """Iteration 0: theta_0 ~ q_0 (injected), w_0 = pi_0(theta_0) / q_0(theta_0)
        (eq. init_weight); the prior cancels, leaving sum_i c_i log p(y_i|theta_0)."""
        self.kind, self.C, self.kappa, self.K, self.k = kind, C, kappa, K, 0
        if kind == schedules.SDA:
            self.sda = schedules.SDAState(self.N, C, kappa, beta0, beta_reinit, delta_s)
        else:
            self.M = schedules.subset_size(kind, 0, self.N, C, kappa, K)
        self.theta = np.array(theta0, dtype=np.float64)
        self.logpi = np.empty(self.J)
        self.la = np.empty(self.J)
        self.lb = np.empty(self.J)
        for j in range(self.J):
            self.logpi[j], _, self.la[j], self.lb[j] = self.target(self.theta[j])
        ra, ca, rb, cb = self.regions()
        self.logw = ca * self.la + cb * self.lb
        self.wn = normalise(self.logw)
        self.ess = ess(self.wn)

    @property
    def subset_rows(self) -> int:
        ra, _, rb, _ = self.regions()
        return ra + rb

    # ------------------------------------------------------------------ move
    def step(self, h: float, S: int, z, inv_mass=None):
        """Leapfrog move under the current target pi_k, then reweight.

        Momentum P^0 ~ N(0, M) is sqrt(M) z for injected standard normals z.
        Each of the S steps (eqs. mom_first, pos_update, mom_second):
            P <- P + h/2 grad log pi(theta);  theta <- theta + h M^-1 P;
            P <- P + h/2 grad log pi(theta).
        The gradient at the start is taken under pi_k (reading r6).  S = 1 is
        Langevin dynamics (Sec. 2.1).  h may be one value or one per particle and
        inv_mass one [D] vector or one per particle ([J, D]): each particle's
        weight then uses its own kernel.  The L-kernel is the reversed-momentum
        kernel, so (eq. weight_update_fp, reading r7)
            log w_k = log w_{k-1} + log pi_k(theta_k) - log pi_{k-1}(theta_{k-1})
                      + log N(-P_k; 0, M) - log N(P^0; 0, M),
        the Gaussian normalisers cancelling.  A non-finite log pi_k gives
        log w_k = -inf (reading r8)."""
        inv_mass = np.ones(self.D) if inv_mass is None else np.asarray(inv_mass, dtype=np.float64)
        hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (self.J,))
        ims = np.broadcast_to(inv_mass, (self.J, self.D))
        z = np.asarray(z, dtype=np.float64)
        for j in range(self.J):
            im = ims[j]
            P0 = z[j] / np.sqrt(im)
            theta, P, (logpi, _, la, lb) = leapfrog(self.target, self.theta[j], P0, float(hs[j]), S, im)
            ke0 = 0.5 * float(P0 @ (im * P0))
            ke1 = 0.5 * float(P @ (im * P))
            inc = logpi - self.logpi[j] - ke1 + ke0
            self.logw[j] = self.logw[j] + inc if math.isfinite(inc) else -math.inf
            self.theta[j], self.logpi[j], self.la[j], self.lb[j] = theta, logpi, la, lb
        self.wn = normalise(self.logw)
        self.ess = ess(self.wn)

    # ----------------------------------------------------------------- anneal
    def anneal_next(self) -> bool:
        """Advance to the target of iteration k+1.  Fixed schedules follow
        `schedules.subset_size`; SDA uses the normalised weights of the current
        (pre-resampling) particles and Omega = -L_a, Omega_hat = -L_b at the
        current particles.  The cached log pi stays under the old target, as
        the weight update of the next move needs.  Returns True when rows
        were added to the subset."""
        before = self.subset_rows
        self.k += 1
        if self.kind == schedules.SDA:
            self.sda.advance(self.wn, -self.la, -self.lb)
        else:
            self.M = schedules.subset_size(self.kind, self.k, self.N, self.C, self.kappa, self.K)
        return self.subset_rows > before

    # --------------------------------------------------------------- resample
    def resample(self, u=None, uniforms=None, kind="systematic", force=False) -> bool:
        """Resample when J_eff < J/2 (Sec. 2, strict) or when forced; weights
        are then reset to 1/J."""
        if not force and not self.ess < self.J / 2:
            return False
        if kind == "systematic":
            anc = systematic_ancestors(self.wn, u)
        else:
            anc = multinomial_ancestors(self.wn, uniforms)
        self.ancestors = anc
        self.theta = self.theta[anc].copy()
        self.logpi = self.logpi[anc].copy()
        self.la, self.lb = self.la[anc].copy(), self.lb[anc].copy()
        self.logw = np.full(self.J, -math.log(self.J))
        self.wn = normalise(self.logw)
        self.ess = ess(self.wn)
        return True

    # ------------------------------------------------------------- predictive
    def predict(self, Xtest):
        """Weighted posterior estimate (Sec. 2, E_pi[f] ~ sum_j w~_j f(theta_j))
        with f the predictive class probabilities."""
        out = np.zeros((Xtest.shape[0], self.spec.out_dim))
        for j in range(self.J):
            out += self.wn[j] * nn.predictive_probs(self.spec, self.theta[j], Xtest)
        return out


def accuracy_nll(probs, y):
    """Test accuracy (argmax, lowest class index on ties) and mean negative
    log predictive probability."""
    y = np.asarray(y, dtype=np.int64)
    pred = np.argmax(probs, axis=1)
    acc = float(np.mean(pred == y))
    nll = float(-np.mean(np.log(np.maximum(probs[np.arange(len(y)), y], 1e-300))))
    return acc, nll
