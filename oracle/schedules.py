"""Data-annealing schedules (oracle side; test infrastructure only).

Sec. 3.1 "Annealing Schemes": C is the initial batch, kappa the mini-batch
increment, K the number of iterations, M_k the subset size at iteration k with
C <= M_k <= N.  All fixed schedules are integer arithmetic; the condition
"k < 0.9K" is evaluated exactly as 10 k < 9 K.

Smooth data annealing (SDA, Sec. 3.1, eqs. sda_initial_target,
beta_initial_data_k, beta_annealed_k and the moment equations after them)
tempers the newest block by beta and raises beta so that the entropy changes
by Delta S per iteration.
"""
from __future__ import annotations

import math

CONSTANT, FULL_BATCH, CTR, LINEAR, AUTOMATED, SDA = "constant", "fb", "ctr", "linear", "automated", "sda"
CONSTANT_FRESH, CTR_FRESH = "constant_fresh", "ctr_fresh"
FIXED_KINDS = (CONSTANT, FULL_BATCH, CTR, LINEAR, AUTOMATED, CONSTANT_FRESH, CTR_FRESH)
FRESH_KINDS = (CONSTANT_FRESH, CTR_FRESH)


def _late(k: int, K: int) -> bool:
    """True when k >= 0.9 K, i.e. not (k < 0.9K), in exact integers."""
    return 10 * k >= 9 * K


def automated_increment(N: int, C: int, K: int) -> int:
    """floor((N - C) / (0.9 K)) of the Automated scheme, as floor(10 (N-C) / (9K))."""
    return (10 * (N - C)) // (9 * K)


def subset_size(kind: str, k: int, N: int, C: int, kappa: int, K: int) -> int:
    """M_k for the five fixed schedules of Sec. 3.1.

    Constant:  M_k = C                                   (eq. Constant)
    FB:        M_k = N                                   (eq. Full-batch)
    CTR:       M_k = C if k < 0.9K else N                 (eq. Constant-to-refine)
    Linear:    M_k = kappa k + C if k < 0.9K else N       (eq. Linear), capped at N
    Automated: M_k = C + floor((N-C)/(0.9K)) k if k < 0.9K else N (eq. Automated),
               rounded to the nearest multiple of kappa (ties upward) because data
               are appended in whole mini-batches, then kept within [C, N].
    """
    C = min(C, N)
    if kind in (CONSTANT, CONSTANT_FRESH):
        return C
    if kind == FULL_BATCH:
        return N
    if kind in (CTR, CTR_FRESH):
        return N if _late(k, K) else C
    if kind == LINEAR:
        return N if _late(k, K) else min(N, kappa * k + C)
    if kind == AUTOMATED:
        if _late(k, K):
            return N
        m = C + automated_increment(N, C, K) * k
        m = ((2 * m + kappa) // (2 * kappa)) * kappa     # nearest multiple, ties up
        return max(C, min(N, m))
    raise ValueError(f"unknown fixed schedule {kind!r}")


def subset_start(kind: str, k: int, N: int, M: int) -> int:
    """First row (in the annealed order) of iteration k's subset.

    The cumulative schedules of Sec. 3 use a prefix (start 0).  The fresh
    variants of Constant and CTR read the mini-batch of Sec. 3 as a
    stochastic-gradient batch: iteration k uses the M rows starting at
    (k M) mod N, wrapping past N to row 0, so consecutive iterations take
    consecutive disjoint batches through the permuted data; the full-batch
    refinement of CTR starts at 0."""
    if kind in FRESH_KINDS and M < N:
        return (k * M) % N
    return 0


def sda_next_beta(beta: float, wn, omega, omega_hat, delta_s: float = 1.0) -> float:
    """One SDA temperature update (Sec. 3.1).

    Weighted plug-in moments with normalised weights wn (the moment equations):
      E[Oh]  = sum_j w_j Oh_j,   E[Oh^2] = sum_j w_j Oh_j^2,  Var(Oh) = E[Oh^2] - E[Oh]^2
      E[O]   = sum_j w_j O_j,    E[O Oh] = sum_j w_j O_j Oh_j, Cov(O, Oh) = E[O Oh] - E[O] E[Oh]
    where Oh_j is the negative log-likelihood of the block being annealed in and
    O_j that of the data already fully included (O = 0 before the first append,
    which turns eq. beta_annealed_k into eq. beta_initial_data_k).
    Update beta' = beta - dS / (Var(Oh) + Cov(O, Oh)); if that does not exceed
    beta, the sign of dS is flipped; beta' is clipped to 1.
    Reading r10: a zero or non-finite denominator gives beta' = 1.
    The last moment, printed with a comma between Omega and Omega_hat, is read
    as the mixed moment E[Omega Omega_hat].
    """
    e_oh = sum(w * oh for w, oh in zip(wn, omega_hat))
    e_oh2 = sum(w * oh * oh for w, oh in zip(wn, omega_hat))
    e_o = sum(w * o for w, o in zip(wn, omega))
    e_ooh = sum(w * o * oh for w, o, oh in zip(wn, omega, omega_hat))
    var = e_oh2 - e_oh * e_oh
    cov = e_ooh - e_o * e_oh
    den = var + cov
    if den == 0.0 or not math.isfinite(den):
        return 1.0
    nb = beta - delta_s / den
    if nb <= beta:
        nb = beta + delta_s / den
    return min(nb, 1.0)


class SDAState:
    """SDA bookkeeping: rows [0, m_full) are fully included (coefficient 1),
    rows [m_full, m_full + block) are tempered by beta.  Starts with m_full = 0
    and the first C rows as the tempered block (eq. sda_initial_target).
    Reading r5: beta_0 = beta_reinit (0.1)."""

    def __init__(self, N: int, C: int, kappa: int, beta0: float = 0.1,
                 beta_reinit: float = 0.1, delta_s: float = 1.0):
        self.N, self.kappa = N, kappa
        self.m_full = 0
        self.block = min(C, N)
        self.beta = beta0
        self.beta_reinit = beta_reinit
        self.delta_s = delta_s

    @property
    def m_total(self) -> int:
        return self.m_full + self.block

    def advance(self, wn, omega, omega_hat) -> bool:
        """Move to the next target.  If beta already reached 1 the block joins
        the fully included data and the next kappa rows become the new block
        with beta restarting at beta_reinit (Sec. 3.1); with no rows left the sampler stays at the full data set.  Otherwise
        beta follows sda_next_beta.  Returns True when data were appended."""
        if self.beta >= 1.0:
            if self.m_total >= self.N:
                self.m_full, self.block, self.beta = self.N, 0, 1.0
                return False
            self.m_full += self.block
            self.block = min(self.kappa, self.N - self.m_full)
            self.beta = self.beta_reinit
            return True
        self.beta = sda_next_beta(self.beta, wn, omega, omega_hat, self.delta_s)
        return False
