"""Pins of the oracle's generators, mini-batch order and schedules against
published known answers and hand-derived sequences (CPU only)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import rng, schedules
from tests.conftest import GOLDEN


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split("#")[0].strip() for ln in f if ln.split("#")[0].strip()]


def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row.split()]
        assert rng.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_splitmix64_known_answers():
    for row in _rows("splitmix64_kat.txt"):
        seed, outs = row.split(":")
        g = rng.SplitMix64(int(seed))
        assert [g.next_u64() for _ in outs.split()] == [int(t) for t in outs.split()]


def test_permutation_is_uniform_permutation():
    for n, seed in [(1, 0), (2, 3), (10, 1), (1000, 7)]:
        p = rng.fisher_yates_permutation(n, seed)
        assert sorted(p.tolist()) == list(range(n))
    # every one of the 3! orders of a 3-element shuffle appears with frequency ~1/6
    counts = {}
    for seed in range(6000):
        key = tuple(rng.fisher_yates_permutation(3, seed).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    chi2 = sum((c - 1000) ** 2 / 1000 for c in counts.values())
    assert chi2 < 25.0        # 5 dof, p ~ 1e-4


def test_box_muller_moments():
    z = rng.philox_normals(seed=11, stream=1, iteration=0, n=40000)
    assert abs(z.mean()) < 0.03
    assert abs(z.var() - 1.0) < 0.03
    assert abs(np.mean(z ** 4) - 3.0) < 0.15     # Gaussian kurtosis
    # offset addressing gives the same numbers as a longer draw
    w = rng.philox_normals(seed=11, stream=1, iteration=0, n=10, offset=5)
    assert np.array_equal(w, z[5:15])


def test_schedule_worked_example():
    N, C, kappa, K = 60000, 500, 500, 200
    for row in _rows("schedules_worked_example.txt"):
        lhs, total = row.split("|")
        parts = lhs.split()
        kind = parts[0]
        for kv in parts[1:]:
            k, m = kv.split(":")
            assert schedules.subset_size(kind, int(k), N, C, kappa, K) == int(m), (kind, k)
        s = sum(schedules.subset_size(kind, k, N, C, kappa, K) for k in range(K))
        assert s == int(total), kind
    assert schedules.automated_increment(N, C, K) == 330


@pytest.mark.parametrize("kind", schedules.FIXED_KINDS)
def test_schedule_invariants(kind):
    for (N, C, kappa, K) in [(2048, 256, 256, 30), (60000, 1000, 1000, 200), (997, 100, 37, 13)]:
        seq = [schedules.subset_size(kind, k, N, C, kappa, K) for k in range(K)]
        assert all(min(C, N) <= m <= N for m in seq)
        assert all(b >= a for a, b in zip(seq, seq[1:])), "subset never shrinks"
        late = [m for k, m in enumerate(seq) if 10 * k >= 9 * K]
        if kind not in (schedules.CONSTANT, schedules.CONSTANT_FRESH):
            assert all(m == N for m in late), "full data from 0.9K on"
        if kind == schedules.AUTOMATED:
            assert all(m % kappa == 0 or m == N for m in seq)


def test_config0_linear_schedule():
    # 2048 samples, C = kappa = 256, K = 30: one mini-batch per iteration until all 8 are in.
    seq = [schedules.subset_size("linear", k, 2048, 256, 256, 30) for k in range(30)]
    assert seq[:9] == [256, 512, 768, 1024, 1280, 1536, 1792, 2048, 2048]
    assert seq[-1] == 2048


def test_sda_worked_example():
    for row in _rows("sda_worked_example.txt"):
        t = row.split()
        w0, w1, oh0, oh1, o0, o1, beta, ds = (float(v) for v in t[:8])
        expect = Fraction(t[8])
        got = schedules.sda_next_beta(beta, [w0, w1], [o0, o1], [oh0, oh1], ds)
        assert abs(got - float(expect)) < 1e-12


def test_sda_state_machine():
    s = schedules.SDAState(N=10, C=4, kappa=3, beta0=0.1)
    assert (s.m_full, s.block, s.beta) == (0, 4, 0.1)
    # a tiny variance drives beta to 1; the next advance appends a block
    s.advance([0.5, 0.5], [0.0, 0.0], [1.0, 1.01])
    assert s.beta == 1.0 and s.m_full == 0
    assert s.advance([0.5, 0.5], [0.0, 0.0], [1.0, 1.01]) is True
    assert (s.m_full, s.block, s.beta) == (4, 3, 0.1)
    s.beta = 1.0
    assert s.advance(None, None, None) is True
    assert (s.m_full, s.block, s.beta) == (7, 3, 0.1)
    s.beta = 1.0
    assert s.advance(None, None, None) is False      # nothing left to append
    assert (s.m_full, s.block, s.beta) == (10, 0, 1.0)
    assert s.advance(None, None, None) is False
    assert (s.m_full, s.block, s.beta) == (10, 0, 1.0)
    # degenerate denominator -> beta jumps to one (reading r10)
    assert schedules.sda_next_beta(0.3, [1.0], [0.0], [5.0]) == 1.0


def test_fresh_batches_walk_the_data_once_per_epoch():
    """Fresh Constant batches: consecutive iterations take consecutive disjoint
    blocks, so N / C iterations use every row exactly once (N = 60000, C = 500);
    with N not a multiple of M the window wraps to row 0 (hand-listed)."""
    N, C = 60000, 500
    seen = np.zeros(N, np.int64)
    for k in range(N // C):
        s = schedules.subset_start(schedules.CONSTANT_FRESH, k, N, C)
        seen[(s + np.arange(C)) % N] += 1
    assert np.all(seen == 1)
    windows = [list((schedules.subset_start("constant_fresh", k, 10, 4) + np.arange(4)) % 10) for k in range(4)]
    assert windows == [[0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 0, 1], [2, 3, 4, 5]]
    # cumulative schedules and the refinement phase of fresh CTR use the prefix
    assert schedules.subset_start(schedules.LINEAR, 5, N, 5500) == 0
    assert schedules.subset_start(schedules.CTR_FRESH, 7, N, C) == 3500
    assert schedules.subset_start(schedules.CTR_FRESH, 190, N, N) == 0
