"""Pins of the fair-sampling oracle (oracle/fairness.py) against closed forms,
a hand-checked shot stream, scipy's chi-square statistic and a Monte Carlo
estimate from numpy's own generator."""

import math

import numpy as np
import pytest
import scipy.stats

from oracle import fairness


def test_expected_shots_to_all_closed_forms():
    # equal probabilities q: the coupon collector, H_M / q
    for M, q in ((1, 0.5), (3, 0.2), (6, 0.1)):
        H = sum(1.0 / k for k in range(1, M + 1))
        assert abs(fairness.expected_shots_to_all(np.full(M, q)) - H / q) < 1e-9 * H / q
    # two outcomes: 1/a + 1/b - 1/(a + b)
    a, b = 0.05, 0.3
    assert abs(fairness.expected_shots_to_all([a, b]) - (1 / a + 1 / b - 1 / (a + b))) < 1e-12


def test_expected_shots_to_all_monte_carlo():
    q = np.array([0.1, 0.3, 0.05])
    rng = np.random.default_rng(7)
    runs = 20000
    u = rng.random((runs, 400))
    cum = np.cumsum(q)
    outcome = np.searchsorted(cum, u, side="right")  # 3 = none of them
    t = np.empty(runs)
    for r in range(runs):
        seen = np.zeros(4, dtype=bool)
        for i, o in enumerate(outcome[r]):
            seen[o] = True
            if seen[:3].all():
                t[r] = i + 1
                break
    exact = fairness.expected_shots_to_all(q)
    assert abs(t.mean() - exact) < 4 * t.std() / math.sqrt(runs)


def test_run_metrics_hand_checked():
    cost = np.ones(8, dtype=np.uint8)
    cost[[3, 5]] = 0
    crit = scipy.stats.chi2.ppf(0.95, 1)   # 3.841
    # one run: the set completes at shot 5; every later draw hits z = 3
    shots = np.array([0, 3, 1, 3, 5] + [3] * 20, dtype=np.uint64)
    to_all, to_rej = fairness.run_metrics(shots, cost, 0, 1, crit, 10)
    assert to_all[0] == 5
    # at d = 10 the counts are (9, 1): X^2 = 2 (16 / 5) = 6.4 > 3.84
    assert to_rej[0] == 10
    assert abs(scipy.stats.chisquare([9, 1]).statistic - 6.4) < 1e-12
    # two interleaved runs, shots 0, 2, 4, ... (3, 5, 3, 3, ...) and
    # 1, 3, 5, ... (0, 5, 3, 5, 5, ...): both draw counts (9, 1) by d = 10
    shots = np.array([3, 0, 5, 5, 3, 3] + [3, 5] * 10, dtype=np.uint64)
    to_all, to_rej = fairness.run_metrics(shots, cost, 0, 2, crit, 10)
    assert list(to_all) == [2, 3]
    assert list(to_rej) == [10, 10]
    # a target class other than 0 (cost 1 everywhere else)
    to_all, _ = fairness.run_metrics(np.array([0, 1, 2, 4, 6, 7], dtype=np.uint64), cost, 1, 1,
                                     crit, 100)
    assert to_all[0] == 6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_incremental_statistic_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 40, size=9)
    d, M = counts.sum(), counts.size
    s2 = int(np.sum(counts.astype(np.int64) ** 2))
    x2 = M * s2 / d - d              # the running form used by the GPU kernel
    assert abs(x2 - scipy.stats.chisquare(counts).statistic) < 1e-9
