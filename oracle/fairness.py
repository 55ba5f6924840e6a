"""Fair-sampling metrics of Section IV (Table I), plain Python/numpy.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Section IV judges how uniformly G-QAOA samples the solutions by two
numbers: (i) the shots needed to observe every solution at least once, and
(ii) the draws from the solution distribution needed before a chi-square
test rejects the hypothesis that the solutions are sampled uniformly (the
median over many trials). Readings where the paper defers to its
references: a run of (i) is a sequence of shots of the full output
distribution and its value is the 1-based index of the shot that completes
the set; in (ii) the draws are the solution hits of the same shot sequence,
the test is applied after every draw once the expected count per solution
reaches 5 (draws >= 5 M), and it rejects when the Pearson statistic
X^2 = sum_j (O_j - d/M)^2 / (d/M) exceeds the (1 - alpha) quantile of the
chi-square law with M - 1 degrees of freedom. With integer counts
X^2 = (M sum_j O_j^2 - d^2) / d, so the decision is taken on the exact
integer numerator: reject when double(M sum O^2 - d^2) > crit * double(d)
(the same IEEE-double comparison as the GPU kernel).

`target` generalises "solution" to any cost class (the lowest non-empty
class for Max-SAT).
"""

from __future__ import annotations

import itertools

import numpy as np


def run_metrics(shots, cost, target: int, runs: int, chi2_crit: float, min_draws: int):
    """Per run r (shots r, r + runs, r + 2 runs, ... in that order): the
    1-based shot index completing the set of target assignments (0: never)
    and the number of target draws at the first rejection (0: never)."""
    shots = np.asarray(shots, dtype=np.int64)
    cost = np.asarray(cost)
    sols = np.nonzero(cost == target)[0]
    M = sols.size
    index = {int(z): j for j, z in enumerate(sols)}
    to_all = np.zeros(runs, dtype=np.int64)
    to_rej = np.zeros(runs, dtype=np.int64)
    for r in range(runs):
        counts = np.zeros(M, dtype=np.int64)
        seen = 0
        d = 0
        for t, z in enumerate(shots[r::runs]):
            j = index.get(int(z))
            if j is None:
                continue
            if counts[j] == 0:
                seen += 1
            counts[j] += 1
            d += 1
            if seen == M and to_all[r] == 0:
                to_all[r] = t + 1
            if d >= min_draws and to_rej[r] == 0:
                num = M * int(np.sum(counts * counts)) - d * d   # d X^2, exact
                if float(num) > chi2_crit * float(d):
                    to_rej[r] = d
            if to_all[r] and to_rej[r]:
                break
    return to_all, to_rej


def expected_shots_to_all(q) -> float:
    """E[shots until every outcome i has appeared], outcome i having
    probability q_i per shot (other outcomes allowed): by inclusion-exclusion
    over the non-empty subsets S of outcomes, sum (-1)^{|S|+1} / q_S."""
    q = np.asarray(q, dtype=np.float64)
    total = 0.0
    for k in range(1, q.size + 1):
        for S in itertools.combinations(range(q.size), k):
            total += (-1) ** (k + 1) / q[list(S)].sum()
    return total
