"""Section IV's fair-sampling metrics on the GPU (gqaoa_fairness) against the
oracle (oracle/fairness.py).

Both metrics are integers decided by integer counts, so on the same seeded
synthetic shot stream the GPU and the oracle must agree exactly, run by run
(solutions as the target, and the lowest non-empty class of an
unsatisfiable instance). End to end, the shots of gqaoa_sample on a G-QAOA
state must give a mean shots-to-every-solution within 4 standard errors of
the oracle's exact expectation for that state.
"""

import math

import numpy as np
import pytest
import scipy.stats
import torch

from oracle import fairness, reduced
from oracle import protocol as oprotocol
from oracle import statevector as sv
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,seed,runs,per_run,hot", [
    (8, 30, 11, 500, 64, 0.6),     # 5 solutions
    (10, 40, 2, 2000, 512, 0.3),   # 16 solutions (about 180 shots to see them all)
    (9, 60, 2, 300, 400, 0.5),     # unsatisfiable: the lowest class c* = 1
    # the kernel with counts in global memory: runs longer than 4095 shots, and n > 15
    (8, 30, 11, 200, 5000, 0.6),
    (16, 67, 3, 300, 700, 0.3),
])
def test_fairness_matches_oracle_exactly(n, m, seed, runs, per_run, hot):
    lits = instances.random_3sat(n, m, seed)
    ocost, ohist = sv.cost_table(lits, n)
    target = reduced.min_class(ohist)
    targets = int(ohist[target])
    shots = instances.synthetic_shots(n, runs * per_run, seed, hot=np.nonzero(ocost == target)[0],
                                      hot_fraction=hot)
    crit = float(scipy.stats.chi2.ppf(0.95, max(targets - 1, 1)))
    min_draws = 5 * targets
    ra, rr = fairness.run_metrics(shots, ocost, target, runs, crit, min_draws)
    cost, _ = core.build_cost(lits, n)
    dev_shots = torch.as_tensor(shots.astype(np.int64)).cuda()
    ga, gr = core.fairness(dev_shots, runs, cost, n, target, targets, crit, min_draws)
    assert np.array_equal(ga.cpu().numpy(), ra)
    assert np.array_equal(gr.cpu().numpy(), rr)
    assert (ra > 0).sum() > runs // 2     # the streams do complete, and ...
    # ... a wrong target count is reported as -1 everywhere
    ga, gr = core.fairness(dev_shots, runs, cost, n, target, targets + 1, crit, min_draws)
    assert int(ga.max()) == -1 and int(ga.min()) == -1 and int(gr.max()) == -1


def test_sampler_shots_to_all_matches_expectation():
    n, m, p = 10, 40, 6
    lits = instances.random_3sat(n, m, 2)
    ocost, ohist = sv.cost_table(lits, n)
    # the single angle pair of highest P on a coarse grid (16 solutions, P ~ 1/2)
    G, B = instances.protocol_grid(3)
    _, P, _ = oprotocol.grid_readouts(ohist, G, B, p)
    a = int(np.argmax(P[:, -1]))
    g, b = [G[a]] * p, [B[a]] * p
    psi = sv.evolve(ocost, n, g, b)
    q = np.abs(psi[ocost == 0]) ** 2
    exact = fairness.expected_shots_to_all(q)
    cost, _ = core.build_cost(lits, n)
    state, _, _ = core.evolve(cost, n, m, g, b)
    runs, per_run = 20000, 2048
    shots = core.sample(state, n, 77, runs * per_run)
    ta, _ = core.fairness(shots, runs, cost, n, 0, int(ohist[0]), 1e30, 10**9)
    ta = ta.cpu().numpy().astype(np.float64)
    assert (ta > 0).all()
    assert abs(ta.mean() - exact) < 4 * ta.std() / math.sqrt(runs), (ta.mean(), exact)
