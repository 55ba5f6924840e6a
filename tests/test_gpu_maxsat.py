"""The Max-SAT readout D and its gradient on the statevector path, and the
protocol with D as its target, against the oracle.

D is the probability of the lowest non-empty cost class c* (the assignments
leaving the fewest clauses unsatisfied; Fig. 1(b)); for an unsatisfiable
instance c* > 0. gqaoa_evolve with GQAOA_READOUT_CLASS(c*) must report D
within the probability tolerance (1e-6) on the small-state and the streaming
paths; gqaoa_grad / gqaoa_grad_batched with GQAOA_OBJ_CLASS(c*) must match
the cost-class adjoint of the oracle within 2e-5 (as for P); the protocol
must return the oracle's fewest rounds for D >= 1/2.
"""

import numpy as np
import pytest
import torch

from oracle import protocol as oprot
from oracle import reduced
from oracle import statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances
from paper_2402_02585_gb300.protocol import Protocol

pytestmark = pytest.mark.gpu


def _unsat(n, m, seed):
    lits = instances.random_3sat(n, m, seed)
    _, hist = sv.cost_table(lits, n)
    cs = reduced.min_class(hist)
    assert cs > 0
    return lits, hist, cs


@pytest.mark.parametrize("n,m,seed,p", [(9, 60, 2, 7), (12, 80, 3, 12), (14, 100, 5, 5)])
def test_evolve_reads_out_the_max_sat_probability(n, m, seed, p):
    lits, hist, cs = _unsat(n, m, seed)
    cost, _ = core.build_cost(lits, n)
    g, b = instances.random_angles(p, seed)
    _, out, _ = core.evolve(cost, n, m, g, b, readout_class=cs)
    ref = reduced.readouts_trace(hist, g, b)[-1]
    o = out.cpu().numpy()
    assert abs(o[0] - ref[2]) < 1e-6
    assert abs(o[1] - ref[1]) < 1e-6 * m
    assert abs(o[2] - 1.0) < 1e-5
    _, out0, _ = core.evolve(cost, n, m, g, b)
    assert abs(out0[0].item()) < 1e-12            # no solution: P(C=0) = 0
    with pytest.raises(C.GQAOAError) as e:         # the trace stays P(C=0): not combined
        core.evolve(cost, n, m, g, b, trace=True, readout_class=cs)
    assert e.value.status == C.GQAOA_EINVAL


@pytest.mark.parametrize("n,m,seed,p", [(9, 60, 2, 5), (12, 80, 3, 6)])
def test_grad_of_the_max_sat_probability(n, m, seed, p):
    lits, hist, cs = _unsat(n, m, seed)
    cost, _ = core.build_cost(lits, n)
    g, b = instances.random_angles(p, seed + 1)
    L, dg, db = core.grad(cost, n, m, g, b, ("class", cs))
    rL, rdg, rdb = reduced.grad(hist, g, b, reduced.OBJ_P0, target=cs)
    assert abs(L.item() - rL) < 1e-6
    assert np.max(np.abs(dg.cpu().numpy() - rdg)) < 2e-5
    assert np.max(np.abs(db.cpu().numpy() - rdb)) < 2e-5
    # batched, two angle sets over the shared cost table
    g2, b2 = instances.random_angles(p, seed + 2)
    G = np.stack([g, g2])
    B = np.stack([b, b2])
    v, DG, DB = core.grad_batched(cost, n, m, G, B, ("class", cs), shared_cost=True)
    for i in range(2):
        rL, rdg, rdb = reduced.grad(hist, G[i], B[i], reduced.OBJ_P0, target=cs)
        assert abs(v[i].item() - rL) < 1e-6
        assert np.max(np.abs(DG[i].cpu().numpy() - rdg)) < 2e-5
        assert np.max(np.abs(DB[i].cpu().numpy() - rdb)) < 2e-5


@pytest.mark.parametrize("n,m,seed", [(9, 60, 2), (12, 80, 3)])
def test_protocol_max_sat_matches_oracle(n, m, seed):
    lits, hist, cs = _unsat(n, m, seed)
    cost, ghist = core.build_cost(lits, n)
    G, B = instances.protocol_grid(2)
    got = Protocol(cost, ghist, n, m).min_rounds(S=0.5, p_max=32, grid=(G, B), target="D")
    k, _, _, val, e = oprot.min_rounds(hist, G, B, S=0.5, p_max=32, target="D")
    assert k is not None and got.p == k
    assert abs(got.energy - e) < 1e-5 * m
    assert abs(got.prob - val) < 2e-4 and got.prob >= 0.5
