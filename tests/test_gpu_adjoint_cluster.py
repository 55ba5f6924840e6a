"""The cluster-resident adjoint (gqaoa_grad_batched for 10 <= n <= 16: one
CTA or thread-block cluster holds an instance for all its forward and
backward rounds) against the oracle's cost-class adjoint and against the
other path of the same call (GQAOA_GRAD_STREAMING: the one-CTA kernels for
n <= 11, the streaming passes above).

Every shape is covered: n = 10, 11, 12 (one CTA of 64, 128, 256 threads), 13
(one 512-thread CTA), 14, 15 and 16 (clusters of 2, 4 and 8 CTAs), with more
instances than resident clusters at n = 16 (clusters loop over instances),
the three objectives (P(C=0), <H_P>, and the probability of the lowest cost
class of an unsatisfiable instance), a cost table shared by every row, and
rows whose leading rounds are identity (gamma = beta = 0), as the protocol's
depth windows pad them. Tolerances are the other gradient tests': 1e-6 on the
value and 2e-5 on each derivative, times m / 8 for <H_P>.
"""

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu

V_TOL, G_TOL = 1e-6, 2e-5


def _rows(n, m, B, seed0):
    cost = torch.empty((B, 1 << n), dtype=torch.uint8, device="cuda")
    hists = []
    for i in range(B):
        lits = instances.random_3sat(n, m, seed0 + i)
        cost[i].copy_(core.build_cost(lits, n, with_hist=False)[0])
        hists.append(sv.histogram(lits, n))
    return cost, hists


def _check(v, dg, db, hists, G, Bt, obj, scale):
    for i in range(len(hists)):
        L, rdg, rdb = reduced.grad(hists[i], G[i], Bt[i], obj)
        assert abs(v[i] - L) < V_TOL * scale, (i, v[i], L)
        assert np.max(np.abs(dg[i] - rdg)) < G_TOL * scale, i
        assert np.max(np.abs(db[i] - rdb)) < G_TOL * scale, i


@pytest.mark.parametrize("n,B,p", [(10, 5, 14), (11, 3, 12), (12, 3, 12), (13, 3, 10), (14, 2, 9),
                                   (15, 2, 8), (16, 40, 6)])
@pytest.mark.parametrize("objective", ["p0", "energy"])
def test_cluster_adjoint_matches_oracle_and_streaming(n, B, p, objective):
    m = int(round(4.2 * n))
    cost, hists = _rows(n, m, B, 7000 + n)
    rng = np.random.default_rng(n)
    G = rng.uniform(0, np.pi, (B, p))
    Bt = rng.uniform(0, np.pi, (B, p))
    code = C.GQAOA_OBJ_P0 if objective == "p0" else C.GQAOA_OBJ_ENERGY
    obj = reduced.OBJ_P0 if objective == "p0" else reduced.OBJ_ENERGY
    scale = 1.0 if objective == "p0" else m / 8
    got = [t.cpu().numpy() for t in core.grad_batched(cost, n, m, G, Bt, code)]
    ref = [t.cpu().numpy() for t in core.grad_batched(cost, n, m, G, Bt,
                                                      code | C.GQAOA_GRAD_STREAMING)]
    _check(*got, hists, G, Bt, obj, scale)
    _check(*ref, hists, G, Bt, obj, scale)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) < G_TOL * scale


def test_cluster_adjoint_class_objective_shared_cost_identity_rounds():
    # an unsatisfiable instance's lowest class (Max-SAT), one cost table for
    # every row, and rows padded in front with identity rounds
    n, m, p = 14, 110, 10
    lits = instances.random_3sat(n, m, 31)
    cost, hist = core.build_cost(lits, n)
    h = hist.cpu().numpy()
    cmin = int(np.nonzero(h)[0][0])
    assert cmin > 0
    rng = np.random.default_rng(5)
    B = 6
    G = rng.uniform(0, np.pi, (B, p))
    Bt = rng.uniform(0, np.pi, (B, p))
    for i in range(B):  # row i: its first i rounds are identity
        G[i, :i] = 0.0
        Bt[i, :i] = 0.0
    v, dg, db = (t.cpu().numpy() for t in core.grad_batched(
        cost, n, m, G, Bt, C.GQAOA_OBJ_CLASS(cmin), shared_cost=True))
    for i in range(B):
        L, rdg, rdb = reduced.grad(h, G[i], Bt[i], reduced.OBJ_P0, cmin)
        assert abs(v[i] - L) < V_TOL
        assert np.max(np.abs(dg[i] - rdg)) < G_TOL
        assert np.max(np.abs(db[i] - rdb)) < G_TOL
    # the single-instance entry point takes the same path
    v1, dg1, db1 = core.grad(cost, n, m, G[2], Bt[2], ("class", cmin))
    assert abs(v1.item() - v[2]) < 1e-12
    assert np.array_equal(dg1.cpu().numpy(), dg[2]) and np.array_equal(db1.cpu().numpy(), db[2])
