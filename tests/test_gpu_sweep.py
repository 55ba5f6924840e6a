"""The single-angle-pair sweep (gqaoa_sweep) against the oracle.

P(C=0) after the requested round counts must agree with the FP64 oracle
within 1e-6 for every (instance, angle point): the full statevector oracle at
small n, the exact cost-class model (pinned against it) at larger n. The
on-chip cases cover one warp per item (n = 9), whole CTAs (n = 12..14),
clusters of 2, 4, 8 and 16 CTAs (n = 15..18), a 16-CTA cluster with half the
state in shared memory (n = 19), and more items than resident CTAs. The
cluster-resident path (GQAOA_SWEEP_L2) covers n = 20..22 (52 % of an n = 20
state on chip, the rest streamed through the workspace) and more items than
resident clusters.
"""

import math

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


def run_sweep(costs, n, m, G, Bt, p, rounds, apt=0):
    B = costs.shape[0]
    A = len(G)
    gd = torch.as_tensor(np.asarray(G, dtype=np.float64), device="cuda")
    bd = torch.as_tensor(np.asarray(Bt, dtype=np.float64), device="cuda")
    out = torch.full((B, A, len(rounds)), -1.0, dtype=torch.float64, device="cuda")
    ws = core.workspace(C.gqaoa_sweep_workspace_size(n, A, apt))
    r = np.ascontiguousarray(rounds, dtype=np.int32)
    C.gqaoa_sweep(costs.data_ptr(), n, m, B, gd.data_ptr(), bd.data_ptr(), A, p, r.ctypes.data,
                  len(rounds), apt, out.data_ptr(), ws.data_ptr(), ws.numel(),
                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("apt", [0, 32])
@pytest.mark.parametrize("n,B,A,p,rounds", [
    (9, 3, 7, 12, [1, 4, 12]),
    (10, 2, 5, 8, [2, 8]),
    (12, 4, 9, 16, [1, 4, 16]),
    (13, 2, 4, 10, [3, 10]),
    (14, 2, 3, 16, [1, 16]),
    (15, 2, 3, 8, [1, 4, 8]),
    (16, 1, 3, 8, [8]),
    (17, 1, 2, 6, [1, 6]),
    (18, 1, 2, 5, [2, 5]),
    (19, 1, 3, 6, [1, 6]),
])
def test_sweep_matches_oracle(n, B, A, p, rounds, apt):
    if apt == 32 and n < 10:
        pytest.skip("32 amplitudes per thread needs n >= 10")
    m = int(math.floor(4.2 * n + 0.5))
    costs, hists, refc = [], [], []
    for i in range(B):
        lits = instances.random_3sat(n, m, 700 + 10 * n + i)
        c, h = core.build_cost(lits, n)
        costs.append(c)
        hists.append(h.cpu().numpy())
        if n <= 12:
            refc.append(sv.cost_table(lits, n)[0])
    rng = np.random.default_rng(n)
    G = rng.uniform(0, np.pi, A)
    Bt = rng.uniform(0, np.pi, A)
    got = run_sweep(torch.stack(costs), n, m, G, Bt, p, rounds, apt)
    for i in range(B):
        for a in range(A):
            if n <= 12:
                _, tr = sv.evolve(refc[i], n, [G[a]] * p, [Bt[a]] * p, trace=True)
            else:
                _, tr = reduced.evolve(hists[i], [G[a]] * p, [Bt[a]] * p, trace=True)
            ref = tr[np.asarray(rounds) - 1]
            assert np.max(np.abs(got[i, a] - ref)) < 1e-6, (i, a, got[i, a], ref)


@pytest.mark.parametrize("n,B,A,p,rounds", [
    (20, 2, 3, 10, [1, 5, 10]),
    (20, 1, 15, 6, [1, 6]),      # 15 items: more than the resident clusters
    (21, 1, 2, 6, [6]),
    (22, 1, 2, 4, [1, 4]),
])
def test_sweep_cluster_resident_matches_oracle(n, B, A, p, rounds):
    m = int(math.floor(4.2 * n + 0.5))
    costs, hists = [], []
    for i in range(B):
        c, h = core.build_cost(instances.random_3sat(n, m, 1700 + 10 * n + i), n)
        costs.append(c)
        hists.append(h.cpu().numpy())
    rng = np.random.default_rng(100 + n)
    G = rng.uniform(0, np.pi, A)
    Bt = rng.uniform(0, np.pi, A)
    G[0] = 0.0  # gamma = 0 keeps the random-guess probability h[0] / 2^n
    got = run_sweep(torch.stack(costs), n, m, G, Bt, p, rounds, C.GQAOA_SWEEP_L2)
    for i in range(B):
        assert np.max(np.abs(got[i, 0] - hists[i][0] / (1 << n))) < 1e-6
        for a in range(A):
            _, tr = reduced.evolve(hists[i], [G[a]] * p, [Bt[a]] * p, trace=True)
            ref = tr[np.asarray(rounds) - 1]
            assert np.max(np.abs(got[i, a] - ref)) < 1e-6, (n, i, a, got[i, a], ref)


def test_sweep_cluster_resident_agrees_with_streaming():
    # n = 20 on the cluster-resident sweep and on batched streaming evolution
    # (independent kernels): the same P within the tolerance
    n, p, rounds = 20, 12, [1, 6, 12]
    m = int(math.floor(4.2 * n + 0.5))
    cost = core.build_cost(instances.random_3sat(n, m, 1900), n)[0]
    rng = np.random.default_rng(20)
    G = rng.uniform(0, np.pi, 9)
    Bt = rng.uniform(0, np.pi, 9)
    a = run_sweep(cost[None], n, m, G, Bt, p, rounds, C.GQAOA_SWEEP_L2)[0]
    gd = torch.as_tensor(np.repeat(G[:, None], p, 1), device="cuda")
    bd = torch.as_tensor(np.repeat(Bt[:, None], p, 1), device="cuda")
    _, _, trace = core.evolve_batched(cost, n, m, gd, bd, shared_cost=True, trace=True)
    b = trace.cpu().numpy()[:, np.asarray(rounds) - 1]
    assert np.max(np.abs(a - b)) < 1e-6


def test_sweep_many_items_and_grid_left_endpoints():
    # more items than resident CTAs: the persistent loop must cover them all
    n, m, p = 12, 50, 8
    costs, hists = [], []
    for i in range(3):
        c, h = core.build_cost(instances.random_3sat(n, m, 900 + i), n)
        costs.append(c)
        hists.append(h.cpu().numpy())
    k = 32  # a 32 x 32 grid over [0, pi)^2, left endpoints
    G = np.repeat(np.arange(k) * np.pi / k, k)
    Bt = np.tile(np.arange(k) * np.pi / k, k)
    got = run_sweep(torch.stack(costs), n, m, G, Bt, p, [1, 4, 8])
    for i in range(3):
        for a in range(0, k * k, 37):
            _, tr = reduced.evolve(hists[i], [G[a]] * p, [Bt[a]] * p, trace=True)
            assert np.max(np.abs(got[i, a] - tr[[0, 3, 7]])) < 1e-6
    # gamma = 0 or beta = 0 rows keep the random-guess probability
    for i in range(3):
        h0 = hists[i][0] / (1 << n)
        assert np.max(np.abs(got[i, :k, :] - h0)) < 1e-6          # gamma = 0
        assert np.max(np.abs(got[i, ::k, :] - h0)) < 1e-6         # beta = 0


def test_sweep_plan_mixed_buckets_and_graph_replay():
    from paper_2402_02585_gb300.sweep import SweepPlan
    p, rounds = 6, [1, 3, 6]
    buckets, hists = {}, {}
    for n, B in ((11, 2), (13, 2), (19, 1)):
        m = int(math.floor(4.2 * n + 0.5))
        cs, hs = [], []
        for i in range(B):
            c, h = core.build_cost(instances.random_3sat(n, m, 1200 + 10 * n + i), n)
            cs.append(c)
            hs.append(h.cpu().numpy())
        buckets[n] = (torch.stack(cs), m)
        hists[n] = hs
    rng = np.random.default_rng(3)
    G = rng.uniform(0, np.pi, 5)
    Bt = rng.uniform(0, np.pi, 5)
    table = {11: {"path": "onchip"}, 13: {"path": "stream", "angle_batch": 2},
             19: {"path": "stream", "angle_batch": 3}}
    plan = SweepPlan(buckets, G, Bt, p, rounds, table=table)
    eager = {n: o.clone() for n, o in plan.run().items()}
    torch.cuda.synchronize()
    for n, hs in hists.items():
        for i, h in enumerate(hs):
            for a in range(5):
                _, tr = reduced.evolve(h, [G[a]] * p, [Bt[a]] * p, trace=True)
                got = eager[n][i, a].cpu().numpy()
                assert np.max(np.abs(got - tr[np.asarray(rounds) - 1])) < 1e-6, (n, i, a)
    plan.capture()
    for o in plan.out.values():
        o.fill_(-1.0)
    plan.replay()
    torch.cuda.synchronize()
    for n in eager:
        assert torch.equal(plan.out[n], eager[n])


def test_sweep_plan_concurrent_replay_matches_sequential():
    # a 16-CTA-cluster bucket (n = 20, cluster-resident) beside smaller
    # on-chip buckets: the two-stream replay must give the same bits
    from paper_2402_02585_gb300.sweep import SweepPlan
    p, rounds = 6, [1, 6]
    buckets = {}
    for n, B in ((11, 2), (15, 1), (20, 1)):
        m = int(math.floor(4.2 * n + 0.5))
        cs = [core.build_cost(instances.random_3sat(n, m, 1500 + 10 * n + i), n)[0]
              for i in range(B)]
        buckets[n] = (torch.stack(cs), m)
    rng = np.random.default_rng(5)
    G = rng.uniform(0, np.pi, 9)
    Bt = rng.uniform(0, np.pi, 9)
    table = {11: {"path": "onchip"}, 15: {"path": "onchip", "apt": 32}, 20: {"path": "l2"}}
    plan = SweepPlan(buckets, G, Bt, p, rounds, table=table)
    assert [plan.lane(st) for st in plan.steps] == ["small", "small", "big"]
    eager = {n: o.clone() for n, o in plan.run().items()}
    plan.capture()
    for o in plan.out.values():
        o.fill_(-1.0)
    plan.replay_concurrent()
    torch.cuda.synchronize()
    for n in eager:
        assert torch.equal(plan.out[n], eager[n])
