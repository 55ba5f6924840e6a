"""The batched adjoint gradient (gqaoa_grad_batched) at the gradient
benchmark's shape: n = 16, m = 67, p = 32 independent angle pairs drawn
uniformly in [0, pi).

At this size the default path holds each instance on one 8-CTA cluster for
all its rounds (the cluster-resident adjoint); with GQAOA_GRAD_STREAMING the
streaming passes run instead, where an instance spans 16 tiles of 4096
amplitudes, so several CTAs share it and each round's mixer sum is combined
from several reduction records per instance (asserted through
gqaoa_batched_geometry). Every instance's value and gradient is compared
with the oracle's cost-class adjoint (exact dynamics, FP64) within the
gradient tolerance of the other parity tests (1e-6 on P, 2e-5 on each
angle's derivative), and some rows with FP64 central differences
(h = 1e-4) within 5e-5.
"""

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances
from paper_2402_02585_gb300.optim import AngleOptimizer

pytestmark = pytest.mark.gpu

N_VARS, M_CLAUSES, P_ROUNDS = 16, 67, 32
V_TOL, G_TOL, FD_TOL = 1e-6, 2e-5, 5e-5


def _instances(B, seed0):
    n, m = N_VARS, M_CLAUSES
    cost = torch.empty((B, 1 << n), dtype=torch.uint8, device="cuda")
    hists = []
    for i in range(B):
        lits = instances.random_3sat(n, m, seed0 + i)
        cost[i].copy_(core.build_cost(lits, n, with_hist=False)[0])
        hists.append(sv.histogram(lits, n))
    return cost, hists


def _angles(B, seed0):
    G = np.stack([instances.random_angles(P_ROUNDS, seed0 + i)[0] for i in range(B)])
    Bt = np.stack([instances.random_angles(P_ROUNDS, seed0 + i)[1] for i in range(B)])
    return G, Bt


@pytest.mark.parametrize("streaming", [False, True])
def test_batched_gradient_several_ctas_per_instance(streaming):
    n, m, p, B = N_VARS, M_CLAUSES, P_ROUNDS, 64
    cost, hists = _instances(B, 500)
    G, Bt = _angles(B, 700)
    if streaming:
        for adjoint in (0, 1):
            cpi, rec = C.gqaoa_batched_geometry(n, B, adjoint)
            print(f"n={n} B={B} adjoint={adjoint}: {cpi} CTAs, {rec} records per instance")
            assert cpi >= 2 and rec >= 2
        v, dg, db = (t.cpu().numpy() for t in core.grad_batched(
            cost, n, m, G, Bt, C.GQAOA_OBJ_P0 | C.GQAOA_GRAD_STREAMING))
    else:
        opt = AngleOptimizer(cost, n, m, p)
        opt.reset(G, Bt)
        v = opt.evaluate().cpu().numpy()
        dg = opt.grad[0].cpu().numpy()
        db = opt.grad[1].cpu().numpy()
    for i in range(B):
        L, rdg, rdb = reduced.grad(hists[i], G[i], Bt[i], reduced.OBJ_P0)
        assert abs(v[i] - L) < V_TOL, (i, v[i], L)
        assert np.max(np.abs(dg[i] - rdg)) < G_TOL, i
        assert np.max(np.abs(db[i] - rdb)) < G_TOL, i
    for i in (0, 17, 63):
        fg, fb = reduced.fd_grad(hists[i], G[i], Bt[i], reduced.OBJ_P0, step=1e-4)
        assert np.max(np.abs(dg[i] - fg)) < FD_TOL, i
        assert np.max(np.abs(db[i] - fb)) < FD_TOL, i


def test_batched_gradient_energy_objective():
    # <H_P> (Eq. 4), the protocol's objective, at the same shape; its scale is m/8
    n, m, p, B = N_VARS, M_CLAUSES, P_ROUNDS, 24
    cost, hists = _instances(B, 900)
    G, Bt = _angles(B, 950)
    opt = AngleOptimizer(cost, n, m, p, objective="energy")
    opt.reset(G, Bt)
    v = opt.evaluate().cpu().numpy()
    dg = opt.grad[0].cpu().numpy()
    db = opt.grad[1].cpu().numpy()
    scale = m / 8
    for i in range(B):
        L, rdg, rdb = reduced.grad(hists[i], G[i], Bt[i], reduced.OBJ_ENERGY)
        assert abs(v[i] - L) < V_TOL * scale
        assert np.max(np.abs(dg[i] - rdg)) < G_TOL * scale
        assert np.max(np.abs(db[i] - rdb)) < G_TOL * scale


def test_adam_step_of_the_full_gradient_batch():
    # 1024 instances, the gradient benchmark's batch: the first evaluation of
    # every instance against the oracle adjoint, the Adam update of a sample of
    # instances against Adam written out in numpy, and the evaluation at the
    # updated angles against the oracle again
    n, m, p, B = N_VARS, M_CLAUSES, P_ROUNDS, 1024
    cpi, rec = C.gqaoa_batched_geometry(n, B, 1)
    print(f"n={n} B={B}: adjoint {cpi} CTAs, {rec} records per instance")
    cost, hists = _instances(B, 0)
    G, Bt = _angles(B, 0)
    opt = AngleOptimizer(cost, n, m, p)
    opt.reset(G, Bt)
    lr, b1, b2, eps = 0.05, 0.9, 0.999, 1e-8
    v0 = opt.step(lr).cpu().numpy()
    g0 = opt.grad.cpu().numpy()
    theta1 = opt.theta.cpu().numpy()
    worst = 0.0
    for i in range(B):
        L, rdg, rdb = reduced.grad(hists[i], G[i], Bt[i], reduced.OBJ_P0)
        assert abs(v0[i] - L) < V_TOL, i
        worst = max(worst, np.max(np.abs(g0[0, i] - rdg)), np.max(np.abs(g0[1, i] - rdb)))
    print(f"largest gradient deviation over {B} instances: {worst:.2e}")
    assert worst < G_TOL
    sample = np.random.default_rng(0).choice(B, 8, replace=False)
    for i in sample:
        for half, start in ((0, G[i]), (1, Bt[i])):
            g = -g0[half, i]  # maximise P: Adam descends on -P
            mt = (1 - b1) * g
            vt = (1 - b2) * g * g
            want = start - lr * (mt / (1 - b1)) / (np.sqrt(vt / (1 - b2)) + eps)
            assert np.max(np.abs(theta1[half, i] - want)) < 1e-12
    v1 = opt.evaluate().cpu().numpy()
    g1 = opt.grad.cpu().numpy()
    for i in sample:
        L, rdg, rdb = reduced.grad(hists[i], theta1[0, i], theta1[1, i], reduced.OBJ_P0)
        assert abs(v1[i] - L) < V_TOL
        assert np.max(np.abs(g1[0, i] - rdg)) < G_TOL
        assert np.max(np.abs(g1[1, i] - rdb)) < G_TOL
