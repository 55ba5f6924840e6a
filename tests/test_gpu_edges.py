"""Edge and extreme cases of the CUDA path against the oracle (GPU).

Degenerate instances (no clauses, tiny n), a single round, a zero state,
single-amplitude sampling, and the largest case a test can afford: n = 30
(8 GiB complex64 state, 1 GiB cost table checked whole and bit-exact).
"""

import math

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_no_clauses_every_assignment_solves(n):
    # m = 0: C = 0 everywhere, H_P = 0, so only the mixer acts and |+> is its
    # eigenvector: psi_p = e^{-i sum beta} |+>, P = 1.
    lits = np.zeros((0, 3), dtype=np.int32)
    cost, hist = core.build_cost(lits, n)
    assert cost.cpu().numpy().tolist() == [0] * (1 << n)
    assert hist.cpu().numpy().tolist() == [1 << n]
    g, b = instances.random_angles(4, n)
    state, out, tr = core.evolve(cost, n, 0, g, b, trace=True)
    ref = sv.evolve(np.zeros(1 << n, np.uint8), n, g, b)
    assert np.max(np.abs(state.cpu().numpy() - ref)) < 1e-6
    assert abs(out[0].item() - 1.0) < 1e-6 and np.max(np.abs(tr.cpu().numpy() - 1.0)) < 1e-6
    phase = np.exp(-1j * np.sum(b)) / math.sqrt(1 << n)
    assert np.max(np.abs(ref - phase)) < 1e-12


def test_single_round_and_single_clause():
    n, p = 3, 1
    lits = np.array([[1, -2, 3]], dtype=np.int32)
    cost, hist = core.build_cost(lits, n)
    assert hist.cpu().numpy().tolist() == [7, 1]
    state, out, _ = core.evolve(cost, n, 1, [1.1], [0.7])
    psi = sv.evolve(sv.cost_table(lits, n)[0], n, [1.1], [0.7])
    assert np.max(np.abs(state.cpu().numpy() - psi)) < 1e-6
    v, dg, db = core.grad(cost, n, 1, [1.1], [0.7])
    L, rdg, rdb = reduced.grad(hist.cpu().numpy(), [1.1], [0.7])
    assert abs(v.item() - L) < 1e-6
    assert abs(dg[0].item() - rdg[0]) < 1e-5 and abs(db[0].item() - rdb[0]) < 1e-5


@pytest.mark.parametrize("n", [5, 13])
def test_zero_state_readout(n):
    cost, _ = core.build_cost(instances.random_3sat(n, 2 * n, 1), n)
    z = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    out = core.prob(z, cost, n).cpu().numpy()
    assert np.all(out == 0.0)


def test_sample_one_variable():
    # n = 1 state (cos t, sin t): shot frequencies follow cos^2 and sin^2
    t = 0.4
    st = torch.tensor([math.cos(t), math.sin(t)], dtype=torch.complex64, device="cuda")
    shots = core.sample(st, 1, seed=9, shots=100000).cpu().numpy()
    psi = np.array([math.cos(t), math.sin(t)], dtype=np.complex128)
    ref = sv.sample(psi.astype(np.complex64).astype(np.complex128), 1, seed=9, shots=100000)
    assert np.mean(shots == ref) > 0.9999
    assert abs(np.mean(shots) - math.sin(t) ** 2) < 0.01


def test_largest_case_n30():
    n, m, p = 30, 126, 3
    lits = instances.random_3sat(n, m, 30)
    g, b = instances.random_angles(p, 30)
    cost, hist = core.build_cost(lits, n)
    state, out, _ = core.evolve(cost, n, m, g, b)
    torch.cuda.synchronize()
    ref_cost, ref_hist = sv.cost_table(lits, n)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref_hist)
    assert torch.equal(cost, torch.as_tensor(ref_cost).cuda())
    f = reduced.evolve(ref_hist, g, b)
    rng = np.random.default_rng(0)
    z = torch.as_tensor(rng.integers(0, 1 << n, 1 << 20), device="cuda")
    got = state[z].cpu().numpy()
    want = f[ref_cost[z.cpu().numpy()]]
    assert np.max(np.abs(got - want)) < 1e-5
    assert abs(out[0].item() - reduced.readout(ref_hist, f)[0]) < 1e-6
    assert abs(out[2].item() - 1.0) < 1e-5
