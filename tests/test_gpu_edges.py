"""Edge and extreme cases of the CUDA path against the oracle (GPU).

Degenerate instances (no clauses, tiny n), a single round, a zero state,
single-amplitude sampling, n = 30 (8 GiB complex64 state, 1 GiB cost table
checked whole and bit-exact), and the largest n the library accepts
(GQAOA_MAX_N = 34: 128 GiB state) on an instance whose histogram has a
closed form.
"""

import math

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
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
    # amplitudes are ~2^(-n/2): the bound is relative to the largest one
    assert np.max(np.abs(got - want)) < 1e-5 * np.max(np.abs(f))
    assert abs(out[0].item() - reduced.readout(ref_hist, f)[0]) < 1e-6
    assert abs(out[2].item() - 1.0) < 1e-5


def test_largest_n_closed_form_histogram():
    # n = GQAOA_MAX_N: 2^34 amplitudes (128 GiB complex64 state, 16 GiB cost
    # table), so every index above 2^32 is exercised. With variable-disjoint
    # clauses C(z) is a sum of m independent indicators, each 1 on one of the
    # 8 assignments of its three variables (Eq. 1), hence exactly
    #   h[c] = binom(m, c) 7^(m - c) 2^(n - 3m),
    # and the cost-class model on that histogram gives every amplitude.
    n = C.GQAOA_MAX_N
    if torch.cuda.get_device_properties(0).total_memory < (200 << 30):
        pytest.skip("needs about 150 GiB of device memory")
    m = n // 3
    rng = np.random.default_rng(34)
    # distinct variables, the lowest and the highest among them
    rest = rng.permutation(np.setdiff1d(np.arange(n), [0, n - 1, n // 2]))
    var = np.concatenate([[0, n - 1, n // 2], rest])[: 3 * m]
    sign = rng.choice([-1, 1], size=3 * m)
    lits = ((var + 1) * sign).reshape(m, 3).astype(np.int32)
    want_hist = np.array([math.comb(m, c) * 7 ** (m - c) * 2 ** (n - 3 * m) for c in range(m + 1)],
                         dtype=np.uint64)
    assert int(want_hist.sum()) == 1 << n
    cost, hist = core.build_cost(lits, n)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), want_hist)

    z = rng.integers(0, 1 << n, 4096, dtype=np.int64)
    z[:4] = [0, (1 << n) - 1, 1 << (n - 1), (1 << (n - 1)) - 1]
    zd = torch.as_tensor(z, device="cuda")
    ref_cost = np.array([sv.cost_at(lits, int(v)) for v in z])
    assert np.array_equal(cost[zd].cpu().numpy(), ref_cost)

    g, b = instances.random_angles(2, 34)
    state, out, _ = core.evolve(cost, n, m, g, b)
    f = reduced.evolve(want_hist, g, b)
    got = state[zd].cpu().numpy()
    assert np.max(np.abs(got - f[ref_cost])) < 1e-5 * np.max(np.abs(f))
    o = out.cpu().numpy()
    assert abs(o[0] - reduced.readout(want_hist, f)[0]) < 1e-6
    assert abs(o[2] - 1.0) < 1e-5

    # shots: cost-class frequencies against the class weights h[c] |f(c)|^2
    shots = 100000
    zs = core.sample(state, n, seed=34, shots=shots)
    assert int(zs.min()) >= 0 and int(zs.max()) < (1 << n)
    cls = np.bincount(cost[zs].cpu().numpy(), minlength=m + 1)
    w = want_hist.astype(np.float64) * np.abs(f) ** 2
    w /= w.sum()
    exp = shots * w
    assert np.all(np.abs(cls - exp) <= 5 * np.sqrt(exp * (1 - w)) + 1), (cls, exp)
    del state, cost, zs, zd
    torch.cuda.empty_cache()
