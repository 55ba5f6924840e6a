"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: cost tables and histograms bit-exact; complex64 amplitudes within
1e-5 max-abs and P(C=0) within 1e-6 absolute of the FP64 oracle; gradients
within 2e-5 absolute (complex64 state, FP64 sums). Sizes span several
4096-amplitude tiles and the single-CTA small-state path (n < 12).
"""

import math

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import core, instances
from tests.golden_io import paper_instances
from tests.shot_compare import compare_same_state

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
P_TOL = 1e-6


def gpu_cost(lits, n):
    cost, hist = core.build_cost(lits, n)
    torch.cuda.synchronize()
    return cost, hist


# ---------------------------------------------------------------- cost table

@pytest.mark.parametrize("n,m,seed", [
    (3, 1, 0), (4, 8, 1), (5, 21, 2), (8, 34, 3), (11, 46, 4),       # per-assignment kernel
    (12, 50, 5), (13, 55, 6), (16, 67, 7), (18, 76, 8), (20, 84, 9),  # bit-sliced kernel
    (12, 0, 10), (12, 255, 11), (14, 1, 12), (15, 9, 13),
])
def test_cost_table_bit_exact(n, m, seed):
    lits = instances.random_3sat(n, m, seed)
    cost, hist = gpu_cost(lits, n)
    ref_cost, ref_hist = sv.cost_table(lits, n)
    assert np.array_equal(cost.cpu().numpy(), ref_cost)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref_hist)


def test_cost_table_paper_instances():
    for inst in paper_instances():
        cost, hist = gpu_cost(inst["lits"], inst["n"])
        ref_cost, ref_hist = sv.cost_table(inst["lits"], inst["n"])
        assert np.array_equal(cost.cpu().numpy(), ref_cost)
        assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref_hist)


def test_cost_table_high_variables_only():
    # clauses touching only variables >= 5 exercise the word-constant branch
    n = 14
    lits = np.array([[6, -7, 8], [-9, 10, -14], [12, 13, -6]], dtype=np.int32)
    cost, hist = gpu_cost(lits, n)
    ref_cost, ref_hist = sv.cost_table(lits, n)
    assert np.array_equal(cost.cpu().numpy(), ref_cost)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref_hist)


def test_cost_table_without_histogram():
    lits = instances.random_3sat(13, 50, 3)
    cost, hist = core.build_cost(lits, 13, with_hist=False)
    assert hist is None
    assert np.array_equal(cost.cpu().numpy(), sv.cost_table(lits, 13)[0])


# ---------------------------------------------------------------- evolution

def check_state(psi_gpu, psi_ref):
    err = np.max(np.abs(psi_gpu.cpu().numpy().astype(np.complex128) - psi_ref))
    assert err < AMP_TOL, err


@pytest.mark.parametrize("n,m,p,seed", [
    (4, 8, 3, 0), (10, 42, 8, 0), (11, 46, 16, 1),   # single-CTA path
    (12, 50, 8, 2), (13, 55, 12, 3), (16, 67, 20, 4), (18, 76, 10, 5),  # streaming path
])
def test_evolve_matches_oracle(n, m, p, seed):
    lits = instances.random_3sat(n, m, seed)
    g, b = instances.random_angles(p, seed)
    cost, _ = gpu_cost(lits, n)
    state, out, tr = core.evolve(cost, n, m, g, b, trace=True)
    torch.cuda.synchronize()
    ref_cost, _ = sv.cost_table(lits, n)
    psi, ref_tr = sv.evolve(ref_cost, n, g, b, trace=True)
    check_state(state, psi)
    r = sv.readout(psi, ref_cost, n)
    o = out.cpu().numpy()
    assert abs(o[0] - r[0]) < P_TOL
    assert abs(o[1] - r[1]) < 1e-5 * max(1.0, m / 8)
    assert abs(o[2] - 1.0) < 1e-5
    assert np.max(np.abs(tr.cpu().numpy() - ref_tr)) < P_TOL


def test_config1_small_instance():
    # n = 10, m = 42 (d = 4.2), seed 0, p = 8, angles uniform in [0, pi)
    n, m, p = 10, 42, 8
    lits = instances.random_3sat(n, m, 0)
    g, b = instances.random_angles(p, 0)
    cost, hist = gpu_cost(lits, n)
    ref_cost, ref_hist = sv.cost_table(lits, n)
    assert np.array_equal(cost.cpu().numpy(), ref_cost)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref_hist)
    state, out, _ = core.evolve(cost, n, m, g, b)
    psi = sv.evolve(ref_cost, n, g, b)
    check_state(state, psi)
    assert abs(out[0].item() - sv.readout(psi, ref_cost, n)[0]) < P_TOL


@pytest.mark.parametrize("n", [9, 13])
def test_evolve_from_given_state(n):
    m, p = 4 * n, 6
    lits = instances.random_3sat(n, m, 21)
    g, b = instances.random_angles(p, 21)
    psi0 = instances.random_state(n, 21)
    cost, _ = gpu_cost(lits, n)
    st = torch.as_tensor(psi0.astype(np.complex64)).cuda()
    state, out, _ = core.evolve(cost, n, m, g, b, state=st, state_in=True)
    ref_cost, _ = sv.cost_table(lits, n)
    psi = sv.evolve(ref_cost, n, g, b, psi0=psi0.astype(np.complex64).astype(np.complex128))
    check_state(state, psi)


def test_special_cases_on_gpu():
    n, m, p = 13, 52, 5
    lits = instances.random_3sat(n, m, 31)
    cost, hist = gpu_cost(lits, n)
    h0 = hist[0].item() / (1 << n)
    g, b = instances.random_angles(p, 31)
    _, out, _ = core.evolve(cost, n, m, np.zeros(p), b)
    assert abs(out[0].item() - h0) < P_TOL
    _, out, _ = core.evolve(cost, n, m, g, np.zeros(p))
    assert abs(out[0].item() - h0) < P_TOL
    # Grover (Appendix A): one clause, gamma = beta = pi, C=1 weight sin^2((2k+1) theta)
    one = np.array([[1, -2, 3]], dtype=np.int32)
    cost1, hist1 = gpu_cost(one, n)
    theta = math.asin(math.sqrt(hist1[1].item() / (1 << n)))
    for k in (1, 3, 7):
        _, out, _ = core.evolve(cost1, n, 1, [math.pi] * k, [math.pi] * k)
        assert abs(out[1].item() - math.sin((2 * k + 1) * theta) ** 2) < 1e-5


def test_reduced_model_at_every_amplitude():
    n, m, p = 16, 67, 24
    lits = instances.random_3sat(n, m, 41)
    g, b = instances.random_angles(p, 41)
    cost, hist = gpu_cost(lits, n)
    state, out, _ = core.evolve(cost, n, m, g, b)
    f = reduced.evolve(hist.cpu().numpy(), g, b)
    ref_cost, _ = sv.cost_table(lits, n)
    check_state(state, reduced.amplitudes(f, ref_cost))
    assert abs(out[0].item() - reduced.readout(hist.cpu().numpy(), f)[0]) < P_TOL


def test_prob_readout():
    for n in (10, 14):
        m = 4 * n
        lits = instances.random_3sat(n, m, 51)
        psi0 = instances.random_state(n, 51).astype(np.complex64)
        cost, _ = gpu_cost(lits, n)
        out = core.prob(torch.as_tensor(psi0).cuda(), cost, n).cpu().numpy()
        ref = sv.readout(psi0.astype(np.complex128), sv.cost_table(lits, n)[0], n)
        assert np.allclose(out, ref, atol=1e-6, rtol=1e-6)


def test_evolve_batched_matches_per_instance():
    n, p, B = 13, 7, 5
    ms = [40, 52, 55, 60, 65]
    m = max(ms)
    costs, refs = [], []
    for i in range(B):
        lits = instances.random_3sat(n, ms[i], 100 + i)
        c, _ = gpu_cost(lits, n)
        costs.append(c)
        refs.append(sv.cost_table(lits, n)[0])
    cost = torch.stack(costs)
    G = np.stack([instances.random_angles(p, 200 + i)[0] for i in range(B)])
    Bt = np.stack([instances.random_angles(p, 200 + i)[1] for i in range(B)])
    state, out, tr = core.evolve_batched(cost, n, m, G, Bt, trace=True)
    torch.cuda.synchronize()
    for i in range(B):
        psi, rtr = sv.evolve(refs[i], n, G[i], Bt[i], trace=True)
        check_state(state[i], psi)
        assert abs(out[i, 0].item() - sv.readout(psi, refs[i], n)[0]) < P_TOL
        assert np.max(np.abs(tr[i].cpu().numpy() - rtr)) < P_TOL


@pytest.mark.parametrize("n", [8, 12])
def test_evolve_batched_shared_cost(n):
    # one formula, many angle sets: the single-angle-pair grid of Eq. 5
    m, p = 4 * n, 6
    lits = instances.random_3sat(n, m, 61)
    cost, hist = gpu_cost(lits, n)
    grid = [(gi * math.pi / 4, bj * math.pi / 4) for gi in range(4) for bj in range(4)]
    G = np.array([[gg] * p for gg, _ in grid])
    Bt = np.array([[bb] * p for _, bb in grid])
    _, out, _ = core.evolve_batched(cost, n, m, G, Bt, shared_cost=True)
    h = hist.cpu().numpy()
    for i in range(len(grid)):
        ref = reduced.readout(h, reduced.evolve(h, G[i], Bt[i]))
        assert abs(out[i, 0].item() - ref[0]) < P_TOL


# ---------------------------------------------------------------- sampling

def check_shots_valid(shots, psi_ref, seed, tol):
    """Every shot z must satisfy CDF(z-1) - tol <= u * total <= CDF(z) + tol."""
    cdf = np.cumsum(np.abs(psi_ref) ** 2)
    total = cdf[-1]
    u = np.array([sv.shot_uniform(seed, s) for s in range(len(shots))])
    t = u * total
    lo = np.where(shots > 0, cdf[np.maximum(shots - 1, 0)], 0.0)
    hi = cdf[shots]
    assert np.all(lo - tol <= t) and np.all(t <= hi + tol)


@pytest.mark.parametrize("n,shots", [(6, 3000), (10, 20000), (12, 20000), (13, 50000),
                                     (15, 1_000_000), (16, 50000), (20, 200000), (16, 1000),
                                     (20, 16384), (22, 65536)])
def test_sample_matches_oracle_on_the_same_state(n, shots):
    # Sampling is index work: given the same complex64 state (upcast to FP64
    # for the oracle) and the same Philox uniforms, every shot must be the
    # oracle's, except where a target lies within the CDFs' rounding (a few
    # FP64 units of the norm on both sides) of a boundary. n = 6, 10: one-CTA
    # path; 12..15: all tiles resident in shared memory; 16 with 50000 and 20
    # with 200000 shots: shots bucketed by tile; 16 with 1000, 20 with 16384
    # and 22 with 65536 shots (at most 64 per tile): each shot resolved from
    # the stored chunk prefixes.
    m, p, seed = 4 * n, 5, 71
    lits = instances.random_3sat(n, m, seed)
    g, b = instances.random_angles(p, seed)
    cost, _ = gpu_cost(lits, n)
    state, _, _ = core.evolve(cost, n, m, g, b)
    got = core.sample(state, n, seed=1234, shots=shots).cpu().numpy()
    psi = state.cpu().numpy().astype(np.complex128)
    ref, cdf = sv.sample(psi, n, seed=1234, shots=shots, return_cdf=True)
    compare_same_state(got, ref, cdf, 1234, eps=1e-14 * cdf[-1], label=f"n={n}")


@pytest.mark.parametrize("n,shots", [(10, 20000), (15, 50000)])
def test_sample_within_state_error_of_the_fp64_evolution(n, shots):
    # against the FP64-evolved state the complex64 state moves the CDF by up
    # to ~1e-6 of the norm, so each shot's target must lie in its
    # amplitude's CDF interval of the exact state up to that much
    m, p, seed = 4 * n, 5, 71
    lits = instances.random_3sat(n, m, seed)
    g, b = instances.random_angles(p, seed)
    cost, _ = gpu_cost(lits, n)
    state, _, _ = core.evolve(cost, n, m, g, b)
    got = core.sample(state, n, seed=1234, shots=shots).cpu().numpy()
    psi = sv.evolve(sv.cost_table(lits, n)[0], n, g, b)
    check_shots_valid(got, psi, 1234, tol=1e-5)


def test_sample_fair_over_solutions():
    import scipy.stats
    n, m, p = 16, 56, 12
    for seed in range(200, 260):
        lits = instances.random_3sat(n, m, seed)
        if sv.histogram(lits, n)[0] >= 8:
            break
    g, b = instances.random_angles(p, seed)
    cost, hist = gpu_cost(lits, n)
    state, out, _ = core.evolve(cost, n, m, g, b)
    shots = core.sample(state, n, seed=5, shots=200000)
    c = cost[shots].cpu().numpy()
    z = shots.cpu().numpy()
    sol = z[c == 0]
    counts = np.bincount(sol, minlength=1 << n)[np.flatnonzero(sv.cost_table(lits, n)[0] == 0)]
    # uniform over the solutions (fair sampling, Section IV)
    stat = np.sum((counts - counts.mean()) ** 2 / counts.mean())
    assert scipy.stats.chi2.sf(stat, len(counts) - 1) > 1e-4
    # weight per cost class matches h[c] |f_p(c)|^2
    h = hist.cpu().numpy()
    f = reduced.evolve(h, g, b)
    w = h * np.abs(f) ** 2
    obs = np.bincount(c, minlength=len(h))
    exp = w * len(c)
    keep = exp > 5
    stat = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert scipy.stats.chi2.sf(stat, keep.sum() - 1) > 1e-4


def test_sample_zero_shots_and_point_mass():
    n = 13
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[777] = 1.0
    got = core.sample(st, n, seed=3, shots=1000).cpu().numpy()
    assert np.all(got == 777)
    st[777] = 0.0
    st[(1 << n) - 1] = 1.0  # last amplitude only
    got = core.sample(st, n, seed=4, shots=1000).cpu().numpy()
    assert np.all(got == (1 << n) - 1)
    assert core.sample(st, n, seed=4, shots=0).numel() == 0


# ---------------------------------------------------------------- gradients

@pytest.mark.parametrize("n,m,p,obj", [(9, 38, 4, "p0"), (10, 42, 6, "energy"),
                                       (13, 55, 5, "p0"), (14, 60, 4, "energy")])
def test_grad_matches_reduced_adjoint_and_fd(n, m, p, obj):
    lits = instances.random_3sat(n, m, 81)
    g, b = instances.random_angles(p, 81)
    cost, hist = gpu_cost(lits, n)
    v, dg, db = core.grad(cost, n, m, g, b, obj)
    h = hist.cpu().numpy()
    code = reduced.OBJ_P0 if obj == "p0" else reduced.OBJ_ENERGY
    L, rdg, rdb = reduced.grad(h, g, b, code)
    scale = 1.0 if obj == "p0" else m / 8
    assert abs(v.item() - L) < 1e-6 * scale
    assert np.max(np.abs(dg.cpu().numpy() - rdg)) < 2e-5 * scale
    assert np.max(np.abs(db.cpu().numpy() - rdb)) < 2e-5 * scale
    fg, fb = reduced.fd_grad(h, g, b, code, step=1e-4)
    assert np.max(np.abs(dg.cpu().numpy() - fg)) < 5e-5 * scale
    assert np.max(np.abs(db.cpu().numpy() - fb)) < 5e-5 * scale


def test_grad_batched_and_autograd():
    n, m, p, B = 12, 50, 5, 4
    costs, hists = [], []
    for i in range(B):
        c, h = gpu_cost(instances.random_3sat(n, m, 300 + i), n)
        costs.append(c)
        hists.append(h.cpu().numpy())
    cost = torch.stack(costs)
    G = torch.tensor(np.stack([instances.random_angles(p, 400 + i)[0] for i in range(B)]),
                     device="cuda", requires_grad=True)
    Bt = torch.tensor(np.stack([instances.random_angles(p, 400 + i)[1] for i in range(B)]),
                      device="cuda", requires_grad=True)
    val = core.objective(G, Bt, cost, n, m, "p0")
    val.sum().backward()
    for i in range(B):
        L, rdg, rdb = reduced.grad(hists[i], G[i].detach().cpu().numpy(), Bt[i].detach().cpu().numpy())
        assert abs(val[i].item() - L) < 1e-6
        assert np.max(np.abs(G.grad[i].cpu().numpy() - rdg)) < 2e-5
        assert np.max(np.abs(Bt.grad[i].cpu().numpy() - rdb)) < 2e-5


@pytest.mark.parametrize("n", [10, 14])
def test_leading_zero_angle_rounds_are_identities(n):
    # gamma = beta = 0: phase factor exactly 1, mixer term exactly 0, so
    # padding a circuit with such rounds in front changes no bit of the state,
    # the readouts or the gradient of the real rounds (the protocol's depth
    # windows batch depths this way). The streaming passes alternate their
    # sweep direction by round parity, which fixes the order of the partial
    # sums, so the padding is even here; an odd one agrees to rounding.
    m, p, pad = 4 * n, 6, 2
    lits = instances.random_3sat(n, m, 17)
    g, b = instances.random_angles(p, 17)
    cost, _ = gpu_cost(lits, n)
    gp = np.concatenate([np.zeros(pad), g])
    bp = np.concatenate([np.zeros(pad), b])
    s1, o1, _ = core.evolve(cost, n, m, g, b)
    s2, o2, _ = core.evolve(cost, n, m, gp, bp)
    assert torch.equal(s1, s2) and torch.equal(o1, o2)
    v1, dg1, db1 = core.grad(cost, n, m, g, b, "energy")
    v2, dg2, db2 = core.grad(cost, n, m, gp, bp, "energy")
    assert torch.equal(v1, v2)
    assert torch.equal(dg1, dg2[pad:]) and torch.equal(db1, db2[pad:])


def test_single_angle_gradient_is_round_sum():
    n, m, p = 12, 50, 8
    lits = instances.random_3sat(n, m, 91)
    cost, hist = gpu_cost(lits, n)
    gam, bet = 0.37, 2.1
    _, dg, db = core.grad(cost, n, m, [gam] * p, [bet] * p)
    h = hist.cpu().numpy()
    eps = 1e-5
    fg = (reduced.objective_value(h, [gam + eps] * p, [bet] * p)
          - reduced.objective_value(h, [gam - eps] * p, [bet] * p)) / (2 * eps)
    fb = (reduced.objective_value(h, [gam] * p, [bet + eps] * p)
          - reduced.objective_value(h, [gam] * p, [bet - eps] * p)) / (2 * eps)
    assert abs(dg.sum().item() - fg) < 1e-4 and abs(db.sum().item() - fb) < 1e-4


@pytest.mark.parametrize("n", [10, 16])
def test_cuda_graph_capture_replays_bit_identical(n):
    # every C-ABI call is asynchronous and allocation-free, so the whole path
    # (cost table, p rounds with programmatic dependent launches, readout,
    # shots) can be captured once and replayed
    from paper_2402_02585_gb300 import _capi as C
    m, p, shots = 4 * n, 9, 5000
    lits = np.ascontiguousarray(instances.random_3sat(n, m, 77), dtype=np.int32)
    g, b = instances.random_angles(p, 77)
    gd = torch.as_tensor(g, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    cost = torch.empty(1 << n, dtype=torch.uint8, device="cuda")
    hist = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    state = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    sh = torch.empty(shots, dtype=torch.int64, device="cuda")
    ws = core.workspace(C.gqaoa_evolve_workspace_size(n, p))
    wss = core.workspace(C.gqaoa_sample_workspace_size(n, shots))

    def path():
        s = torch.cuda.current_stream().cuda_stream
        C.gqaoa_build_cost(lits.ctypes.data, n, m, cost.data_ptr(), hist.data_ptr(), s)
        C.gqaoa_evolve(cost.data_ptr(), n, m, gd.data_ptr(), bd.data_ptr(), p, state.data_ptr(),
                       out.data_ptr(), None, ws.data_ptr(), ws.numel(), 0, s)
        C.gqaoa_sample(state.data_ptr(), n, 3, shots, sh.data_ptr(), wss.data_ptr(), wss.numel(), s)

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        path()
    torch.cuda.synchronize()
    eager = (state.clone(), out.clone(), sh.clone(), cost.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        path()
    for t in (state, out, sh, cost):
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(state, eager[0]) and torch.equal(out, eager[1])
    assert torch.equal(sh, eager[2]) and torch.equal(cost, eager[3])
    psi = sv.evolve(sv.cost_table(lits, n)[0], n, g, b)
    assert np.max(np.abs(state.cpu().numpy() - psi)) < AMP_TOL
