"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it cannot agree with by
construction: brute force, a closed form, a textbook special case, a library
routine, or numbers the paper prints.
"""

import itertools
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import protocol, reduced, statevector as sv
from paper_2402_02585_gb300 import instances
from tests.golden_io import paper_instances


def brute_cost(lits, n):
    """Appendix B, written as plain Python loops over assignments and literals."""
    out = []
    for z in range(1 << n):
        tau = [(z >> v) & 1 for v in range(n)]
        unsat = 0
        for clause in lits:
            ok = False
            for lit in clause:
                v = abs(int(lit)) - 1
                if (lit > 0 and tau[v] == 1) or (lit < 0 and tau[v] == 0):
                    ok = True
            unsat += 0 if ok else 1
        out.append(unsat)
    return np.array(out)


# --------------------------------------------------------------------------
# cost table and histogram
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,seed", [(3, 1, 0), (4, 8, 1), (5, 21, 2), (6, 25, 3), (8, 34, 4)])
def test_cost_table_matches_brute_force(n, m, seed):
    lits = instances.random_3sat(n, m, seed)
    cost, hist = sv.cost_table(lits, n)
    ref = brute_cost(lits, n)
    assert np.array_equal(cost.astype(np.int64), ref)
    assert np.array_equal(hist, np.bincount(ref, minlength=m + 1).astype(np.uint64))


@pytest.mark.parametrize("n,m,seed", [(10, 42, 0), (12, 50, 7), (14, 70, 9)])
def test_histogram_closed_forms(n, m, seed):
    # Each clause has 3 distinct variables, so exactly 1/8 of the 2^n
    # assignments violate it: sum_c c h[c] = m 2^{n-3}; and sum_c h[c] = 2^n.
    lits = instances.random_3sat(n, m, seed)
    hist = sv.histogram(lits, n).astype(np.int64)
    assert hist.sum() == 1 << n
    assert int(np.dot(np.arange(m + 1), hist)) == m * (1 << (n - 3))


def test_cost_single_clause_counts():
    # One clause over n variables: 2^{n-3} violating assignments (Eq. 1 is a
    # rank-1 projector on the three variables).
    for n in range(3, 9):
        for sgn in itertools.product((1, -1), repeat=3):
            lits = np.array([[sgn[0] * 1, sgn[1] * 2, sgn[2] * n]], np.int32)
            _, hist = sv.cost_table(lits, n)
            assert hist.tolist() == [(1 << n) - (1 << (n - 3)), 1 << (n - 3)]


@pytest.mark.parametrize("n", [6, 10, 13, 17])
def test_disjoint_clauses_binomial_histogram(n):
    # Clauses on disjoint variable triples violate independently, each on 1 of
    # its 8 assignments: h[c] = binom(m, c) 7^(m - c) 2^(n - 3m).
    m = n // 3
    rng = np.random.default_rng(n)
    var = rng.permutation(n)[: 3 * m]
    lits = ((var + 1) * rng.choice([-1, 1], size=3 * m)).reshape(m, 3).astype(np.int32)
    want = [math.comb(m, c) * 7 ** (m - c) * 2 ** (n - 3 * m) for c in range(m + 1)]
    assert sv.histogram(lits, n).tolist() == want


def test_cost_at_matches_table():
    lits = instances.random_3sat(11, 46, 5)
    cost, _ = sv.cost_table(lits, 11)
    for z in [0, 1, 77, 1023, 2047]:
        assert sv.cost_at(lits, z) == cost[z]


def test_cost_rejects_bad_literals():
    with pytest.raises(ValueError):
        sv.cost_table(np.array([[1, 2, 9]], np.int32), 4)
    with pytest.raises(ValueError):
        sv.cost_table(np.array([[1, 0, 2]], np.int32), 4)


def test_paper_instances_solution_counts():
    # Section IV footnote instances; the counts follow from brute force.
    for inst in paper_instances():
        cost, hist = sv.cost_table(inst["lits"], inst["n"])
        ref = brute_cost(inst["lits"], inst["n"])
        assert int(hist[0]) == int(np.sum(ref == 0))
        assert np.array_equal(cost.astype(np.int64), ref)


# --------------------------------------------------------------------------
# evolution
# --------------------------------------------------------------------------

def dense_evolution(cost, n, gammas, betas):
    """Eq. 3 with dense matrices: expm of H_P = diag(C) and H_M = |+><+|."""
    N = 1 << n
    plus = np.full(N, 1 / math.sqrt(N), dtype=np.complex128)
    HM = np.outer(plus, plus.conj())
    HP = np.diag(cost.astype(np.float64))
    psi = plus.copy()
    for g, b in zip(gammas, betas):
        psi = scipy.linalg.expm(-1j * g * HP) @ psi
        psi = scipy.linalg.expm(-1j * b * HM) @ psi
    return psi


@pytest.mark.parametrize("n,m,p,seed", [(3, 2, 1, 0), (4, 8, 3, 1), (5, 14, 4, 2)])
def test_evolve_matches_dense_expm(n, m, p, seed):
    lits = instances.random_3sat(n, m, seed)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, seed)
    psi = sv.evolve(cost, n, g, b)
    ref = dense_evolution(cost, n, g, b)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_p1_closed_form():
    # One round from |+>: psi_1(z) = N^{-1/2}(e^{-i g C(z)} + (e^{-i b} - 1) hh(g))
    # with hh(g) = sum_c h[c] e^{-i g c} / N, so
    # P = (h[0]/N) |1 + (e^{-i b} - 1) hh(g)|^2.
    n, m = 8, 30
    lits = instances.random_3sat(n, m, 11)
    cost, hist = sv.cost_table(lits, n)
    N = 1 << n
    for g, b in [(0.3, 1.1), (2.0, 0.4), (1.234, 2.9)]:
        hh = np.sum(hist.astype(float) * np.exp(-1j * g * np.arange(m + 1))) / N
        P = hist[0] / N * abs(1 + (np.exp(-1j * b) - 1) * hh) ** 2
        psi = sv.evolve(cost, n, [g], [b])
        assert abs(sv.readout(psi, cost, n)[0] - P) < 1e-13
        # the phase sign matters: e^{+i g C} gives a different value here
        Pwrong = hist[0] / N * abs(1 + (np.exp(-1j * b) - 1) * np.conj(hh)) ** 2
        assert abs(Pwrong - P) > 1e-6


@pytest.mark.parametrize("n,k_max", [(6, 6), (9, 12)])
def test_grover_special_case(n, k_max):
    # Appendix A / Grover: a single clause makes C take values {0, 1}; at
    # gamma = beta = pi each round is (up to sign) a Grover iteration that
    # amplifies the C=1 states, so after k rounds their weight is
    # sin^2((2k+1) theta) with sin^2 theta = h[1]/N.
    lits = np.array([[1, -2, 3]], np.int32)
    cost, hist = sv.cost_table(lits, n)
    theta = math.asin(math.sqrt(hist[1] / (1 << n)))
    for k in range(1, k_max + 1):
        psi = sv.evolve(cost, n, [math.pi] * k, [math.pi] * k)
        r = sv.readout(psi, cost, n)
        w1 = r[1]  # <H_P> = weight of the C=1 class here
        assert abs(w1 - math.sin((2 * k + 1) * theta) ** 2) < 1e-12


def test_zero_angles_leave_random_guess():
    lits = instances.random_3sat(9, 36, 3)
    cost, hist = sv.cost_table(lits, 9)
    g, b = instances.random_angles(5, 3)
    for gg, bb in [(np.zeros(5), b), (g, np.zeros(5))]:
        psi = sv.evolve(cost, 9, gg, bb)
        assert abs(sv.readout(psi, cost, 9)[0] - hist[0] / 512) < 1e-13


def test_norm_and_fairness():
    n, m, p = 11, 46, 20
    lits = instances.random_3sat(n, m, 4)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 4)
    psi = sv.evolve(cost, n, g, b)
    assert abs(sv.readout(psi, cost, n)[2] - 1.0) < 1e-12
    # every state in one cost class carries the same amplitude, hence every
    # solution has the same probability (the fair-sampling property)
    for c in np.unique(cost):
        sel = psi[cost == c]
        assert np.max(np.abs(sel - sel[0])) < 1e-13


def test_arbitrary_initial_state_dense():
    n, m, p = 5, 12, 3
    lits = instances.random_3sat(n, m, 8)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 8)
    psi0 = instances.random_state(n, 8)
    N = 1 << n
    plus = np.full(N, 1 / math.sqrt(N))
    ref = psi0.copy()
    for gg, bb in zip(g, b):
        ref = np.exp(-1j * gg * cost) * ref
        ref = scipy.linalg.expm(-1j * bb * np.outer(plus, plus)) @ ref
    psi = sv.evolve(cost, n, g, b, psi0=psi0)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_trace_matches_prefix_runs():
    n, m, p = 8, 33, 12
    lits = instances.random_3sat(n, m, 6)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 6)
    _, tr = sv.evolve(cost, n, g, b, trace=True)
    for k in (1, 4, 12):
        psi = sv.evolve(cost, n, g[:k], b[:k])
        assert abs(sv.readout(psi, cost, n)[0] - tr[k - 1]) < 1e-14


# --------------------------------------------------------------------------
# reduced (m+1)-dimensional model (Appendix C)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,p,seed", [(6, 26, 5, 0), (10, 42, 8, 0), (12, 50, 30, 1)])
def test_reduced_equals_statevector(n, m, p, seed):
    lits = instances.random_3sat(n, m, seed)
    cost, hist = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, seed)
    psi = sv.evolve(cost, n, g, b)
    f = reduced.evolve(hist, g, b)
    assert np.max(np.abs(psi - reduced.amplitudes(f, cost))) < 1e-13
    assert np.allclose(reduced.readout(hist, f), sv.readout(psi, cost, n), atol=1e-13, rtol=0)


@pytest.mark.parametrize("objective", [reduced.OBJ_P0, reduced.OBJ_ENERGY])
def test_reduced_grad_matches_finite_differences(objective):
    n, m, p = 10, 42, 6
    lits = instances.random_3sat(n, m, 2)
    _, hist = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 2)
    L, dg, db = reduced.grad(hist, g, b, objective)
    assert abs(L - reduced.objective_value(hist, g, b, objective)) < 1e-14
    fg, fb = reduced.fd_grad(hist, g, b, objective, step=1e-5)
    scale = 1.0 if objective == reduced.OBJ_P0 else m / 8
    assert np.max(np.abs(dg - fg)) < 1e-8 * scale
    assert np.max(np.abs(db - fb)) < 1e-8 * scale


def test_reduced_grad_matches_statevector_fd():
    n, m, p = 7, 28, 3
    lits = instances.random_3sat(n, m, 12)
    cost, hist = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 12)
    _, dg, db = reduced.grad(hist, g, b)
    h = 1e-4
    for k in range(p):
        for arr, ref in ((g, dg), (b, db)):
            a0 = arr[k]
            arr[k] = a0 + h
            up = sv.readout(sv.evolve(cost, n, g, b), cost, n)[0]
            arr[k] = a0 - h
            dn = sv.readout(sv.evolve(cost, n, g, b), cost, n)[0]
            arr[k] = a0
            assert abs((up - dn) / (2 * h) - ref[k]) < 1e-7


def test_reduced_readouts_trace_matches_statevector_unsat():
    # n = 7 at density 9: unsatisfiable, so the lowest class c* > 0 and
    # D = sum over C(z) = c* of |psi|^2 is read off the statevector directly
    n, m, p = 7, 63, 6
    lits = instances.random_3sat(n, m, 21)
    cost, hist = sv.cost_table(lits, n)
    cs = reduced.min_class(hist)
    assert cs > 0 and hist[cs] > 0 and np.all(np.asarray(hist)[:cs] == 0)
    assert cs == int(np.min(cost))
    g, b = instances.random_angles(p, 21)
    tr = reduced.readouts_trace(hist, g, b)
    for k in range(1, p + 1):
        psi = sv.evolve(cost, n, g[:k], b[:k])
        w = np.abs(psi) ** 2
        assert abs(tr[k - 1, 0] - w[cost == 0].sum()) < 1e-14      # P = 0 here
        assert abs(tr[k - 1, 1] - np.sum(cost * w)) < 1e-12
        assert abs(tr[k - 1, 2] - w[cost == cs].sum()) < 1e-14


def test_reduced_readouts_trace_satisfiable_and_gamma_zero():
    n, m, p = 9, 38, 5
    lits = instances.random_3sat(n, m, 21)   # satisfiable (4 solutions)
    cost, hist = sv.cost_table(lits, n)
    assert hist[0] > 0 and reduced.min_class(hist) == 0
    g, b = instances.random_angles(p, 21)
    tr = reduced.readouts_trace(hist, g, b)
    assert np.array_equal(tr[:, 0], tr[:, 2])                        # D = P when satisfiable
    _, trp = reduced.evolve(hist, g, b, trace=True)
    assert np.max(np.abs(tr[:, 0] - trp)) < 1e-15
    # gamma = 0: the phase is the identity and |+> is the mixer's fixed point,
    # so <H_P> stays the mean cost, m / 8 for clauses over distinct variables
    tr0 = reduced.readouts_trace(hist, np.zeros(p), b)
    assert np.max(np.abs(tr0[:, 1] - m / 8)) < 1e-12
    assert np.max(np.abs(tr0[:, 0] - hist[0] / 2 ** n)) < 1e-15


def test_reduced_class_gradient_matches_statevector_fd_unsat():
    # the Max-SAT objective D (probability of the lowest non-empty class) of an
    # unsatisfiable instance: adjoint against central differences of the
    # statevector oracle's class weight
    n, m, p = 7, 63, 4
    lits = instances.random_3sat(n, m, 21)
    cost, hist = sv.cost_table(lits, n)
    cs = reduced.min_class(hist)
    assert cs > 0
    g, b = instances.random_angles(p, 23)
    L, dg, db = reduced.grad(hist, g, b, reduced.OBJ_P0, target=cs)
    psi = sv.evolve(cost, n, g, b)
    assert abs(L - np.sum(np.abs(psi[cost == cs]) ** 2)) < 1e-14
    h = 1e-4
    for k in range(p):
        for arr, ref in ((g, dg), (b, db)):
            a0 = arr[k]
            arr[k] = a0 + h
            up = np.sum(np.abs(sv.evolve(cost, n, g, b)[cost == cs]) ** 2)
            arr[k] = a0 - h
            dn = np.sum(np.abs(sv.evolve(cost, n, g, b)[cost == cs]) ** 2)
            arr[k] = a0
            assert abs((up - dn) / (2 * h) - ref[k]) < 1e-7


def test_single_angle_gradient_is_sum_over_rounds():
    n, m, p = 9, 38, 7
    lits = instances.random_3sat(n, m, 13)
    _, hist = sv.cost_table(lits, n)
    gam, bet = 0.4, 2.2
    _, dg, db = reduced.grad(hist, [gam] * p, [bet] * p)
    h = 1e-5
    fg = (reduced.objective_value(hist, [gam + h] * p, [bet] * p)
          - reduced.objective_value(hist, [gam - h] * p, [bet] * p)) / (2 * h)
    fb = (reduced.objective_value(hist, [gam] * p, [bet + h] * p)
          - reduced.objective_value(hist, [gam] * p, [bet - h] * p)) / (2 * h)
    assert abs(dg.sum() - fg) < 1e-8 and abs(db.sum() - fb) < 1e-8


# --------------------------------------------------------------------------
# Table I: noiseless G-QAOA solution probability of the worked instances
# --------------------------------------------------------------------------

def _energy_optimal_P(hist, p):
    """Minimise <H_P> (Eq. 4) the way Appendix C describes, with the protocol
    oracle's steps: a grid over the single angle pair (pi/90 here), then
    L-BFGS-B over all 2p angles. The paper does not print its angles, so the
    40 best grid seeds are refined and the lowest energy kept (one more
    local optimum of the same landscape would otherwise decide the test)."""
    G, B = instances.protocol_grid(2)
    G = np.concatenate([G, 2 * np.pi - G])  # both halves of the torus
    B = np.concatenate([B, (2 * np.pi - B) % (2 * np.pi)])
    E, _, _ = protocol.grid_readouts(hist, G, B, p)
    best = None
    for a in np.argsort(E[:, p - 1], kind="stable")[:40]:
        g, b, e, _ = protocol.refine(hist, [G[a]] * p, [B[a]] * p, single=False)
        if best is None or e < best[2] - 1e-12:
            best = (g, b, e)
    f = reduced.evolve(hist, best[0], best[1])
    return reduced.readout(hist, f)[0]


def _two_class(M: int, N: int) -> np.ndarray:
    """A cost-class histogram with M solutions and N - M assignments of cost 1."""
    return np.array([M, N - M], dtype=np.int64)


def test_two_class_model_is_grover_at_pi_pi():
    # costs in {0, 1}: e^{-i pi C} = -(-1)^{[C=0]} and e^{-i pi} - 1 = -2, so a
    # round at (gamma, beta) = (pi, pi) is Grover's iteration up to a global
    # sign and P after k rounds is sin^2((2k + 1) theta), sin^2 theta = M / N
    M, N, p = 3, 1024, 12
    theta = math.asin(math.sqrt(M / N))
    tr = reduced.readouts_trace(_two_class(M, N), [math.pi] * p, [math.pi] * p)
    k = np.arange(1, p + 1)
    assert np.max(np.abs(tr[:, 0] - np.sin((2 * k + 1) * theta) ** 2)) < 1e-12
    assert np.max(np.abs(tr[:, 1] - (1 - tr[:, 0]))) < 1e-12        # <H_P> = 1 - P


def test_protocol_min_rounds_two_class_closed_form():
    # Two classes: <H_P> = 1 - P, so the protocol maximises P; with k oracle
    # rounds no choice of phases beats sin^2((2k + 1) theta) while
    # (2k + 1) theta <= pi/2, and (pi, pi) on the grid attains it, so the fewest
    # rounds reaching P >= 1/2 is the smallest k with (2k + 1) theta >= pi/4
    M, N = 3, 1024
    theta = math.asin(math.sqrt(M / N))
    k_star = math.ceil((math.pi / (4 * theta) - 1) / 2)
    G, B = instances.protocol_grid(4)
    k, g, b, val, e = protocol.min_rounds(_two_class(M, N), G, B, S=0.5, p_max=16)
    assert k == k_star == 7
    assert abs(val - math.sin((2 * k + 1) * theta) ** 2) < 1e-9
    assert abs(e - (1 - val)) < 1e-9


def test_protocol_refines_every_depth():
    # Appendix C optimises every depth from its grid seed. Here the accepted
    # depth of the per-round-angle protocol has a seed below S/2, which
    # L-BFGS-B over the 2k angles lifts above S; the depth before it stays
    # below S after the same refinement.
    n, m, seed = 10, 35, 21
    _, hist = sv.cost_table(instances.random_3sat(n, m, seed), n)
    G, B = instances.protocol_grid(2)
    k, g, b, val, e = protocol.min_rounds(hist, G, B, S=0.5, p_max=24, single=False)
    assert k == 17 and val >= 0.5
    E, P, _ = protocol.grid_readouts(hist, G, B, k)
    a = int(np.argmin(E[:, k - 1]))
    assert P[a, k - 1] < 0.25
    a = int(np.argmin(E[:, k - 2]))
    g1, b1, _, _ = protocol.refine(hist, [G[a]] * (k - 1), [B[a]] * (k - 1), single=False)
    assert reduced.readouts_trace(hist, g1, b1)[-1][0] < 0.5


def test_protocol_grid_readouts_match_single_evolutions():
    n, m, p = 8, 34, 9
    _, hist = sv.cost_table(instances.random_3sat(n, m, 31), n)
    G, B = instances.protocol_random_angles(6, 31)
    E, P, D = protocol.grid_readouts(hist, G, B, p)
    for a in range(6):
        tr = reduced.readouts_trace(hist, [G[a]] * p, [B[a]] * p)
        assert np.max(np.abs(P[a] - tr[:, 0])) < 1e-13
        assert np.max(np.abs(E[a] - tr[:, 1])) < 1e-12
        assert np.max(np.abs(D[a] - tr[:, 2])) < 1e-13


def test_table1_noiseless_solution_probability():
    # Table I prints the noiseless solution % of G-QAOA at p = 1, 2 for the
    # Section IV instances, at angles that minimise <H_P>. The paper rounds to
    # 0.1 pp and does not print its angles; 0.25 pp covers the rounding and a
    # slightly different local optimum of the same landscape.
    for inst in paper_instances():
        _, hist = sv.cost_table(inst["lits"], inst["n"])
        for p in (1, 2):
            P = _energy_optimal_P(hist, p)
            assert abs(100 * P - inst["table1"][f"p{p}"]) < 0.25, (inst["name"], p, 100 * P)


# --------------------------------------------------------------------------
# Philox4x32-10 and sampling
# --------------------------------------------------------------------------

def test_philox_known_answers():
    # Known-answer vectors published with Random123 for philox4x32_10.
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert sv.philox4x32_10(ctr, key).tolist() == want


def test_sample_is_inverse_cdf():
    n, m, p = 10, 42, 6
    lits = instances.random_3sat(n, m, 0)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 0)
    psi = sv.evolve(cost, n, g, b)
    shots, cdf = sv.sample(psi, n, seed=1234, shots=5000, return_cdf=True)
    assert np.allclose(cdf, np.cumsum(np.abs(psi) ** 2), rtol=0, atol=1e-14)
    u = np.array([sv.shot_uniform(1234, s) for s in range(5000)])
    ref = np.searchsorted(cdf, u * cdf[-1], side="right")
    assert np.array_equal(shots, ref.astype(np.uint32))


def test_sample_cdf_is_exact_sum_of_weights():
    # Every assignment of one cost class has the same weight, so a plain FP64
    # running sum rounds the same way again and again and drifts; the CDF must
    # instead stay within a few units in the last place of the exact prefix
    # sum (checked in rational arithmetic) over 2^20 terms.
    from fractions import Fraction
    n = 20
    a = float(np.float32(0.3))  # a complex64 amplitude: a^2 is exact in FP64
    psi = np.full(1 << n, a, dtype=np.complex128)
    _, cdf = sv.sample(psi, n, seed=1, shots=1, return_cdf=True)
    w = Fraction(a * a)
    assert a * a == float(w)
    for z in (0, 1, 1000, 123457, (1 << 19) + 3, (1 << n) - 1):
        exact = (z + 1) * w
        assert abs(Fraction(cdf[z]) - exact) <= 4 * np.spacing(cdf[z]), z
    run = np.cumsum(np.full(1 << n, a * a))  # the plain running sum drifts here
    assert abs(Fraction(run[-1]) - (1 << n) * w) > 100 * np.spacing(run[-1])


def test_sample_distribution_chi_square():
    import scipy.stats
    n, m, p = 6, 24, 4
    lits = instances.random_3sat(n, m, 5)
    cost, _ = sv.cost_table(lits, n)
    g, b = instances.random_angles(p, 5)
    psi = sv.evolve(cost, n, g, b)
    prob = np.abs(psi) ** 2
    shots = sv.sample(psi, n, seed=7, shots=200000)
    counts = np.bincount(shots, minlength=1 << n)
    keep = prob * 200000 > 5
    stat = np.sum((counts[keep] - 200000 * prob[keep]) ** 2 / (200000 * prob[keep]))
    assert scipy.stats.chi2.sf(stat, keep.sum() - 1) > 1e-4
    assert counts[~keep].sum() <= 200000 * prob[~keep].sum() * 3 + 20


def test_uniforms_in_unit_interval():
    u = np.array([sv.shot_uniform(99, s) for s in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01


def test_readout_of_uniform_state():
    # |+> weighs every assignment 2^-n: P = h[0]/2^n and, each clause being
    # violated by 1/8 of the assignments, <H_P> = m/8
    n, m = 9, 37
    lits = instances.random_3sat(n, m, 14)
    cost, hist = sv.cost_table(lits, n)
    r = sv.readout(sv.plus_state(n), cost, n)
    assert abs(r[0] - hist[0] / (1 << n)) < 1e-15
    assert abs(r[1] - m / 8) < 1e-12
    assert abs(r[2] - 1.0) < 1e-14
