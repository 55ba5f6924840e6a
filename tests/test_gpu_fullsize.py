"""Parity at the benchmark's full size, in the launch configuration bench.py
times: n = 28, m = 118 (seed 0), p = 100 random angles, 10^6 shots, through
gqaoa_build_cost / gqaoa_evolve / gqaoa_sample with caller-owned buffers.

The oracle checks every output it can compute one by one: the whole cost
table and histogram (FP64 C oracle, all 2^28 assignments), every amplitude
psi_p(z) = f_p(C(z)) from the exact cost-class model (pinned against the
full statevector oracle at small n), P(C=0), and each shot against the exact
cumulative distribution.
"""

import numpy as np
import pytest
import torch

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances
from tests.shot_compare import compare_same_state

pytestmark = pytest.mark.gpu

N_VARS, M_CLAUSES, P_ROUNDS, SHOTS, SEED = 28, 118, 100, 1_000_000, 0


@pytest.fixture(scope="module")
def run():
    n, m, p = N_VARS, M_CLAUSES, P_ROUNDS
    N = 1 << n
    lits = instances.random_3sat(n, m, SEED)
    g, b = instances.random_angles(p, SEED)
    dev = torch.device("cuda")
    s = torch.cuda.current_stream().cuda_stream
    cost = torch.empty(N, dtype=torch.uint8, device=dev)
    hist = torch.empty(m + 1, dtype=torch.int64, device=dev)
    state = torch.empty(N, dtype=torch.complex64, device=dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    trace = torch.empty(p, dtype=torch.float64, device=dev)
    shots = torch.empty(SHOTS, dtype=torch.int64, device=dev)
    gd = torch.as_tensor(g, device=dev)
    bd = torch.as_tensor(b, device=dev)
    ws_ev = core.workspace(C.gqaoa_evolve_workspace_size(n, p))
    ws_sa = core.workspace(C.gqaoa_sample_workspace_size(n, SHOTS))
    lc = np.ascontiguousarray(lits, dtype=np.int32)
    C.gqaoa_build_cost(lc.ctypes.data, n, m, cost.data_ptr(), hist.data_ptr(), s)
    C.gqaoa_evolve(cost.data_ptr(), n, m, gd.data_ptr(), bd.data_ptr(), p, state.data_ptr(),
                   out.data_ptr(), trace.data_ptr(), ws_ev.data_ptr(), ws_ev.numel(), 0, s)
    C.gqaoa_sample(state.data_ptr(), n, 12345, SHOTS, shots.data_ptr(), ws_sa.data_ptr(),
                   ws_sa.numel(), s)
    torch.cuda.synchronize()
    ref_cost, ref_hist = sv.cost_table(lits, n)
    f = reduced.evolve(ref_hist, g, b)
    return dict(lits=lits, g=g, b=b, cost=cost.cpu().numpy(), hist=hist.cpu().numpy(),
                state=state, out=out.cpu().numpy(), trace=trace.cpu().numpy(),
                shots=shots.cpu().numpy(), ref_cost=ref_cost, ref_hist=ref_hist, f=f)


def test_cost_table_and_histogram_bit_exact(run):
    assert np.array_equal(run["cost"], run["ref_cost"])
    assert np.array_equal(run["hist"].astype(np.uint64), run["ref_hist"])


def test_every_amplitude_matches_cost_class_model(run):
    f = run["f"].astype(np.complex64)
    cost = torch.as_tensor(run["ref_cost"].astype(np.int64), device="cuda")
    ref = torch.as_tensor(f, device="cuda")[cost]
    err = torch.max(torch.abs(run["state"] - ref)).item()
    assert err < 1e-5, err
    # also relative to the amplitude scale 2^-14 of this size
    assert err < 0.01 * 2.0 ** -14


def test_readout_and_trace(run):
    # P(C=0) is about 7e-8 here, so an absolute 1e-6 would accept P = 0: the
    # solution probability and its per-round trace are bounded relative to
    # their own size (complex64 rounding over 100 rounds moves P by ~1e-6 of
    # itself; 1e-4 leaves that margin and still catches a wrong amplitude)
    h = run["ref_hist"]
    _, tr = reduced.evolve(h, run["g"], run["b"], trace=True)
    r = reduced.readout(h, run["f"])
    rel = abs(run["out"][0] - r[0]) / r[0]
    rel_tr = np.max(np.abs(run["trace"] - tr) / (tr + 1e-300))
    print(f"P(C=0) = {run['out'][0]:.6e} (oracle {r[0]:.6e}), relative error {rel:.2e}; "
          f"largest relative error of the per-round trace {rel_tr:.2e}")
    assert r[0] > 0 and abs(run["out"][0] - r[0]) <= 1e-4 * r[0] + 1e-12
    assert np.all(np.abs(run["trace"] - tr) <= 1e-4 * tr + 1e-12)
    assert abs(run["out"][1] - r[1]) < 1e-4 * M_CLAUSES / 8
    assert abs(run["out"][2] - 1.0) < 1e-5


def test_shots_valid_against_exact_cdf(run):
    # exact distribution: |f_p(C(z))|^2, CDF in index order (FP64)
    w = (np.abs(run["f"]) ** 2)[run["ref_cost"]]
    cdf = np.cumsum(w)
    total = cdf[-1]
    shots = run["shots"]
    assert shots.min() >= 0 and shots.max() < (1 << N_VARS)
    sel = np.arange(0, SHOTS, 97)  # every 97th shot: the oracle's uniforms one by one
    u = np.array([sv.shot_uniform(12345, int(s)) for s in sel])
    t = u * total
    z = shots[sel]
    lo = np.where(z > 0, cdf[np.maximum(z - 1, 0)], 0.0)
    hi = cdf[z]
    # Single probabilities are ~2^-28 here while the complex64 state moves the
    # CDF by up to ~1e-6 of the total, so the exact index can shift by
    # hundreds of amplitudes; what must hold is that every shot's target lies
    # in its amplitude's CDF interval up to that state error.
    tol = 1e-5 * total
    miss = np.maximum(np.maximum(lo - t, t - hi), 0.0)
    assert np.max(miss) <= tol, np.max(miss) / total


def test_shots_match_oracle_on_the_same_state(run):
    # the oracle samples the GPU's own complex64 state (upcast to FP64): the
    # shots are index work and must be identical except where a target lies
    # within the CDFs' rounding (a few FP64 units of the norm) of a boundary
    psi = run["state"].cpu().numpy().astype(np.complex128)
    ref, cdf = sv.sample(psi, N_VARS, seed=12345, shots=SHOTS, return_cdf=True)
    del psi
    compare_same_state(run["shots"], ref, cdf, 12345, eps=1e-14 * cdf[-1], label="n=28")


def test_fused_evolve_sample_equals_separate_calls(run):
    # the benchmark's call: gqaoa_evolve_sample adds a_p on the fly instead of
    # materialising psi_p; readouts and every one of the 10^6 shots must equal
    # those of gqaoa_evolve followed by gqaoa_sample
    n, m, p = N_VARS, M_CLAUSES, P_ROUNDS
    dev = torch.device("cuda")
    s = torch.cuda.current_stream().cuda_stream
    cost = torch.as_tensor(run["cost"], device=dev)
    gd = torch.as_tensor(run["g"], device=dev)
    bd = torch.as_tensor(run["b"], device=dev)
    state = torch.empty(1 << n, dtype=torch.complex64, device=dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    trace = torch.empty(p, dtype=torch.float64, device=dev)
    shots = torch.empty(SHOTS, dtype=torch.int64, device=dev)
    ws = core.workspace(C.gqaoa_evolve_sample_workspace_size(n, p, SHOTS))
    C.gqaoa_evolve_sample(cost.data_ptr(), n, m, gd.data_ptr(), bd.data_ptr(), p, state.data_ptr(),
                          out.data_ptr(), trace.data_ptr(), 12345, SHOTS, shots.data_ptr(),
                          ws.data_ptr(), ws.numel(), 0, s)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), run["out"])
    assert np.array_equal(trace.cpu().numpy(), run["trace"])
    assert np.array_equal(shots.cpu().numpy(), run["shots"])


def test_shot_classes_follow_cost_class_weights(run):
    import scipy.stats
    c = run["ref_cost"][run["shots"]]
    h = run["ref_hist"].astype(np.float64)
    wts = h * np.abs(run["f"]) ** 2
    obs = np.bincount(c, minlength=len(h)).astype(np.float64)
    exp = wts / wts.sum() * SHOTS
    keep = exp > 5
    stat = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert scipy.stats.chi2.sf(stat, keep.sum() - 1) > 1e-4
    assert obs[~keep].sum() <= exp[~keep].sum() * 3 + 30
