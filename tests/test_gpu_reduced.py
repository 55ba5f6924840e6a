"""The cost-class (reduced) model on the GPU (gqaoa_reduced_sweep) against
the FP64 oracle.

After every round the kernel's P(C=0), <H_P> and Max-SAT weight D must agree
with oracle.reduced.readouts_trace (itself pinned against the statevector
oracle) within the complex64 tolerance used for the statevector path: P and
D within 1e-6, and <H_P> = sum_c c q_c (q the cost distribution of the state,
summing to 1) within 1e-6 times the largest cost value m, on satisfiable and unsatisfiable
instances, class counts for every lane-group shape (1 to 16 lanes per item,
groups filled or not, warps with idle groups), and batches of
instances with different clause counts; the statevector sweep (an
independent kernel family) must give the same P; the per-round argmin must be
the first minimum of the written <H_P>.
"""

import math

import numpy as np
import pytest
import torch

from oracle import reduced
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


def _hist_rows(shapes, seed0):
    rows, ms = [], []
    for i, (n, m) in enumerate(shapes):
        _, h = core.build_cost(instances.random_3sat(n, m, seed0 + i), n)
        rows.append(h.cpu().numpy())
        ms.append(m)
    stride = max(ms) + 1
    H = np.zeros((len(rows), stride), dtype=np.int64)
    for i, h in enumerate(rows):
        H[i, :h.shape[0]] = h
    return H


@pytest.mark.parametrize("n,ms,A,p", [
    (8, [5], 6, 10),             # 6 classes: one lane per item, 8 slots, 6 of a warp's 32 items
    (9, [10], 40, 12),           # 11 classes: one lane per item, 12 slots, one instance per warp
    (9, [12], 5, 10),            # 13 classes: one lane per item, 16 slots
    (8, [20], 37, 12),           # 21 classes: lane pairs, 12 slots each
    (7, [20, 30], 5, 12),        # 31 classes: lane pairs
    (6, [10, 40], 7, 12),        # 11 / 41 classes: groups of 4 lanes, partly filled
    (10, [42, 60, 90], 5, 20),   # density 9: unsatisfiable, D != P
    (14, [59], 9, 40),
    (20, [84, 100], 4, 16),
    (24, [101], 3, 8),
    (12, [180], 3, 10),          # 181 classes: groups of 16 lanes, 12 classes each
    (11, [230], 2, 6),           # 231 classes: groups of 16 lanes, 16 classes each
    (13, [55, 56], 70, 24),      # groups of 4 lanes, warps of one instance and mixed ones
])
def test_reduced_sweep_matches_oracle(n, ms, A, p):
    H = _hist_rows([(n, m) for m in ms], 3000 + n)
    rng = np.random.default_rng(n)
    G = rng.uniform(0, np.pi, A)
    Bt = rng.uniform(0, 2 * np.pi, A)
    G[0] = 0.0  # gamma = 0: <H_P> stays the mean cost
    out, best = core.reduced_sweep(torch.as_tensor(H, device="cuda"), n, G, Bt, p)
    out = out.cpu().numpy()
    for b in range(H.shape[0]):
        h = H[b, :ms[b] + 1]
        for a in range(A):
            ref = reduced.readouts_trace(h, [G[a]] * p, [Bt[a]] * p)
            got = out[b, a]
            assert np.max(np.abs(got[:, 0] - ref[:, 0])) < 1e-6, (b, a)
            assert np.max(np.abs(got[:, 2] - ref[:, 2])) < 1e-6, (b, a)
            assert np.max(np.abs(got[:, 1] - ref[:, 1])) < 1e-6 * ms[b], (b, a)
        assert abs(out[b, 0, -1, 1] - ms[b] / 8) < 1e-6 * ms[b]
    bst = best.cpu().numpy()
    for b in range(H.shape[0]):
        for k in range(p):
            assert bst[b, k] == int(np.argmin(out[b, :, k, 1]))


def test_reduced_sweep_cut_histogram():
    # a row cut after its last non-empty class (a shorter stride, so smaller
    # lane groups) gives the same readouts and argmin within the tolerance
    n, m, p = 14, 60, 32
    _, hist = core.build_cost(instances.random_3sat(n, m, 4300), n)
    h = hist.cpu().numpy()
    nz = np.nonzero(h)[0]
    rng = np.random.default_rng(5)
    G = rng.uniform(0, np.pi, 300)
    Bt = rng.uniform(0, 2 * np.pi, 300)
    full, bf = core.reduced_sweep(hist[None], n, G, Bt, p)
    cut, bc = core.reduced_sweep(hist[:nz[-1] + 1][None], n, G, Bt, p)
    assert nz[-1] + 1 <= 24 < m + 1  # lane pairs instead of groups of 4
    assert torch.max(torch.abs(full - cut)).item() < 1e-6 * m
    ref = np.stack([reduced.readouts_trace(h, [G[a]] * p, [Bt[a]] * p) for a in range(0, 300, 37)])
    got = cut[0, ::37].cpu().numpy()
    assert np.max(np.abs(got[..., 0] - ref[..., 0])) < 1e-6
    assert np.max(np.abs(got[..., 1] - ref[..., 1])) < 1e-6 * m
    e = cut[0, :, :, 1].cpu().numpy()
    assert np.array_equal(bc[0].cpu().numpy(), np.argmin(e, axis=0))


def test_reduced_sweep_agrees_with_statevector_sweep():
    n, m, p, rounds = 12, 50, 16, [1, 5, 16]
    lits = instances.random_3sat(n, m, 4100)
    cost, hist = core.build_cost(lits, n)
    rng = np.random.default_rng(12)
    G = rng.uniform(0, np.pi, 11)
    Bt = rng.uniform(0, np.pi, 11)
    out, _ = core.reduced_sweep(hist[None], n, G, Bt, p, best=False)
    r = np.asarray(rounds, dtype=np.int32)
    sv = torch.full((1, len(G), len(rounds)), -1.0, dtype=torch.float64, device="cuda")
    ws = core.workspace(C.gqaoa_sweep_workspace_size(n, len(G), 0))
    gd = torch.as_tensor(G, device="cuda")
    bd = torch.as_tensor(Bt, device="cuda")
    C.gqaoa_sweep(cost.data_ptr(), n, m, 1, gd.data_ptr(), bd.data_ptr(), len(G), p, r.ctypes.data,
                  len(rounds), 0, sv.data_ptr(), ws.data_ptr(), ws.numel(),
                  torch.cuda.current_stream().cuda_stream)
    got = out[0, :, r - 1, 0].cpu().numpy()
    assert np.max(np.abs(got - sv[0].cpu().numpy())) < 1e-6


def test_reduced_sweep_edge_cases():
    # m = 0: every assignment is a solution, P = D = 1 and <H_P> = 0 always
    H = np.array([[1 << 8]], dtype=np.int64)
    out, best = core.reduced_sweep(torch.as_tensor(H, device="cuda"), 8, [0.3, 1.1], [0.7, 2.0], 5)
    o = out.cpu().numpy()
    assert np.max(np.abs(o[..., 0] - 1)) < 1e-6 and np.max(np.abs(o[..., 2] - 1)) < 1e-6
    assert np.max(np.abs(o[..., 1])) < 1e-6
    # equal angle points: the argmin is the first of them
    H = _hist_rows([(9, 38)], 4200)
    out, best = core.reduced_sweep(torch.as_tensor(H, device="cuda"), 9, [0.5] * 4, [1.5] * 4, 6)
    assert torch.equal(out[0, 0], out[0, 3])
    assert int(best.min()) == 0 and int(best.max()) == 0
    # NaN angles: NaN readouts, and no argmin (-1)
    H1 = _hist_rows([(9, 30)], 4250)
    out, best = core.reduced_sweep(torch.as_tensor(H1, device="cuda"), 9, [float("nan")] * 3,
                                   [0.5] * 3, 4)
    assert torch.isnan(out[..., 1]).all() and int(best.max()) == -1 and int(best.min()) == -1
    # a workspace one byte short is refused before any launch
    need = C.gqaoa_reduced_sweep_workspace_size(H.shape[1], 1, 4, 6)
    ws = core.workspace(need)
    g = torch.zeros(4, dtype=torch.float64, device="cuda")
    hist = torch.as_tensor(H, device="cuda")
    o = torch.empty((1, 6, 3, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_reduced_sweep(hist.data_ptr(), H.shape[1], 9, 1, g.data_ptr(), g.data_ptr(), 4, 6,
                              o.data_ptr(), None, ws.data_ptr(), need - 1,
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.status == C.GQAOA_ENOMEM
