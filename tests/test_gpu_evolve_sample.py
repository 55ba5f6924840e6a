"""gqaoa_evolve_sample against gqaoa_evolve followed by gqaoa_sample.

The fused call never writes psi_p = chi_p + a_p back: the readout pass and
the sampler add a_p to chi_p as they read it, with the same FP32 addition the
materialising pass makes, and the readouts come from the same reduction. So
the readouts, the per-round trace and every shot must equal those of the two
separate calls exactly, on the fused path (2^n >= 4096 amplitudes and at
most 64 shots per 4096 amplitudes) and on the fallback paths (one-CTA
states, resident-tile and bucketed sampling).
"""

import numpy as np
import pytest
import torch

from oracle import statevector as sv
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,shots,trace,cls,state_in", [
    (16, 1000, True, 0, False),      # fused
    (20, 16000, False, 0, False),    # fused, about 62 shots per tile
    (18, 4000, False, "min", False),  # fused, Max-SAT class readout
    (17, 2000, True, 0, True),       # fused, from a given initial state
    (10, 5000, True, 0, False),      # one-CTA state: evolve, then sample
    (14, 3000, False, 0, False),     # four tiles: resident-tile sampler
    (16, 200000, True, 0, False),    # many shots per tile: bucketed sampler
])
def test_evolve_sample_equals_evolve_then_sample(n, shots, trace, cls, state_in):
    m, p, seed = 4 * n + 3, 9, 40 + n
    lits = instances.random_3sat(n, m, seed)
    g, b = instances.random_angles(p, seed)
    cost, hist = core.build_cost(lits, n)
    c = int(np.nonzero(hist.cpu().numpy())[0][0]) if cls == "min" else cls
    psi0 = None
    if state_in:
        psi0 = torch.as_tensor(instances.random_state(n, seed).astype(np.complex64), device="cuda")
    st = psi0.clone() if state_in else None
    state, out, tr = core.evolve(cost, n, m, g, b, state=st, state_in=state_in, trace=trace,
                                 readout_class=c)
    ref_shots = core.sample(state, n, seed=99, shots=shots)
    st2 = psi0.clone() if state_in else None
    out2, tr2, shots2 = core.evolve_sample(cost, n, m, g, b, seed=99, shots=shots, state=st2,
                                           state_in=state_in, trace=trace, readout_class=c)
    torch.cuda.synchronize()
    assert torch.equal(out2, out), (out2, out)
    if trace:
        assert torch.equal(tr2, tr)
    assert torch.equal(shots2, ref_shots)


def test_evolve_sample_matches_oracle_shots():
    # and against the oracle's sampler on the materialised state (same-state
    # parity as for gqaoa_sample)
    from tests.shot_compare import compare_same_state
    n, m, p, shots = 18, 76, 12, 40000
    lits = instances.random_3sat(n, m, 7)
    g, b = instances.random_angles(p, 7)
    cost, _ = core.build_cost(lits, n)
    state, _, _ = core.evolve(cost, n, m, g, b)
    _, _, got = core.evolve_sample(cost, n, m, g, b, seed=5, shots=shots)
    psi = state.cpu().numpy().astype(np.complex128)
    ref, cdf = sv.sample(psi, n, seed=5, shots=shots, return_cdf=True)
    compare_same_state(got.cpu().numpy(), ref, cdf, 5, eps=1e-14 * cdf[-1], label="fused n=18")
