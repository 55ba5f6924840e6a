"""gqaoa_evolve_noalloc: the evolve entry point for callers that cannot
allocate device memory (no workspace argument; the library's fixed static
scratch is used instead). It must give the same results as gqaoa_evolve with
a caller workspace, on consecutive calls that share that scratch.

The file name sorts last, so a run that stops at its first failure has run
every other test before this one. The test does not rely on that order: it
waits for all earlier GPU work before its first call, so it passes alone in
a fresh process as well as after the other tests.
"""

import numpy as np
import pytest
import torch

from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances

pytestmark = pytest.mark.gpu


# (22, 92, 256): the streaming path on clustered CTAs at the largest round
# count the static scratch takes, i.e. its largest workspace layout
@pytest.mark.parametrize("n,m,p", [(10, 42, 8), (16, 67, 12), (20, 84, 5), (22, 92, 256)])
def test_noalloc_matches_workspace_evolve_twice(n, m, p):
    lits = instances.random_3sat(n, m, 5)
    g, b = instances.random_angles(p, 5)
    cost, _ = core.build_cost(lits, n)
    ref_state, ref_out, ref_tr = core.evolve(cost, n, m, g, b, trace=True)
    assert C.gqaoa_evolve_workspace_size(n, p) <= C.GQAOA_NOALLOC_SCRATCH_BYTES
    gd = torch.as_tensor(g, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()  # nothing else in flight may still use the shared scratch
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        state = torch.full((1 << n,), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        tr = torch.full((p,), -1.0, dtype=torch.float64, device="cuda")
        C.gqaoa_evolve_noalloc(cost.data_ptr(), n, m, gd.data_ptr(), bd.data_ptr(), p,
                               state.data_ptr(), out.data_ptr(), tr.data_ptr(), 0, stream)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(state - ref_state)).item() < 1e-5
        assert np.max(np.abs(out.cpu().numpy() - ref_out.cpu().numpy())) < 1e-6
        assert np.max(np.abs(tr.cpu().numpy() - ref_tr.cpu().numpy())) < 1e-6


def test_noalloc_rejects_too_many_rounds():
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_evolve_noalloc(1 << 20, 12, 50, 1 << 20, 1 << 20, 257, 1 << 20, None, None, 0, None)
    assert e.value.status == C.GQAOA_ERANGE
