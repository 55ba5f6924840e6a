"""C-ABI library checks that need no GPU: it loads, exports every declared
symbol, sizes workspaces and rejects bad arguments before launching."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gqaoa_\w+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    # and the binding covers each of them
    for s in syms:
        assert s in C.SIGNATURES, s


def test_version_and_strerror():
    assert C.gqaoa_version() >= 100
    for code in (0, -1, -2, -3, -4, -5):
        assert C.strerror(code)
    assert C.strerror(-99) == "unknown status"


def test_workspace_sizes_monotone():
    a = C.gqaoa_evolve_workspace_size(20, 10)
    b = C.gqaoa_evolve_workspace_size(20, 100)
    assert b > a > 0
    g1 = C.gqaoa_grad_workspace_size(16, 4)
    assert g1 >= 4 * (1 << 16) * 8
    gb = C.gqaoa_grad_batched_workspace_size(16, 8, 4)
    assert gb >= 8 * 4 * (1 << 16) * 8
    s = C.gqaoa_sample_workspace_size(20, 1000)
    assert s > 1000 * 4
    assert C.gqaoa_prob_workspace_size(28) > 0


def test_evolve_sample_workspace_and_arguments():
    # the fused call's workspace holds the evolution's and the sampler's
    assert C.gqaoa_evolve_sample_workspace_size(20, 8, 1000) >= (
        C.gqaoa_evolve_workspace_size(20, 8) + C.gqaoa_sample_workspace_size(20, 1000))
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_evolve_sample_workspace_size(20, 8, 1 << 32)
    assert e.value.status == C.GQAOA_ERANGE
    fake = 1 << 20
    with pytest.raises(C.GQAOAError) as e:  # a workspace one byte short, before any launch
        need = C.gqaoa_evolve_sample_workspace_size(20, 8, 1000)
        C.gqaoa_evolve_sample(fake, 20, 84, fake, fake, 8, fake, None, None, 1, 1000, fake, fake,
                              need - 1, 0, None)
    assert e.value.status == C.GQAOA_ENOMEM
    ws = C.gqaoa_evolve_sample_workspace_size(20, 8, 1000)
    bad = [
        # (n, shots, out_idx, trace, flags) -> status, all before any launch
        ((20, 1000, fake, fake, C.GQAOA_READOUT_CLASS(3)), C.GQAOA_EINVAL),  # class + trace
        ((20, 1000, fake, None, 1 << 20), C.GQAOA_EINVAL),                    # unknown flag
        ((20, 1000, None, None, 0), C.GQAOA_EINVAL),                          # shots, no output
        ((20, -1, fake, None, 0), C.GQAOA_ERANGE),
        ((40, 1000, fake, None, 0), C.GQAOA_ERANGE),
        ((20, 1000, fake + 4, None, 0), C.GQAOA_EINVAL),                      # misaligned
    ]
    for (n, shots, oi, tr, flags), code in bad:
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_evolve_sample(fake, n, 84, fake, fake, 8, fake, None, tr, 1, shots, oi, fake,
                                  ws, flags, None)
        assert e.value.status == code, (n, shots, flags)


def test_batched_geometry_query():
    # below one 4096-amplitude tile an instance is one CTA; at n = 16 a batch
    # spreads each instance over several CTAs and reduction records, never
    # more CTAs than tiles. (Without a device the library assumes 152 SMs.)
    assert C.gqaoa_batched_geometry(11, 64, 0) == (1, 1)
    for B in (8, 64, 1024):
        for adjoint in (0, 1):
            cpi, rec = C.gqaoa_batched_geometry(16, B, adjoint)
            assert 1 <= rec <= cpi <= 16
    cpi, rec = C.gqaoa_batched_geometry(16, 64, 1)
    assert cpi >= 2 and rec == cpi  # a batch runs without clusters
    cpi, rec = C.gqaoa_batched_geometry(24, 1, 0)
    assert cpi > rec >= 1  # one instance: clusters of CTAs, one record per cluster
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_batched_geometry(16, 0, 0)
    assert e.value.status == C.GQAOA_ERANGE


@pytest.mark.parametrize("args,code", [
    ((0, 10), C.GQAOA_ERANGE),
    ((35, 10), C.GQAOA_ERANGE),
    ((10, 0), C.GQAOA_ERANGE),
])
def test_workspace_size_ranges(args, code):
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_evolve_workspace_size(*args)
    assert e.value.status == code


def test_build_cost_rejects_bad_literals_before_launch():
    lits = np.array([[1, 2, 9]], dtype=np.int32)  # |9| > n
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_build_cost(lits.ctypes.data, 4, 1, 16, None, None)
    assert e.value.status == C.GQAOA_EINVAL
    lits = np.array([[1, 0, 2]], dtype=np.int32)
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_build_cost(lits.ctypes.data, 4, 1, 16, None, None)
    assert e.value.status == C.GQAOA_EINVAL
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_build_cost(lits.ctypes.data, 40, 1, 16, None, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_build_cost(lits.ctypes.data, 4, 300, 16, None, None)
    assert e.value.status == C.GQAOA_ERANGE


def test_evolve_rejects_bad_arguments_before_launch():
    fake = 1 << 20  # aligned non-null addresses; nothing is dereferenced
    ws = C.gqaoa_evolve_workspace_size(12, 4)
    cases = [
        ((0, 12, 10, fake, fake, 4, fake, None, None, fake, ws, 0, None), C.GQAOA_EINVAL),  # null cost
        ((fake, 12, 10, fake, fake, 0, fake, None, None, fake, ws, 0, None), C.GQAOA_ERANGE),  # p = 0
        ((fake, 12, 10, fake, fake, 4, fake + 8, None, None, fake, ws, 0, None), C.GQAOA_EINVAL),
        ((fake, 12, 10, fake, fake, 4, fake, None, None, fake, ws - 1, 0, None), C.GQAOA_ENOMEM),
        ((fake, 12, 10, fake, fake, 4, fake, None, None, fake, ws, 4, None), C.GQAOA_EINVAL),  # flag
        ((fake, 12, 256, fake, fake, 4, fake, None, None, fake, ws, 0, None), C.GQAOA_ERANGE),
    ]
    for args, code in cases:
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_evolve(*args)
        assert e.value.status == code, args


def test_sample_and_grad_reject_bad_arguments_before_launch():
    fake = 1 << 20
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sample(fake, 20, 1, -1, fake, fake, 1 << 30, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sample(fake, 20, 1, 100, fake, fake, 16, None)
    assert e.value.status == C.GQAOA_ENOMEM
    # shot numbers and per-tile offsets are 32-bit: 2^32 shots is out of range
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sample(fake, 20, 1, 1 << 32, fake, fake, 1 << 40, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sample_workspace_size(20, 1 << 32)
    assert e.value.status == C.GQAOA_ERANGE
    assert C.gqaoa_sample_workspace_size(20, (1 << 32) - 1) > 0
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_grad(fake, 16, 60, fake, fake, 4, 7, fake, fake, fake, fake, 1 << 40, None)
    assert e.value.status == C.GQAOA_EINVAL
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_grad(fake, 16, 60, fake, fake, 4, 0, fake, fake, fake, fake, 1024, None)
    assert e.value.status == C.GQAOA_ENOMEM


def test_reduced_sweep_rejects_bad_arguments_before_launch():
    fake = 1 << 20
    for args in ((fake, 257, 10, 1, fake, fake, 4, 4, fake, None, fake, 1 << 20, None),   # stride
                 (fake, 43, 0, 1, fake, fake, 4, 4, fake, None, fake, 1 << 20, None),     # n
                 (fake, 43, 10, 1, fake, fake, 4, 0, fake, None, fake, 1 << 20, None)):   # p
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_reduced_sweep(*args)
        assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:  # misaligned output (FP32: 4-byte aligned)
        C.gqaoa_reduced_sweep(fake, 43, 10, 1, fake, fake, 4, 4, fake + 2, None, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_EINVAL
    # phase tables of 64 entries (stride 43 rounded up to 32), alpha, the
    # minima of 1 x 4 rounds, the per-warp minima (4 lanes per item: 8 items
    # per warp, one block), two FP32 weight rows of 64 entries and the lowest
    # class per instance, each region 256-byte aligned
    need = C.gqaoa_reduced_sweep_workspace_size(43, 1, 4, 4)
    assert need == 4 * 64 * 8 + 6 * 256
    # 16 lanes per item: 2 items per warp, 15 blocks of 30 items x 7 rounds
    assert (C.gqaoa_reduced_sweep_workspace_size(256, 3, 10, 7)
            == 10 * 256 * 8 + 256 + 256 + 1024 + 2 * 3 * 256 * 4 + 256)
    for bad in ((0, 1, 4, 4), (257, 1, 4, 4), (43, 0, 4, 4), (43, 1, 0, 4), (43, 1, 4, 0),
                (43, 1 << 12, 4, 1 << 19)):  # batch * p = 2^31
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_reduced_sweep_workspace_size(*bad)
        assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:  # batch * p = 2^31, refused before any launch
        C.gqaoa_reduced_sweep(fake, 43, 10, 1 << 12, fake, fake, 4, 1 << 19, fake, None, fake,
                              1 << 40, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_reduced_sweep(fake, 43, 10, 1, fake, fake, 4, 4, fake, None, fake, need - 1, None)
    assert e.value.status == C.GQAOA_ENOMEM


def test_sweep_workspace_sizes():
    small = C.gqaoa_sweep_workspace_size(12, 4, 0)
    assert 0 < small < 1 << 16
    # [A][256] complex64 phase tables | [A] complex128 mixer coefficients |
    # a 256-byte block for the status word of the clusters' bounded waits,
    # each part starting on a 256-byte boundary
    up = lambda b: (b + 255) // 256 * 256
    for A in (1, 4, 33):
        assert C.gqaoa_sweep_workspace_size(12, A, 0) == up(8 * 256 * A) + up(16 * A) + 256
    assert C.gqaoa_sweep_workspace_size(19, 4, 32) == small
    resident = C.gqaoa_sweep_workspace_size(20, 4, C.GQAOA_SWEEP_L2)
    assert resident == small + 16 * 8 * (1 << 20)       # 16 slots of 2^20 complex64
    assert C.gqaoa_sweep_workspace_size(20, 4, 0) == resident
    for n, apt in ((20, 16), (20, 32), (25, 0), (19, C.GQAOA_SWEEP_L2)):
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_sweep_workspace_size(n, 4, apt)
        assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sweep_workspace_size(12, 4, 8)
    assert e.value.status == C.GQAOA_EINVAL


def test_sweep_rejects_bad_arguments_before_launch():
    fake = 1 << 20
    r = np.array([2, 1], dtype=np.int32)
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sweep(fake, 12, 50, 1, fake, fake, 4, 4, r.ctypes.data, 2, 0, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_EINVAL
    r = np.array([5], dtype=np.int32)
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sweep(fake, 12, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, 0, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_ERANGE
    r = np.array([4], dtype=np.int32)
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sweep(fake, 25, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, 0, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:  # the cluster-resident path starts at n = 20
        C.gqaoa_sweep(fake, 19, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, C.GQAOA_SWEEP_L2, fake,
                      fake, 1 << 30, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:  # 16 slots of 2^20 amplitudes do not fit in 1 MiB
        C.gqaoa_sweep(fake, 20, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, 0, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_ENOMEM
    with pytest.raises(C.GQAOAError) as e:  # 16 per thread cannot hold n = 19
        C.gqaoa_sweep(fake, 19, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, 16, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_ERANGE
    with pytest.raises(C.GQAOAError) as e:
        C.gqaoa_sweep(fake, 12, 50, 1, fake, fake, 4, 4, r.ctypes.data, 1, 8, fake, fake, 1 << 20, None)
    assert e.value.status == C.GQAOA_EINVAL


def test_fairness_workspace_and_bad_arguments_before_launch():
    fake = 1 << 20
    runs, targets = 1000, 25
    need = C.gqaoa_fairness_workspace_size(14, runs, targets)
    # a label per assignment, a counter, and the per-run counts of every target
    assert need >= 4 * (1 << 14) + 4 * runs * targets
    for args in ((0, runs, targets), (31, runs, targets), (14, 0, targets), (14, runs, 0),
                 (4, runs, 17)):  # more targets than assignments
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_fairness_workspace_size(*args)
        assert e.value.status == C.GQAOA_ERANGE, args
    ok = (fake, runs, 2048, fake, 14, 0, targets, 36.4, 125, fake, fake, fake, need, None)

    def call(**kw):
        a = list(ok)
        for k, v in kw.items():
            a[{"shots": 0, "runs": 1, "per_run": 2, "n": 4, "target": 5, "targets": 6,
               "min_draws": 8, "to_all": 9, "ws_bytes": 12}[k]] = v
        with pytest.raises(C.GQAOAError) as e:
            C.gqaoa_fairness(*a)
        return e.value.status

    assert call(n=31) == C.GQAOA_ERANGE
    assert call(target=256) == C.GQAOA_ERANGE
    assert call(targets=0) == C.GQAOA_ERANGE
    assert call(min_draws=0) == C.GQAOA_ERANGE
    assert call(per_run=-1) == C.GQAOA_ERANGE
    assert call(per_run=1 << 31, targets=1 << 12) == C.GQAOA_ERANGE  # M sum O^2 would overflow
    assert call(shots=0) == C.GQAOA_EINVAL
    assert call(to_all=fake + 4) == C.GQAOA_EINVAL  # misaligned output
    assert call(ws_bytes=need - 1) == C.GQAOA_ENOMEM


def test_gradient_path_helpers_agree():
    # grad_launches and grad_hbm_bytes follow the same choice of path: the
    # state stays on chip (cluster-resident adjoint, or the one-CTA kernels)
    # exactly where the streaming passes' 2p + 3 launches are not made
    from paper_2402_02585_gb300 import core
    for p in (1, 4, 32):
        for n in range(6, 29):
            for streaming in (False, True):
                on_chip = core.grad_launches(n, p, streaming) != 2 * p + 3
                assert (core.grad_hbm_bytes(n, p, streaming) == 1 + 16 * p) == on_chip, (n, p, streaming)
    assert core.grad_hbm_bytes(16, 32) < core.grad_hbm_bytes(16, 32, streaming=True)
