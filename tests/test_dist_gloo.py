"""Multi-rank host logic on CPU with gloo, world size 2 (no GPU).

An instance whose state is split by the top bit of z over two ranks must
evolve exactly like the single-process oracle when the only exchange per
round is the Combiner's 16-byte sum; the weak-scaling helpers must partition
units disjointly and report the slowest rank's time.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import statevector as sv
from paper_2402_02585_gb300 import dist as gdist
from paper_2402_02585_gb300 import instances

N_VARS, M, P = 10, 42, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lits = instances.random_3sat(N_VARS, M, 3)
        cost, _ = sv.cost_table(lits, N_VARS)
        g, b = instances.random_angles(P, 3)
        N = 1 << N_VARS
        z0, z1 = gdist.shard_range(N, rank, world)
        c = cost[z0:z1].astype(np.float64)
        psi = np.full(z1 - z0, 1 / np.sqrt(N), dtype=np.complex128)
        comb = gdist.Combiner()
        for k in range(P):
            # this rank's slice of one round (test-side arithmetic); the mixer
            # needs the global sum, which only the combiner provides
            psi = np.exp(-1j * g[k] * c) * psi
            S = comb.sum(complex(psi.sum()))
            psi = psi + (np.exp(-1j * b[k]) - 1) * S / N
        units = gdist.partition(11, rank, world)
        t = gdist.max_over_ranks(0.5 + rank)
        total = gdist.sum_over_ranks(len(units))
        q.put((rank, z0, psi, units, t, total, S))
    finally:
        dist.destroy_process_group()


def test_sharded_rounds_with_combiner_match_oracle():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    lits = instances.random_3sat(N_VARS, M, 3)
    cost, _ = sv.cost_table(lits, N_VARS)
    g, b = instances.random_angles(P, 3)
    ref = sv.evolve(cost, N_VARS, g, b)
    full = np.concatenate([r[2] for r in res])
    assert np.max(np.abs(full - ref)) < 1e-13
    # both ranks derived the identical last sum
    assert res[0][6] == res[1][6]
    # disjoint round-robin partition covering all units; slowest time; unit total
    assert sorted(res[0][3] + res[1][3]) == list(range(11))
    assert not set(res[0][3]) & set(res[1][3])
    assert res[0][4] == res[1][4] == 1.5
    assert res[0][5] == 11


def test_shard_range_rules():
    assert gdist.shard_range(16, 1, 4) == (4, 8)
    with pytest.raises(ValueError):
        gdist.shard_range(16, 0, 3)
    with pytest.raises(ValueError):
        gdist.shard_range(2, 0, 4)
