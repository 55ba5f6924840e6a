"""Multi-GPU host logic: sharding and the per-round scalar combiner.

Independent problems (instances, angle points) shard with no exchange: each
rank takes every world-th unit and the job's throughput is the units of all
ranks over the slowest rank's time (weak scaling). One instance split over
ranks partitions z by its top log2(world) bits; the only exchange per round
is the mixer sum S_k = sum_z chi_k(z), a complex FP64 scalar (16 bytes).
`Combiner` all-gathers the per-rank partial sums and adds them in rank order,
so every rank derives the same S_k bit for bit whatever the backend's own
reduction order (gloo on CPU, NCCL on GPUs).
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(N: int, rank: int, world: int) -> tuple[int, int]:
    """[z0, z1) of rank's slice: the top log2(world) bits of z equal rank."""
    if world < 1 or world & (world - 1) or world > N:
        raise ValueError("world must be a power of two not larger than N")
    per = N // world
    return rank * per, (rank + 1) * per


def partition(count: int, rank: int, world: int) -> list[int]:
    """Unit indices of this rank for independent problems (round robin)."""
    return list(range(rank, count, world))


class Combiner:
    """Deterministic all-reduce of complex FP64 partial sums."""

    def __init__(self, group=None, device="cpu"):
        self.group = group
        self.world = dist.get_world_size(group)
        self.device = torch.device(device)
        self.buf = torch.zeros((self.world, 2), dtype=torch.float64, device=self.device)

    def sum(self, partial: complex) -> complex:
        mine = torch.tensor([[partial.real, partial.imag]], dtype=torch.float64, device=self.device)
        parts = list(self.buf.unbind(0))
        dist.all_gather(parts, mine[0], group=self.group)
        re = 0.0
        im = 0.0
        for r in range(self.world):  # fixed rank order
            re += float(parts[r][0])
            im += float(parts[r][1])
        return complex(re, im)


def max_over_ranks(seconds: float, group=None, device="cpu") -> float:
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(units: int, group=None, device="cpu") -> int:
    t = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())
