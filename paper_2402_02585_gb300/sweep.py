"""Batched single-angle-pair sweeps (Eq. 5, Appendix C's grid scan) over many
instances of uneven n, as one replayable CUDA graph.

Instances are bucketed by n. Each bucket runs on the path the tuning table
chooses for its n:
  * "onchip": gqaoa_sweep, one CTA or thread-block cluster per
    (instance, angle point) holding the state on chip (9 <= n <= 19), with
    16 amplitudes per thread in registers ("apt": 16) or 16 more in shared
    memory ("apt": 32);
  * "l2": gqaoa_sweep's cluster-resident path (20 <= n <= 24): one 16-CTA
    cluster per item keeps part of the state in registers and shared memory
    and streams the rest through a workspace slot that stays in L2 while the
    few items in flight fit there;
  * "stream": gqaoa_evolve_batched with the instance's cost table shared by a
    chunk of angle points and a per-round trace of P(C=0).
Every buffer and workspace is allocated when the plan is built. The
gqaoa_sweep buckets (one persistent launch each) are captured into one CUDA
graph and replayed; the streaming buckets issue p + 3 launches per chunk of
several GB each, so they run eagerly after the graph (launch overhead ~2 %
there, and a graph of hundreds of thousands of nodes would cost more than it
saves).
"""

from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import _capi as C
from . import core

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def load_table(path: str = TABLE_PATH) -> dict:
    try:
        with open(path) as fh:
            return {int(k): v for k, v in json.load(fh)["sweep"].items()}
    except (OSError, KeyError, ValueError):
        return {}


def default_choice(n: int) -> dict:
    if C.GQAOA_SWEEP_MIN_N <= n <= C.GQAOA_SWEEP_MAX_N:
        return {"path": "onchip"}
    if n <= C.GQAOA_SWEEP_L2_MAX_N:
        return {"path": "l2"}
    return {"path": "stream", "angle_batch": max(1, (1 << 30) // ((1 << n) * 8))}


def sweep_apt(choice: dict) -> int:
    """The amps_per_thread argument of gqaoa_sweep for an "onchip" or "l2" choice."""
    if choice["path"] == "l2":
        return C.GQAOA_SWEEP_L2
    return int(choice.get("apt", 0))


class SweepPlan:
    """P(C=0) after `rounds` for every (instance, angle point), single angle pair.

    buckets: dict n -> (cost [B_n, 2^n] uint8 on the device, m_max)
    gammas, betas: [A] angle points; p rounds; rounds: ascending 1-based list.
    """

    def __init__(self, buckets: dict, gammas, betas, p: int, rounds, table: dict | None = None,
                 device="cuda"):
        self.device = torch.device(device)
        self.p = p
        self.rounds = np.ascontiguousarray(rounds, dtype=np.int32)
        self.R = len(self.rounds)
        self.A = len(gammas)
        self.table = table if table is not None else load_table()
        self.g = torch.as_tensor(np.asarray(gammas, np.float64), device=self.device).contiguous()
        self.b = torch.as_tensor(np.asarray(betas, np.float64), device=self.device).contiguous()
        self.gp = self.g[:, None].repeat(1, p).contiguous()  # [A, p] for the streaming path
        self.bp = self.b[:, None].repeat(1, p).contiguous()
        self.ridx = torch.as_tensor(self.rounds.astype(np.int64) - 1, device=self.device)
        self.steps = []
        self.out = {}
        for n in sorted(buckets):
            cost, m = buckets[n]
            B = cost.shape[0]
            choice = self.table.get(n, default_choice(n))
            out = torch.empty((B, self.A, self.R), dtype=torch.float64, device=self.device)
            self.out[n] = out
            if choice["path"] in ("onchip", "l2"):
                apt = sweep_apt(choice)
                ws = core.workspace(C.gqaoa_sweep_workspace_size(n, self.A, apt), self.device)
                self.steps.append((choice["path"], n, m, cost, out, (ws, apt)))
            else:
                S = int(min(self.A, choice["angle_batch"]))
                state = torch.empty((S, 1 << n), dtype=torch.complex64, device=self.device)
                trace = torch.empty((S, p), dtype=torch.float64, device=self.device)
                res = torch.empty((S, 3), dtype=torch.float64, device=self.device)
                ws = core.workspace(C.gqaoa_evolve_batched_workspace_size(n, S, p), self.device)
                self.steps.append(("stream", n, m, cost, out, (S, state, trace, res, ws)))

    def amp_rounds(self) -> int:
        return sum(st[3].shape[0] * self.A * self.p * (1 << st[1]) for st in self.steps)

    def kinds(self) -> list:
        """The paths this plan uses, in launch order."""
        return [k for k in ("onchip", "l2", "stream") if any(st[0] == k for st in self.steps)]

    def amp_rounds_of(self, kind: str) -> int:
        return sum(st[3].shape[0] * self.A * self.p * (1 << st[1]) for st in self.steps
                   if st[0] == kind)

    @staticmethod
    def lane(step) -> str:
        """"big" for the persistent launches on 16-CTA clusters (one per GPC:
        the cluster-resident path and the on-chip path at its largest n),
        "small" for the other persistent launches, "stream" otherwise."""
        kind, n = step[0], step[1]
        if kind == "l2":
            return "big"
        if kind == "onchip":
            apt = step[5][1] or (16 if n <= 18 else 32)
            return "big" if (1 << n) // apt >= 16 * 1024 else "small"
        return "stream"

    def run(self, kinds=("onchip", "l2", "stream"), lanes=("big", "small", "stream")):
        s = torch.cuda.current_stream().cuda_stream
        for step in self.steps:
            kind, n, m, cost, out, extra = step
            B = cost.shape[0]
            if kind not in kinds or self.lane(step) not in lanes:
                continue
            if kind in ("onchip", "l2"):
                ws, apt = extra
                C.gqaoa_sweep(cost.data_ptr(), n, m, B, self.g.data_ptr(), self.b.data_ptr(),
                              self.A, self.p, self.rounds.ctypes.data, self.R, apt,
                              out.data_ptr(), ws.data_ptr(), ws.numel(), s)
                continue
            S, state, trace, res, ws = extra
            for i in range(B):
                for a0 in range(0, self.A, S):
                    k = min(S, self.A - a0)
                    C.gqaoa_evolve_batched(cost[i].data_ptr(), 0, n, m, k,
                                           self.gp[a0].data_ptr(), self.bp[a0].data_ptr(), self.p,
                                           state.data_ptr(), res.data_ptr(), trace.data_ptr(),
                                           ws.data_ptr(), ws.numel(), 0, s)
                    out[i, a0:a0 + k].copy_(trace[:k].index_select(1, self.ridx))
        return self.out

    def capture(self):
        """Record the persistent gqaoa_sweep launches into one CUDA graph per
        path ("onchip", "l2") and one per lane ("big", "small"), after one
        eager warm-up run of everything."""
        self.run()
        torch.cuda.synchronize()
        self.graphs = {}
        for kind in ("onchip", "l2"):
            if kind in self.kinds():
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self.run(kinds=(kind,))
                self.graphs[kind] = g
        self.lane_graphs = {}
        for lane in ("big", "small"):
            if any(self.lane(st) == lane for st in self.steps):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self.run(lanes=(lane,))
                self.lane_graphs[lane] = g
        # the 16-CTA-cluster lane on a high-priority stream: when SMs free up,
        # the scheduler places its pending clusters before the smaller CTAs
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") \
            else (0, -1)
        self._big = torch.cuda.Stream(self.device, priority=hi)
        self._side = torch.cuda.Stream(self.device, priority=lo)
        return self.graphs

    def replay(self):
        """One path after the other (each path's launches alone on the GPU)."""
        for g in self.graphs.values():
            g.replay()
        self.run(kinds=("stream",))
        return self.out

    def replay_concurrent(self):
        """The 16-CTA-cluster launches first, on a high-priority stream, and
        the other persistent launches on a low-priority one: a 16-CTA
        cluster occupies a whole GPC and only seven are resident on GB300, so
        the smaller items fill the SMs those clusters leave idle. Items are
        independent; the outputs are those of replay()."""
        main = torch.cuda.current_stream(self.device)
        fork = torch.cuda.Event()
        fork.record(main)
        for lane, stream in (("big", self._big), ("small", self._side)):
            if lane in self.lane_graphs:
                stream.wait_event(fork)
                with torch.cuda.stream(stream):
                    self.lane_graphs[lane].replay()
                main.wait_stream(stream)
        self.run(kinds=("stream",))
        return self.out


def grid_angles(k: int = 32):
    """The k x k grid over [0, pi)^2 with left endpoints: gamma_i = i pi / k,
    beta_j = j pi / k (gamma-major)."""
    G = np.repeat(np.arange(k) * np.pi / k, k)
    B = np.tile(np.arange(k) * np.pi / k, k)
    return G, B
