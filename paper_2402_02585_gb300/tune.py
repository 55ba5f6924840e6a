"""Autotuner of the sweep paths: times the candidate execution shapes per n on
the current GPU with CUDA events and writes the winning choice per n to a
JSON table that SweepPlan loads.

    python -m paper_2402_02585_gb300.tune [--out PATH] [--n 12 13 ...]

Candidates: the on-chip sweep with 16 amplitudes per thread in registers
(9 <= n <= 18) or 16 more in shared memory (10 <= n <= 19), the
cluster-resident sweep with L2-resident workspace slots (20 <= n <= 24), and
the streaming path with chunks of 16..256 angle points sharing the instance's
cost table. The score is
amplitude-rounds per second on a small synthetic bucket of the workload's
recipe (d = 4.2, p = 16).
"""

from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import _capi as C
from . import core, instances
from .sweep import SweepPlan


def _time_plan(plan: SweepPlan, reps: int = 3) -> float:
    plan.run()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        plan.run()
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / 1e3 / reps


def tune(n_values, p: int = 16, angles: int = 256, verbose: bool = True) -> dict:
    table = {}
    for n in n_values:
        m = int(math.floor(4.2 * n + 0.5))
        B = max(1, min(8, (1 << 20) >> n))
        cost = torch.stack([core.build_cost(instances.random_3sat(n, m, 5000 + i), n)[0]
                            for i in range(B)])
        rng = np.random.default_rng(n)
        G = rng.uniform(0, np.pi, angles)
        Bt = rng.uniform(0, np.pi, angles)
        cands = []
        if C.GQAOA_SWEEP_MIN_N <= n <= 18:
            cands.append({"path": "onchip", "apt": 16})
        if 10 <= n <= C.GQAOA_SWEEP_MAX_N:
            cands.append({"path": "onchip", "apt": 32})
        if C.GQAOA_SWEEP_L2_MIN_N <= n <= C.GQAOA_SWEEP_L2_MAX_N:
            cands.append({"path": "l2"})
        for S in (16, 64, 256):
            if S <= angles and (S << n) * 8 <= (4 << 30):
                cands.append({"path": "stream", "angle_batch": S})
        best = None
        for cand in cands:
            try:
                plan = SweepPlan({n: (cost, m)}, G, Bt, p, [p], table={n: cand})
                t = _time_plan(plan)
            except C.GQAOAError as exc:  # a shape this GPU cannot launch
                if verbose:
                    print(f"n={n} {cand}: {exc}")
                continue
            rate = plan.amp_rounds() / t
            if verbose:
                print(f"n={n} {cand}: {rate:.3e} amp-rounds/s")
            if best is None or rate > best[0]:
                best = (rate, cand)
        table[n] = dict(best[1], amp_rounds_per_s=best[0])
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--n", type=int, nargs="*", default=list(range(9, 23)))
    ap.add_argument("--p", type=int, default=16)
    args = ap.parse_args()
    table = tune(args.n, p=args.p)
    doc = {"gpu": torch.cuda.get_device_name(), "p": args.p, "sweep": table}
    text = json.dumps(doc, indent=1, sort_keys=True)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
