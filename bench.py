"""Benchmark of the G-QAOA statevector hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|small]

Workload "large" (default): one random 3-SAT instance with n = 28 variables
and m = 118 clauses (d ~ 4.2, seed 0), p = 100 G-QAOA rounds with angles
uniform in [0, pi), 10^6 fair-sampled shots. A step is the whole hot path on
that input: cost table + histogram, p fused rounds + final readout, shots.
Metric: amplitude-rounds per second, p * 2^n per step, whole job.

Under torchrun (N > 1) each rank runs its own instance (seed = rank): the
problems are independent, so there is no collective on the data path;
value = all ranks' amplitude-rounds / max-over-ranks time ("weak" scaling).

--impl reference times the FP64 CPU oracle (the plain reference written from
the paper) on the host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (n, d, p, shots, seed)
    "large": dict(n=28, m=118, p=100, shots=1_000_000, seed=0,
                  desc="random 3-SAT n=28 m=118 (d~4.2) seed 0, p=100 random angles, 1e6 shots"),
    "small": dict(n=10, m=42, p=8, shots=10_000, seed=0,
                  desc="random 3-SAT n=10 m=42 (d=4.2) seed 0, p=8 random angles, 1e4 shots"),
    # the batched single-angle-pair sweep: one step = the whole sweep
    "sweep": dict(kind="sweep", count=4096, grid=32, p=64, rounds=[1, 4, 16, 64], seed=0,
                  desc="4096 random 3-SAT instances, n uniform in 12..20, d in {3.0, 4.2, 5.0}; "
                       "single angle pair on a 32x32 grid over [0,pi)^2, p=64 with P read out "
                       "at p=1,4,16,64 (prefix reuse); one CUDA graph per step"),
    # batched adjoint gradient + Adam over all 2p angles (one step = one Adam step)
    "grad": dict(kind="grad", n=16, m=67, p=32, batch=1024, seed=0, lr=0.05,
                 desc="1024 random 3-SAT instances n=16 m=67 (d~4.2), p=32 random angles; "
                      "one step = adjoint gradient of P(C=0) for all + one Adam update (lr 0.05)"),
    # the gradient's profiling case: same recipe, 512 instances, p = 4 (256 MiB per
    # state pass, 1 GiB of checkpoints: larger than L2, small enough for ncu)
    "grad_profile": dict(kind="grad", n=16, m=67, p=4, batch=512, seed=0, lr=0.05,
                         desc="512 random 3-SAT instances n=16 m=67 (d~4.2), p=4 random angles; "
                              "one step = adjoint gradient of P(C=0) for all + one Adam update"),
    # the paper's angle protocol (Appendix C) on satisfiable instances of
    # Section III's density range; one step = the protocol for every instance
    "protocol": dict(kind="protocol", count=32, n_values=list(range(10, 17)), d_lo=2.0, d_hi=4.5,
                     S=0.5, p_max=64, seed=0, window=16, workers=4,
                     desc="32 satisfiable random 3-SAT instances, n uniform in 10..16, d uniform "
                          "in (2, 4.5); pi/180 <H_P> grid (cost-class model), L-BFGS-B with "
                          "statevector adjoint gradients, fewest single-angle-pair rounds to "
                          "P >= 50 % on the statevector"),
    # the same protocol for Max-SAT on unsatisfiable instances of the (4.6, 8)
    # range, target D = probability of the lowest non-empty cost class
    "protocol_maxsat": dict(kind="protocol", count=32, n_values=list(range(10, 17)), d_lo=4.6,
                            d_hi=8.0, S=0.5, p_max=64, seed=1, target="D", window=16, workers=4,
                            desc="32 unsatisfiable random 3-SAT instances, n uniform in 10..16, d "
                                 "uniform in (4.6, 8); pi/180 <H_P> grid (cost-class model), "
                                 "L-BFGS-B with statevector adjoint gradients, fewest "
                                 "single-angle-pair rounds to a Max-SAT probability D >= 50 % on "
                                 "the statevector"),
    # the same protocol over the paper's sizes (Section III: up to 26 qubits;
    # the pi/180 grid up to n = 20, 4000 sampled angle pairs above), for the
    # fitted exponent of the fewest rounds against 1/P over that range; a
    # warm-up pass runs the first warm_count instances only
    "protocol_scaling": dict(kind="protocol", count=45, n_values=list(range(10, 25)), d_lo=2.0,
                             d_hi=4.5, S=0.5, p_max=64, retry_p_max=256, seed=2, warm_count=4,
                             window=8, workers=4,
                             desc="45 satisfiable random 3-SAT instances, n uniform in 10..24, d "
                                  "uniform in (2, 4.5); <H_P> on the pi/180 grid (n <= 20) or 4000 "
                                  "sampled angle pairs (n > 20) by the cost-class model, L-BFGS-B "
                                  "with statevector adjoint gradients at every depth, fewest "
                                  "single-angle-pair rounds to P >= 50 % on the statevector"),
    # Section IV's fair-sampling metrics on a satisfiable instance at the
    # protocol's fewest-rounds angles: one step = sample runs x shots_per_run
    # shots and compute both metrics for every run
    "grid": dict(kind="grid", n=16, m=67, p=64, seed=0,
                 desc="cost-class model (Appendix C) of the first satisfiable random 3-SAT "
                      "instance n=16 m=67 (d~4.2) from seed 0, histogram cut after its last "
                      "non-empty class: the pi/180 grid (65160 single angle pairs) x p = 64 "
                      "rounds, P/<H_P>/D after every round and the per-round argmin of <H_P>"),
    "fairness": dict(kind="fairness", n=14, d_lo=3.8, d_hi=4.2, runs=100_000, shots_per_run=2048,
                     alpha=0.05, seed=3,
                     desc="one satisfiable random 3-SAT instance n=14, d in (3.8, 4.2), at the "
                          "protocol's fewest single-angle-pair rounds to P >= 50 %; 100000 runs "
                          "of 2048 shots from gqaoa_sample; shots to see every solution and "
                          "chi-square draws (alpha 0.05, from 5 M draws) to reject uniform "
                          "solution sampling, per run"),
    # the learned angle proposer (config 5): labels from the batched gradient
    # optimizer on 20000 training instances, the MLP trained on them, and the
    # wall time to 95 % of the plain optimizer's P(C=0) on 2000 held-out n = 20
    # instances; one step = the whole study (a warm-up step is the same study
    # at 1/100 of the instance counts)
    "study": dict(kind="study", train=20000, train_n=list(range(10, 19)), test=2000, test_n=[20],
                  d_lo=3.0, d_hi=5.0, p=16, seed=0,
                  desc="learned angle proposer: MLP 130-256-256-32 (GELU) trained on 20000 "
                       "satisfiable random 3-SAT instances, n uniform in 10..18, d uniform in "
                       "[3, 5], labels from Adam over all 2p angles (p = 16) after a 16x16 "
                       "single-angle-pair grid; evaluated on 2000 satisfiable n = 20 instances: "
                       "wall time to 95 % of the plain optimizer's final P(C=0)"),
    # the profiling case: same recipe, state (512 MiB) still far larger than L2
    "profile": dict(n=26, m=109, p=8, shots=100_000, seed=0,
                    desc="random 3-SAT n=26 m=109 (d~4.2) seed 0, p=8 random angles, 1e5 shots"),
}
METRIC = "G-QAOA amp-rounds/s"
UNIT = "amp-rounds/s"
PEAK_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (100 ms period)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- peaks / profiles
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return PEAK_FALLBACK_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the fused round's source: its tile pipeline and kernel, and the
    grid geometry it is launched with (an edit elsewhere in the file does not
    change the kernel the ncu counters were taken on)."""
    path = os.path.join(ROOT, "paper_2402_02585_gb300", "csrc", "stream.cu")
    with open(path) as fh:
        text = fh.read()
    k0 = text.index("struct TileRegs {")
    k1 = text.index("// K4: readout")
    g0 = text.index("static Geometry make_geometry(")
    g1 = text.index("\n}\n", g0)
    part = text[k0:k1] + text[g0:g1]
    return hashlib.sha256(part.encode()).hexdigest()[:16]


def profiled_traffic(n: int):
    """dram bytes per round-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "round_kernel.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    mh = re.search(r"round kernel source sha256\[:16\]:\s*`?([0-9a-f]{16})", text)
    mt = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not mh or not mt or mh.group(1) != kernel_source_hash():
        return None
    return float(mt.group(1))


# ----------------------------------------------------------------- oracle (CPU) timing
class OracleSample:
    """The FP64 oracle on a bounded sample of the workload.

    The cost table is built once at the workload's full n (timed); a step
    sample then times `rounds` statevector rounds on the full 2^n state and
    `shots` of the workload's shots. One step is extrapolated as
    cost table + p x (time per round) + (time per shot) x all shots."""

    def __init__(self, wl: dict, rounds: int = 1, shots: int = 50_000):
        from oracle import statevector as sv
        from paper_2402_02585_gb300 import instances
        self.sv = sv
        self.wl = wl
        self.rounds = min(rounds, wl["p"])
        self.shots = min(shots, wl["shots"])
        n, m, p = wl["n"], wl["m"], wl["p"]
        lits = instances.random_3sat(n, m, wl["seed"])
        self.g, self.b = instances.random_angles(p, wl["seed"])
        t0 = time.perf_counter()
        self.cost, _ = sv.cost_table(lits, n)
        self.t_cost = time.perf_counter() - t0
        self.cores = sv.num_threads()

    def one_core(self) -> float:
        """amp-rounds/s of one statevector round on a single host thread."""
        sv, wl = self.sv, self.wl
        full = sv.num_threads()
        sv.set_threads(1)
        try:
            t0 = time.perf_counter()
            sv.evolve(self.cost, wl["n"], self.g[:1], self.b[:1])
            t = time.perf_counter() - t0
        finally:
            sv.set_threads(full)
        return (1 << wl["n"]) / t

    def reduced_context(self) -> float:
        """Seconds of the paper's own method (Appendix C) for the same P:
        the (m+1)-dimensional cost-class evolution, after the histogram that
        the cost-table time above already includes."""
        from oracle import reduced
        hist = np.bincount(self.cost, minlength=self.wl["m"] + 1)
        t0 = time.perf_counter()
        reduced.readout(hist, reduced.evolve(hist, self.g, self.b))
        return time.perf_counter() - t0

    def step(self):
        sv, wl = self.sv, self.wl
        n, p = wl["n"], wl["p"]
        t1 = time.perf_counter()
        psi = sv.evolve(self.cost, n, self.g[:self.rounds], self.b[:self.rounds])
        t2 = time.perf_counter()
        sv.sample(psi, n, seed=1, shots=self.shots)
        t3 = time.perf_counter()
        t_round = (t2 - t1) / self.rounds
        t_shots = (t3 - t2) * wl["shots"] / self.shots
        step = self.t_cost + p * t_round + t_shots
        self.desc = (f"n={n} m={wl['m']}: full FP64 cost table once ({self.t_cost:.2f} s), "
                     f"{self.rounds} of {p} rounds on the full state ({t_round:.3f} s/round), "
                     f"{self.shots} of {wl['shots']} shots ({t3 - t2:.2f} s); step = cost table "
                     f"+ {p} rounds + all shots, extrapolated linearly")
        return p * (1 << n) / step, step


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    total_t0 = time.perf_counter()
    sample = OracleSample(wl)
    per_step = []
    for i in range(args.warmup + args.steps):
        _, step = sample.step()
        if i >= args.warmup:
            per_step.append(step)
    step = float(np.mean(per_step))
    value = wl["p"] * (1 << wl["n"]) / step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["desc"], "n": wl["n"], "m": wl["m"],
                                        "p": wl["p"], "shots": wl["shots"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sample.cores, "kind": "oracle",
                         "sample": sample.desc, "cpu_model": cpu_model(),
                         "one_core_round_amp_rounds_per_s": sample.one_core(),
                         "context_reduced_model_s": sample.reduced_context()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - total_t0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    from paper_2402_02585_gb300 import _capi as C
    from paper_2402_02585_gb300 import core, instances

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    C.load()

    n, m, p, shots = wl["n"], wl["m"], wl["p"], wl["shots"]
    seed = wl["seed"] + rank
    N = 1 << n
    lits = instances.random_3sat(n, m, seed)
    g_np, b_np = instances.random_angles(p, seed)
    gam = torch.as_tensor(g_np, device=dev)
    bet = torch.as_tensor(b_np, device=dev)

    # caller-owned device buffers, allocated once
    cost = torch.empty(N, dtype=torch.uint8, device=dev)
    hist = torch.empty(m + 1, dtype=torch.int64, device=dev)
    state = torch.empty(N, dtype=torch.complex64, device=dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    shots_out = torch.empty(shots, dtype=torch.int64, device=dev)
    ws_es = core.workspace(C.gqaoa_evolve_sample_workspace_size(n, p, shots), dev)
    lits_c = np.ascontiguousarray(lits, dtype=np.int32)
    sh = stream.cuda_stream
    # the fused call (rounds, readout pass with the sampler's tile pass, the
    # tile scan, the shots) applies when 2^n >= 4096 and shots <= 64 per tile
    fused = N >= 4096 and shots <= 64 * (N // 4096) and N // 4096 > 8

    ev_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]

    def step(pair=None):
        C.gqaoa_build_cost(lits_c.ctypes.data, n, m, cost.data_ptr(), hist.data_ptr(), sh)
        if pair:
            pair[0].record(stream)
        C.gqaoa_evolve_sample(cost.data_ptr(), n, m, gam.data_ptr(), bet.data_ptr(), p,
                              state.data_ptr(), out.data_ptr(), None, 12345, shots,
                              shots_out.data_ptr(), ws_es.data_ptr(), ws_es.numel(), 0, sh)
        if pair:
            pair[1].record(stream)

    # cost table; phase tables, p rounds, readout + tile pass, finalize, two
    # scan launches, resolve (fused); else the evolve and sample launches
    launches_per_step = 1 + ((p + 3 + 3) if fused else (p + 3) + (6 if N >= 4096 else 1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        step(ev_pairs[i])
    stop.record(stream)
    torch.cuda.synchronize(dev)
    evolve_ms = [a.elapsed_time(b) for a, b in ev_pairs]
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed = start.elapsed_time(stop) / 1e3
    t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed = float(t.item())
    units = p * N * args.steps * world
    value = units / elapsed

    # ---- end-to-end through the public API with host buffers -------------
    h_g = torch.as_tensor(g_np).pin_memory()
    h_b = torch.as_tensor(b_np).pin_memory()
    h_shots = torch.empty(shots, dtype=torch.int64).pin_memory()
    h_out = torch.empty(3, dtype=torch.float64).pin_memory()

    def e2e_step():
        gam.copy_(h_g, non_blocking=True)
        bet.copy_(h_b, non_blocking=True)
        step()
        h_out.copy_(out, non_blocking=True)
        h_shots.copy_(shots_out, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_elapsed = time.perf_counter() - t0
    te = torch.tensor([e2e_elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = units / float(te.item())
    h2d = lits_c.nbytes + h_g.numel() * 8 + h_b.numel() * 8
    d2h = h_shots.numel() * 8 + h_out.numel() * 8

    # ---- roofline of the fused round (the evolve_sample call) -------------
    # algorithmic bytes: round 1 reads 1 B cost + writes 8 B; rounds 2..p read
    # 8 B + 1 B and write 8 B; the readout + tile pass reads 8 B + 1 B (fused
    # path; the materialising readout pass also writes 8 B). The sampler's scan
    # and shot passes move a few MB and are counted as time only.
    alg_bytes = N * (9 + 17 * (p - 1) + (9 if fused else 17 + 8))
    ev_s = statistics.median(evolve_ms) / 1e3
    achieved = alg_bytes / ev_s / 1e9
    peak, peak_kind = hbm_peak()
    traffic = profiled_traffic(n) if n == 28 else None

    if rank == 0:
        cpu = None
        if world == 1 and os.environ.get("GQAOA_BENCH_NO_CPU") != "1":
            try:
                osamp = OracleSample(wl)
                v, _ = osamp.step()
                cpu = {"value": v, "unit": UNIT, "cores": osamp.cores, "kind": "oracle",
                       "sample": osamp.desc, "cpu_model": cpu_model(),
                       "one_core_round_amp_rounds_per_s": osamp.one_core(),
                       "context_reduced_model_s": osamp.reduced_context()}
            except Exception as exc:  # keep the GPU line even if the host run fails
                cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                       "sample": f"failed: {exc!r}"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "m": m, "p": p, "shots": shots,
                       "parallelism": f"replicas x{world} (independent instances)",
                       "l2": f"inputs larger than L2 ({(8 << n) >> 20} MiB state, "
                             f"{(1 << n) >> 20} MiB cost table)"
                       if n >= 26 else "small case: L2-resident"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "alg_bytes_per_launch": 17 * N,
                         "kernel": "round_kernel (K2): mean over the p+1 streaming passes of "
                                   "the evolve_sample call (p rounds, the readout + sampler tile "
                                   "pass; the sampler's scans and shots included in the time)",
                         "peak_kind": peak_kind,
                         "evolve_sample_ms": statistics.median(evolve_ms)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "P0": float(out[0].item()),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_grad(args, wl):
    """Workload "grad": forward rounds with checkpoints + backward rounds for
    every instance, then one Adam step over all angles (gqaoa_grad_batched +
    gqaoa_adam_f64). Metric: forward amplitude-rounds per second, B * p * 2^n
    per step (the backward pass is extra work not counted)."""
    import torch

    from paper_2402_02585_gb300 import _capi as C
    from paper_2402_02585_gb300 import core, instances
    from paper_2402_02585_gb300.optim import AngleOptimizer

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    n, m, p, B = wl["n"], wl["m"], wl["p"], wl["batch"]
    N = 1 << n
    costs = torch.empty((B, N), dtype=torch.uint8, device="cuda")
    for i in range(B):
        lits = instances.random_3sat(n, m, wl["seed"] + 1_000_003 * rank + i)
        costs[i].copy_(core.build_cost(lits, n, with_hist=False)[0])
    opt = AngleOptimizer(costs, n, m, p)
    G = np.stack([instances.random_angles(p, wl["seed"] + i)[0] for i in range(B)])
    Bt = np.stack([instances.random_angles(p, wl["seed"] + i)[1] for i in range(B)])
    opt.reset(G, Bt)
    for _ in range(args.warmup):
        opt.step(wl["lr"])
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    start.record()
    for _ in range(args.steps):
        opt.step(wl["lr"])
    stop.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = start.elapsed_time(stop) / 1e3
    units = B * p * N * args.steps
    cluster = 10 <= n <= 16  # the library's cluster-resident adjoint (gqaoa.h)
    # algorithmic bytes per step (core.grad_hbm_bytes): on the cluster path
    # the cost table read once (1 B per amplitude) and every checkpoint
    # written forward and read backward (8 + 8 B per amplitude-round), the
    # state and lambda staying on chip; on the streaming passes the forward
    # 9 B (round 1) + 17 B (rounds 2..p) per amplitude, lambda init 17 B,
    # backward 25 B per amplitude-round
    alg = B * N * core.grad_hbm_bytes(n, p)
    if cluster:
        kernel = ("adjoint_cluster_kernel (one cluster per instance for all rounds, 16 B per "
                  "amplitude-round of checkpoints; bound by its per-round cluster reductions, "
                  "not by HBM; streaming_grad below: the streaming passes, 42 B per "
                  "amplitude-round, timed on the same angles)")
    else:
        kernel = "forward rounds + backward rounds (mean over the step)"
    achieved = alg * args.steps / el / 1e9
    peak, kind = hbm_peak()
    streaming = None
    if cluster:
        # the same gradient call by the streaming passes, for context
        code = C.GQAOA_OBJ_P0 | C.GQAOA_GRAD_STREAMING
        th = opt.theta
        for _ in range(2):
            core.grad_batched(costs, n, m, th[0], th[1], code, ws=opt.ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            core.grad_batched(costs, n, m, th[0], th[1], code, ws=opt.ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        s_alg = B * N * core.grad_hbm_bytes(n, p, streaming=True)
        streaming = {"ms_per_call": ms, "hbm_gbs": s_alg / (ms / 1e3) / 1e9,
                     "frac": s_alg / (ms / 1e3) / 1e9 / peak,
                     "note": "gradient call only (no Adam step), GQAOA_GRAD_STREAMING"}
    v = opt.evaluate().cpu().numpy()
    line = {"metric": METRIC, "value": units / el, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "n": n, "m": m, "p": p,
                                            "batch": B, "l2": "inputs larger than L2 "
                                            f"({(B * N * 8) >> 20} MiB states, "
                                            f"{(p * B * N * 8) >> 20} MiB checkpoints)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": kind,
                         "kernel": kernel},
            "adam_steps_per_s": args.steps / el, "mean_P_after": float(v.mean()),
            "streaming_grad": streaming,
            "cpu_baseline": cpu_grad_baseline(wl),
            "gpu_launches": (core.grad_launches(n, p) + 1) * args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def l2_rmw_peak(device) -> float:
    """Read-modify-write bandwidth of a 64 MiB L2-resident buffer, measured
    live (GB/s, read + write bytes): torch's in-place multiply, 100 launches
    replayed from a CUDA graph so no host launch gap sits between them."""
    import torch

    x = torch.ones(16 << 20, dtype=torch.float32, device=device)
    s = torch.cuda.Stream(device)
    s.wait_stream(torch.cuda.current_stream(device))
    with torch.cuda.stream(s):
        for _ in range(3):
            x.mul_(0.999999)
    torch.cuda.current_stream(device).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(100):
            x.mul_(0.999999)
    g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * x.numel() * 4 * 100 / (e0.elapsed_time(e1) / 1e3) / 1e9


# on-chip share of the state on the cluster-resident sweep path: 16 CTAs x
# 256 on-chip threads x (18 float4 in registers + 48 in shared memory) x 2
L2_PATH_ONCHIP_AMPS = 16 * 256 * (18 + 48) * 2


def run_sweep(args, wl):
    """Workload "sweep": all instances x all grid points through SweepPlan (the
    on-chip sweep for n <= 19, the cluster-resident sweep with L2-resident
    slots for n = 20; streaming chunks where the tuning table says so), the
    16-CTA-cluster launches and the others replayed as two CUDA graphs on two
    streams. Metric: amplitude-rounds per second, sum over items of p * 2^n."""
    import torch

    from paper_2402_02585_gb300 import core, instances
    from paper_2402_02585_gb300.sweep import SweepPlan, grid_angles

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    count = int(os.environ.get("GQAOA_SWEEP_INSTANCES", wl["count"]))
    shapes = instances.sweep_shapes(count, wl["seed"])
    per_n: dict[int, list] = {}
    mmax: dict[int, int] = {}
    for i, (n, m, _) in enumerate(shapes):
        if i % world != rank:
            continue
        lits = instances.random_3sat(n, m, wl["seed"] * 1_000_003 + i)
        per_n.setdefault(n, []).append(core.build_cost(lits, n, with_hist=False)[0])
        mmax[n] = max(mmax.get(n, 0), m)
    buckets = {n: (torch.stack(v), mmax[n]) for n, v in per_n.items()}
    G, B = grid_angles(wl["grid"])
    plan = SweepPlan(buckets, G, B, wl["p"], wl["rounds"])
    plan.capture()  # includes one eager run
    kinds = plan.kinds()

    def one_step(marks):
        for j, kind in enumerate(kinds):
            if kind in plan.graphs:
                plan.graphs[kind].replay()
            else:
                plan.run(kinds=(kind,))
            if marks is not None:
                marks[j + 1].record()

    for _ in range(max(0, args.warmup - 1)):
        plan.replay_concurrent()
    l2_peak = l2_rmw_peak(local) if "l2" in kinds else None
    # one sequential pass, each path alone on the GPU: the per-path rooflines
    torch.cuda.synchronize()
    seq = [torch.cuda.Event(enable_timing=True) for _ in range(len(kinds) + 1)]
    seq[0].record()
    one_step(seq)
    torch.cuda.synchronize()
    t_kind = {kind: seq[j].elapsed_time(seq[j + 1]) / 1e3 for j, kind in enumerate(kinds)}
    ar_kind = {kind: plan.amp_rounds_of(kind) for kind in kinds}
    t_seq = seq[0].elapsed_time(seq[-1]) / 1e3
    # the timed steps: the 16-CTA-cluster buckets and the others on two streams
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    ev[0].record()
    for i in range(args.steps):
        plan.replay_concurrent()
        ev[i + 1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = ev[0].elapsed_time(ev[-1]) / 1e3
    units = plan.amp_rounds() * args.steps
    peak, peak_kind = hbm_peak()
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    def bucket_list(kind):
        return ",".join(str(st[1]) for st in plan.steps if st[0] == kind)

    def share(kind):
        return f"{100 * t_kind[kind] / t_seq:.0f} % of a sequential pass"

    roof = {}
    if "onchip" in kinds:
        # issue ceiling from unit counts and clocks: 4 warp-instructions per clock
        # per SM x 32 lanes x SMs x max SM clock, over the 12 instructions of one
        # amplitude-round (phase lookup, complex multiply-add, sums, cost byte)
        alu_peak = 4 * 32 * sms * 2.07e9 / 12
        a = ar_kind["onchip"] / t_kind["onchip"]
        roof["onchip"] = {"bound": "alu", "achieved": a, "peak": alu_peak, "unit": "amp-rounds/s",
                          "frac": a / alu_peak, "kernel": f"sweep_kernel (n = {bucket_list('onchip')}"
                          f" buckets, {share('onchip')})",
                          "peak_derivation": "4 warp-instr/clk/SM x 32 x SMs x 2.07 GHz / 12 "
                                             "instructions per amplitude-round"}
    if "l2" in kinds:
        # 8 B read + 8 B write + 1 B cost per amplitude-round outside shared memory
        l2_bytes = sum(17.0 * st[3].shape[0] * plan.A * plan.p * max(0, (1 << st[1]) - L2_PATH_ONCHIP_AMPS)
                       for st in plan.steps if st[0] == "l2")   # one sequential pass
        a = l2_bytes / t_kind["l2"] / 1e9
        roof["l2"] = {"bound": "l2", "achieved": a, "peak": l2_peak, "unit": "GB/s",
                      "frac": a / l2_peak, "traffic": None,
                      "peak_kind": "measured live: in-place multiply of a 64 MiB tensor "
                                   "(L2-resident), 100 launches from a CUDA graph",
                      "kernel": f"sweep_l2_kernel (n = {bucket_list('l2')} buckets, {share('l2')})",
                      "alg_bytes": "17 B per amplitude-round outside registers and shared "
                                   f"memory ({L2_PATH_ONCHIP_AMPS} amplitudes per item stay on chip)",
                      "amp_rounds_per_s": ar_kind["l2"] / t_kind["l2"]}
    if "stream" in kinds:
        # 8 B read + 8 B write per amplitude-round (the shared cost table stays in
        # L2 across a chunk of angle points)
        a = 16 * ar_kind["stream"] / t_kind["stream"] / 1e9
        roof["stream"] = {"bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s",
                          "frac": a / peak, "traffic": None, "peak_kind": peak_kind,
                          "kernel": f"streaming round_kernel (n = {bucket_list('stream')} buckets, "
                                    f"{share('stream')})", "alg_bytes_per_amp_round": 16}
    dominant = max(kinds, key=lambda k: t_kind[k])
    launches = 0
    for kind, n, m, c, o, x in plan.steps:
        if kind == "stream":
            S = x[0]
            launches += c.shape[0] * -(-plan.A // S) * (plan.p + 3)
        else:
            launches += 2  # phase tables + the persistent sweep kernel
    best = {n: float(o[..., -1].max().item()) for n, o in plan.out.items()}
    if rank == 0:
        line = {
            "metric": METRIC, "value": units / el, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f32/f64 sums", "data": "synthetic",
            "config": {"workload": wl["desc"], "instances": count,
                       "amp_rounds_per_step": plan.amp_rounds(),
                       "buckets": {n: int(c.shape[0]) for n, (c, _) in buckets.items()},
                       "paths": {str(st[1]): st[0] for st in plan.steps},
                       "schedule": "16-CTA-cluster buckets and the others on two streams; "
                                   "per-path rooflines from one sequential pass "
                                   f"({t_seq:.1f} s)"},
            "roofline": roof[dominant]}
        for kind in kinds:
            if kind != dominant:
                line[f"roofline_{kind}"] = roof[kind]
        line.update({"cpu_baseline": cpu_sweep_baseline(wl) if world == 1 else None,
                     "gpu_launches": launches * args.steps,
                     "per_n_best_P_at_p64": best, "clocks": clk})
        print(json.dumps(line), flush=True)
    return 0


def grid_instance(wl):
    """The grid workload's instance: the first satisfiable seed from
    wl["seed"] on, its histogram by the oracle's cost table (host, int64)."""
    from oracle import statevector as sv
    from paper_2402_02585_gb300 import instances
    seed = wl["seed"]
    while True:
        lits = instances.random_3sat(wl["n"], wl["m"], seed)
        _, hist = sv.cost_table(lits, wl["n"])
        if hist[0] > 0:
            return seed, lits, np.asarray(hist, dtype=np.int64)
        seed += 1


def cpu_grid_baseline(wl, hist, G, B, points: int = 20000):
    """The oracle's cost-class model (numpy FP64, one core) on a bounded
    sample of the grid: `points` angle pairs spread over it, all p rounds
    (20000 points, about 10 s)."""
    from oracle import reduced
    idx = np.linspace(0, len(G) - 1, points).astype(np.int64)
    t0 = time.perf_counter()
    for a in idx:
        reduced.readouts_trace(hist, [G[a]] * wl["p"], [B[a]] * wl["p"])
    t = time.perf_counter() - t0
    return {"value": points * wl["p"] / t, "unit": "item-rounds/s", "cores": 1, "kind": "oracle",
            "sample": f"{points} of the {len(G)} grid angle pairs (evenly spaced), p = {wl['p']} "
                      f"rounds each, oracle.reduced.readouts_trace ({t:.1f} s)"}


def run_grid(args, wl):
    """Workload "grid": gqaoa_reduced_sweep of one instance over the protocol's
    pi/180 grid, the protocol's grid call. Metric: item-rounds per second
    (angle pairs x rounds). Each timed call follows an L2 flush (the call's
    buffers, 117 MB at this size, would otherwise stay in L2); the e2e figure
    goes through core.reduced_sweep from host inputs (histogram and angles
    copied in, the per-round argmin copied out)."""
    import torch

    from paper_2402_02585_gb300 import _capi as C
    from paper_2402_02585_gb300 import core, instances

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed, lits, hist = grid_instance(wl)
    nz = np.nonzero(hist)[0]
    cut = hist[:nz[-1] + 1]
    classes = int(nz[-1] - nz[0] + 1)
    n, p = wl["n"], wl["p"]
    G, B = instances.protocol_grid()
    A = len(G)
    hd = torch.as_tensor(cut, device=dev).reshape(1, -1)
    Gd = torch.as_tensor(G, dtype=torch.float64, device=dev)
    Bd = torch.as_tensor(B, dtype=torch.float64, device=dev)
    out = torch.empty((1, p, 3, A), dtype=torch.float32, device=dev)
    best = torch.empty((1, p), dtype=torch.int32, device=dev)
    ws = core.workspace(C.gqaoa_reduced_sweep_workspace_size(hd.shape[1], 1, A, p), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream

    def call():
        C.gqaoa_reduced_sweep(hd.data_ptr(), hd.shape[1], n, 1, Gd.data_ptr(), Bd.data_ptr(), A, p,
                              out.data_ptr(), best.data_ptr(), ws.data_ptr(), ws.numel(), st)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record()
        call()
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    el = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3
    # end to end through the Python API: host histogram and angles in, the
    # per-round argmin out
    hh = torch.as_tensor(cut).reshape(1, -1).pin_memory()
    Gh = torch.as_tensor(G, dtype=torch.float64).pin_memory()
    Bh = torch.as_tensor(B, dtype=torch.float64).pin_memory()
    bh = torch.empty((1, p), dtype=torch.int32).pin_memory()
    for _ in range(args.warmup):
        core.reduced_sweep(hh.to(dev, non_blocking=True), n, Gh.to(dev, non_blocking=True),
                           Bh.to(dev, non_blocking=True), p, ws=ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, bd = core.reduced_sweep(hh.to(dev, non_blocking=True), n, Gh.to(dev, non_blocking=True),
                                   Bh.to(dev, non_blocking=True), p, ws=ws)
        bh.copy_(bd)
    torch.cuda.synchronize()
    e2e = time.perf_counter() - t0
    units = A * p
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # 11 FP32 instructions per class and round (complex phase multiply 4, the
    # S sum 2, mixer add 2, the <H_P> term 3) over the classes from the lowest
    # to the highest non-empty one, at 4 warp-instructions (128 lanes) per
    # clock per SM
    alu_peak = 4 * sms * 2.07e9 / (11 * classes / 32)
    rate = units * args.steps / el
    line = {"metric": "cost-class item-rounds/s", "value": rate, "unit": "item-rounds/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 (class amplitudes), f32 sums and readouts",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "m": wl["m"], "instance_seed": seed,
                       "angle_pairs": A, "p": p, "classes": classes,
                       "histogram_stride": int(hd.shape[1]),
                       "l2": "flushed (256 MiB write) before every timed call"},
            "roofline": {"bound": "alu", "achieved": rate, "peak": alu_peak,
                         "unit": "item-rounds/s", "frac": rate / alu_peak, "traffic": None,
                         "kernel": "the whole call (phase tables, weights, reduced_sweep_kernel, "
                                   "argmin reduce); the kernel's own share is in the profile",
                         "peak_derivation": "4 warp-instr/clk/SM x SMs x 2.07 GHz / (11 FP32 "
                                            f"instructions x {classes} classes / 32 lanes) per "
                                            "item-round"},
            "e2e": {"value": units * args.steps / e2e, "unit": "item-rounds/s",
                    "h2d_bytes_per_step": int(cut.nbytes + 16 * A),
                    "d2h_bytes_per_step": int(4 * p)},
            "cpu_baseline": (cpu_grid_baseline(wl, cut, G, B)
                             if os.environ.get("GQAOA_BENCH_NO_CPU") != "1" else None),
            "gpu_launches": 4 * args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_grid_reference(args, wl):
    """The grid workload's oracle arm: the FP64 cost-class model on a bounded
    sample of the grid per step, on the host."""
    from paper_2402_02585_gb300 import instances
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    seed, _, hist = grid_instance(wl)
    cut = hist[:np.nonzero(hist)[0][-1] + 1]
    G, B = instances.protocol_grid()
    per = []
    for i in range(args.warmup + args.steps):
        r = cpu_grid_baseline(wl, cut, G, B, points=2000)
        if i >= args.warmup:
            per.append(r["value"])
    value = float(np.mean(per))
    print(json.dumps({
        "impl": "reference", "metric": "cost-class item-rounds/s", "value": value,
        "unit": "item-rounds/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 2000 * wl["p"] / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "instance_seed": seed, "p": wl["p"]},
        "cpu_baseline": {"value": value, "unit": "item-rounds/s", "cores": 1, "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": value, "unit": "item-rounds/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)
    return 0


def run_protocol(args, wl):
    """Workloads "protocol" and "protocol_maxsat": the paper's angle protocol
    for every instance (target P, or D for unsatisfiable instances). Metric:
    instances per second. Also reported: the fewest rounds per instance
    against the target's random-guess probability (h[0] / 2^n, or h[c*] / 2^n)
    and the fitted exponent of p_min ~ (1/P)^x (Section III's evidence for a
    quadratic speedup: x ~ 0.5), and the cost-class grid kernel's rate."""
    import torch

    from paper_2402_02585_gb300 import _capi as C
    from paper_2402_02585_gb300 import core, instances
    from paper_2402_02585_gb300.protocol import Protocol, min_rounds_many, satisfiable_shapes

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    target = wl.get("target", "P")
    shapes = satisfiable_shapes(wl["count"], wl["seed"] + rank, wl["n_values"], wl["d_lo"],
                                wl["d_hi"], satisfiable=target == "P")
    prots = [(n, m, hist, Protocol(cost, hist, n, m)) for n, m, _, _, cost, hist in shapes]

    workers = int(os.environ.get("GQAOA_PROTOCOL_WORKERS", str(wl.get("workers", 8))))
    window = int(os.environ.get("GQAOA_PROTOCOL_WINDOW", str(wl.get("window", 8))))

    retry = wl.get("retry_p_max", 4 * wl["p_max"])

    def one_pass(count=None):
        # several instances in flight (host threads, one CUDA stream each)
        sel = prots if count is None else prots[:count]
        return min_rounds_many([pr for _, _, _, pr in sel], workers=workers, retry_p_max=retry,
                               S=wl["S"], p_max=wl["p_max"], target=target, window=window)

    for _ in range(args.warmup):
        one_pass(wl.get("warm_count"))
    # the grid call alone as the protocol makes it (phase tables, cost-class
    # kernel with the per-round argmin), on the full pi/180 grid of the first
    # instance, buffers resident
    G, B = instances.protocol_grid()
    n0, _, h0, prot0 = prots[0]
    dev = torch.device("cuda", local)
    h0d = prot0.grid_hist
    Gd = torch.as_tensor(G, dtype=torch.float64, device=dev)
    Bd = torch.as_tensor(B, dtype=torch.float64, device=dev)
    grid_out = torch.empty((1, wl["p_max"], 3, len(G)), dtype=torch.float32, device=dev)
    grid_best = torch.empty((1, wl["p_max"]), dtype=torch.int32, device=dev)
    grid_ws = core.workspace(
        C.gqaoa_reduced_sweep_workspace_size(h0d.shape[1], 1, len(G), wl["p_max"]), dev)
    st = torch.cuda.current_stream().cuda_stream

    def grid_call():
        C.gqaoa_reduced_sweep(h0d.data_ptr(), h0d.shape[1], n0, 1, Gd.data_ptr(), Bd.data_ptr(),
                              len(G), wl["p_max"], grid_out.data_ptr(), grid_best.data_ptr(),
                              grid_ws.data_ptr(), grid_ws.numel(), st)

    grid_call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        grid_call()
    e1.record()
    torch.cuda.synchronize()
    t_grid = e0.elapsed_time(e1) / 5 / 1e3
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        results = one_pass()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    if world > 1:
        te = torch.tensor([el], dtype=torch.float64, device="cuda")
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        el = float(te.item())
    count = len(prots) * world * args.steps
    # the random-guess probability of the target: h[c*] / 2^n (c* = 0 when satisfiable)
    pr = np.array([int(h[prot.min_class].item()) / (1 << n) for n, m, h, prot in prots])
    pm = np.array([r.p if r.p is not None else np.nan for r in results], dtype=np.float64)
    ok = np.isfinite(pm)
    slope = float(np.polyfit(np.log(1 / pr[ok]), np.log(pm[ok]), 1)[0]) if ok.sum() > 2 else None
    big = ok & (pr < 1e-3)  # the large-1/P regime of Section III's asymptotic claim
    slope_big = (float(np.polyfit(np.log(1 / pr[big]), np.log(pm[big]), 1)[0])
                 if big.sum() > 2 else None)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # grid call: the cost-class arithmetic is 11 FP32 instructions per class
    # and round (complex phase multiply 4, the S sum 2, mixer add 2, the
    # <H_P> term 3) over the classes from the lowest to the highest non-empty
    # one; the ceiling issues them at 4 warp-instructions (128 lanes) per
    # clock per SM, so an item-round of that many classes costs 11 classes / 32
    nz = torch.nonzero(h0).flatten()
    classes = int(nz[-1]) - int(nz[0]) + 1
    alu_peak = 4 * sms * 2.07e9 / (11 * classes / 32)
    grid_rate = len(G) * wl["p_max"] / t_grid
    if rank == 0:
        print(json.dumps({
            "metric": "protocol instances/s", "value": count / el, "unit": "instances/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 (grid, statevector) + f64 optimiser",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "instances": len(prots), "S": wl["S"],
                       "p_max": wl["p_max"], "retry_p_max": retry, "host_threads": workers,
                       "depth_window": window,
                       "warmup_pass": "all instances" if wl.get("warm_count") is None
                       else f"the first {wl['warm_count']} instances"},
            "roofline": {"bound": "alu", "achieved": grid_rate, "peak": alu_peak,
                         "unit": "item-rounds/s", "frac": grid_rate / alu_peak,
                         "kernel": f"gqaoa_reduced_sweep (phase tables, reduced_sweep_kernel "
                                   f"with the per-round argmin): pi/180 grid ({len(G)} angle "
                                   f"pairs) x p = {wl['p_max']}, n = {n0}, {classes} classes "
                                   f"(histogram stride {h0d.shape[1]}), {t_grid * 1e3:.3f} ms",
                         "peak_derivation": "4 warp-instr/clk/SM x SMs x 2.07 GHz / (11 FP32 "
                                            f"instructions x {classes} classes / 32 lanes) per "
                                            "item-round"},
            "p_min": [None if r.p is None else int(r.p) for r in results],
            "n": [int(n) for n, _, _, _ in prots],
            "seconds_per_instance": [round(float(r.seconds), 4) for r in results],
            "evaluations_per_instance": [int(r.evaluations) for r in results],
            "target": target,
            "random_guess_probability": [float(x) for x in pr],
            "fitted_exponent": slope,
            "fitted_exponent_one_over_P_above_1e3": slope_big,
            "median_p_sqrt_P": float(np.median(pm[ok] * np.sqrt(pr[ok]))) if ok.any() else None,
            "gradient_evaluations_per_instance": float(np.mean([r.evaluations for r in results])),
            "cpu_baseline": cpu_protocol_baseline(wl, shapes) if world == 1 else None,
            "gpu_launches": int(sum(r.launches for r in results)) * args.steps, "clocks": clk}),
              flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_fairness(args, wl):
    """Workload "fairness": Section IV's metrics. Metric: shots per second
    through sampling and both metrics (whole step)."""
    import scipy.stats
    import torch

    from paper_2402_02585_gb300 import core
    from paper_2402_02585_gb300.protocol import Protocol, satisfiable_shapes

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    n, m, iseed, lits, cost, hist = satisfiable_shapes(1, wl["seed"] + rank, [wl["n"]], wl["d_lo"],
                                                       wl["d_hi"])[0]
    res = Protocol(cost, hist, n, m).min_rounds(S=0.5, p_max=64)
    state, out, _ = core.evolve(cost, n, m, res.gammas, res.betas)
    M = int(hist[0].item())
    runs, per_run = wl["runs"], wl["shots_per_run"]
    shots_n = runs * per_run
    crit = float(scipy.stats.chi2.ppf(1 - wl["alpha"], max(M - 1, 1)))
    shots = torch.empty(shots_n, dtype=torch.int64, device="cuda")
    ws_s = core.workspace(C_size_sample(n, shots_n), "cuda")
    ws_f = core.workspace(C_size_fair(n, runs, M), "cuda")

    def step(i, ev=None):
        core.sample(state, n, 1000 + i, shots_n, ws=ws_s, out=shots)
        if ev is not None:
            ev.record()
        return core.fairness(shots, runs, cost, n, 0, M, crit, 5 * M, ws=ws_f)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    for i in range(args.steps):
        evs[i][0].record()
        ta, tr = step(args.warmup + i, evs[i][1])
        evs[i][2].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_samp = sum(a.elapsed_time(b) for a, b, c in evs) / 1e3
    t_fair = sum(b.elapsed_time(c) for a, b, c in evs) / 1e3
    el = evs[0][0].elapsed_time(evs[-1][2]) / 1e3
    ta = ta.cpu().numpy()
    tr = tr.cpu().numpy()
    done = ta[ta > 0].astype(np.float64)
    # the sampler's ceiling is its issue rate: per shot Philox4x32-10, the tile
    # search, the chunk search and the search of the chunk's running sums
    # execute ~307 thread-instructions (ncu instruction count of this path)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = 4 * 32 * sms * 2.07e9 / 307
    samp_rate = shots_n * args.steps / t_samp
    if rank == 0:
        print(json.dumps({
            "metric": "fair-sampling shots/s", "value": shots_n * args.steps / el, "unit": "shots/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 state, f64 CDF, int64 metrics", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "m": m, "solutions": M, "p": res.p,
                       "P": float(out[0].item()), "runs": runs, "shots_per_run": per_run},
            "roofline": {"bound": "alu", "achieved": samp_rate, "peak": alu_peak,
                         "unit": "shots/s", "frac": samp_rate / alu_peak,
                         "kernel": f"gqaoa_sample, resident-tile path ({100 * t_samp / el:.0f} % "
                                   "of the step)",
                         "peak_derivation": "4 warp-instr/clk/SM x 32 x SMs x 2.07 GHz / 307 "
                                            "instructions per shot (measured count)"},
            "metrics_kernel_shots_per_s": shots_n * args.steps / t_fair,
            "shots_to_all_solutions": {"mean": float(done.mean()),
                                       "ci95": float(1.96 * done.std() / math.sqrt(done.size)),
                                       "completed_runs": int(done.size)},
            "shots_to_reject_fairness": {"median": float(np.median(tr[tr > 0]))
                                         if (tr > 0).any() else None,
                                         "rejected_runs": int((tr > 0).sum())},
            "cpu_baseline": cpu_fairness_baseline(wl, n, lits, res, runs) if world == 1 else None,
            # sampler: tile sums, tile scan, shot tiles, count scan, scatter, resolve;
            # metrics: labels, runs
            "gpu_launches": 8 * args.steps, "clocks": clk}), flush=True)
    return 0


def run_study(args, wl):
    """Workload "study": the learned-initialisation study of the proposer
    (study.run). Value: the median wall time for the optimizer started from the
    proposal to reach 95 % of the plain optimizer's final P(C=0) (Adam from
    angles uniform in [0, pi), 200 steps), fallbacks charged both runs; the
    plain optimizer's own median, the grid-protocol baseline, hit and
    fallback rates and each phase's time beside it."""
    import torch

    from paper_2402_02585_gb300 import study

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    quiet = lambda *a, **k: None  # noqa: E731
    for i in range(args.warmup):
        study.run(train_count=max(1, wl["train"] // 100), train_n=wl["train_n"],
                  test_count=max(1, wl["test"] // 100), test_n=wl["test_n"], d_lo=wl["d_lo"],
                  d_hi=wl["d_hi"], p=wl["p"], epochs=5, seed=wl["seed"] + 100 + i, log=quiet)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    results = []
    for i in range(args.steps):
        results.append(study.run(train_count=wl["train"], train_n=wl["train_n"],
                                 test_count=wl["test"], test_n=wl["test_n"], d_lo=wl["d_lo"],
                                 d_hi=wl["d_hi"], p=wl["p"], seed=wl["seed"] + i, log=quiet))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    r = results[-1]
    # the dominant kernels are the batched adjoint gradients of the label
    # phase: per Adam step and instance the algorithmic bytes of the path the
    # library takes for its n (core.grad_hbm_bytes: 1 + 16 p per amplitude
    # with the state on chip, n <= 16; the streaming passes' 9 + 17 (p - 1)
    # + 17 + 25 p above)
    p = wl["p"]
    label_bytes = r["label_hbm_bytes"]
    achieved = label_bytes / r["timings"]["labels_s"] / 1e9
    peak, peak_kind = hbm_peak()
    if rank == 0:
        print(json.dumps({
            "metric": "learned-init angle optimisation: median wall-s to 95 % of plain P(C=0)",
            "value": r["median_wall_proposer"], "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 state + f64 angles (optimizer), f32 MLP", "data": "synthetic",
            "config": {"workload": wl["desc"], "train_instances": r["train_instances"],
                       "test_instances": r["test_instances"], "p": p,
                       "warmup_step": "the same study at 1/100 of the instance counts"},
            "plain": {"median_wall_s": r["median_wall_plain"],
                      "median_steps": r["median_steps_plain"], "mean_P": r["mean_P_plain"]},
            "proposer": {"median_wall_s": r["median_wall_proposer"],
                         "median_steps": r["median_steps_proposer"], "hit_rate": r["hit_rate"],
                         "fallback_rate": r["fallback_rate"],
                         "mean_P_final": r["mean_P_proposer_final"],
                         "inference_s_total": r["proposer_inference_s"]},
            "grid_protocol_baseline": r["grid"],
            "timings_s": r["timings"], "loss": [r["loss_first"], r["loss_last"]],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "label phase: batched adjoint gradient + Adam (algorithmic "
                                   "bytes of each n's gradient path, cluster-resident for "
                                   "n <= 16 and streaming above, over the phase's wall time, "
                                   "host work included)"},
            "cpu_baseline": None,
            "gpu_launches": r["gpu_launches"], "clocks": clk}), flush=True)
    return 0


def C_size_sample(n, shots):
    from paper_2402_02585_gb300 import _capi as C
    return C.gqaoa_sample_workspace_size(n, shots)


def C_size_fair(n, runs, M):
    from paper_2402_02585_gb300 import _capi as C
    return C.gqaoa_fairness_workspace_size(n, runs, M)


def cpu_fairness_baseline(wl, n, lits, res, runs):
    """The oracle on a bounded sample: statevector, its sampler and both
    metrics for 200 runs of the stream."""
    import scipy.stats

    from oracle import fairness as ofair
    from oracle import statevector as sv
    if os.environ.get("GQAOA_BENCH_NO_CPU") == "1":
        return None
    cost, hist = sv.cost_table(lits, n)
    M = int(hist[0])
    k = 200
    t0 = time.perf_counter()
    psi = sv.evolve(cost, n, res.gammas, res.betas)
    shots = sv.sample(psi, n, 1000, k * wl["shots_per_run"])
    crit = float(scipy.stats.chi2.ppf(1 - wl["alpha"], max(M - 1, 1)))
    ofair.run_metrics(shots, cost, 0, k, crit, 5 * M)
    t = time.perf_counter() - t0
    return {"value": k * wl["shots_per_run"] / t, "unit": "shots/s", "cores": _oracle_threads(),
            "kind": "oracle", "sample": f"{k} runs of {wl['shots_per_run']} shots: statevector, "
                                        "sampler and both metrics (plain Python loop)"}


def cpu_protocol_baseline(wl, shapes):
    """The protocol oracle (FP64 cost-class model for the grid and the
    gradients) on the first two instances, on the host cores."""
    from oracle import protocol as oprot
    from paper_2402_02585_gb300 import instances
    if os.environ.get("GQAOA_BENCH_NO_CPU") == "1":
        return None
    from paper_2402_02585_gb300.protocol import grid_for
    t0 = time.perf_counter()
    for n, m, _, _, _, hist in shapes[:2]:
        G, B = grid_for(n)
        oprot.min_rounds(hist.cpu().numpy(), G, B, S=wl["S"], p_max=wl["p_max"],
                         target=wl.get("target", "P"))
    t = time.perf_counter() - t0
    return {"value": 2 / t, "unit": "instances/s", "cores": 1, "kind": "oracle",
            "sample": "the first two instances, full protocol up to p_max (numpy/scipy, FP64 "
                      "cost-class model for grid, refinement and probability)"}


def cpu_sweep_baseline(wl):
    """The FP64 statevector oracle on a bounded sample of the sweep: one
    (instance, grid point) per n in 12..20 for all p rounds with the P trace."""
    from oracle import statevector as sv
    from paper_2402_02585_gb300 import instances
    if os.environ.get("GQAOA_BENCH_NO_CPU") == "1":
        return None
    done = 0
    t = 0.0
    for n in range(12, 21):
        m = instances.clause_count(n, 4.2)
        cost, _ = sv.cost_table(instances.random_3sat(n, m, n), n)
        t0 = time.perf_counter()
        sv.evolve(cost, n, [0.4] * wl["p"], [2.0] * wl["p"], trace=True)
        t += time.perf_counter() - t0
        done += wl["p"] * (1 << n)
    return {"value": done / t, "unit": UNIT, "cores": _oracle_threads(), "kind": "oracle",
            "sample": f"one single-angle-pair item per n = 12..20 (m = round(4.2 n)), p = {wl['p']} "
                      "rounds with the P(C=0) trace, statevector oracle; cost tables untimed"}


def _oracle_threads():
    from oracle import statevector as sv
    return sv.num_threads()


def cpu_grad_baseline(wl):
    """The oracle's gradient on one instance of the workload: central finite
    differences (h = 1e-4) of the statevector oracle, 4p evolutions of p rounds.
    Value in the same unit as the GPU line: p * 2^n amplitude-rounds per gradient."""
    from oracle import statevector as sv
    from paper_2402_02585_gb300 import instances
    if os.environ.get("GQAOA_BENCH_NO_CPU") == "1":
        return None
    n, m, p = wl["n"], wl["m"], wl["p"]
    cost, _ = sv.cost_table(instances.random_3sat(n, m, wl["seed"]), n)
    g, b = instances.random_angles(p, wl["seed"])
    t0 = time.perf_counter()
    for arr in (g, b):
        for k in range(p):
            for d in (1e-4, -2e-4):
                arr[k] += d
                sv.readout(sv.evolve(cost, n, g, b), cost, n)
            arr[k] += 1e-4
    t = time.perf_counter() - t0
    return {"value": p * (1 << n) / t, "unit": UNIT, "cores": _oracle_threads(), "kind": "oracle",
            "sample": f"one instance n={n} m={m} p={p}: central-difference gradient of P(C=0) "
                      f"by the statevector oracle ({4 * p} evolutions, {t:.1f} s)"}


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        if wl.get("kind") == "grid":
            return run_grid_reference(args, wl)
        if wl.get("kind") is not None:
            print(json.dumps({"impl": "reference", "unavailable": "this workload has no "
                              "bounded oracle arm of its own (its GPU line carries the oracle's "
                              "rate as cpu_baseline); run the default workload"}))
            return 0
        return run_reference(args, wl)
    if wl.get("kind") == "grid":
        return run_grid(args, wl)
    if wl.get("kind") == "grad":
        return run_grad(args, wl)
    if wl.get("kind") == "protocol":
        return run_protocol(args, wl)
    if wl.get("kind") == "fairness":
        return run_fairness(args, wl)
    if wl.get("kind") == "sweep":
        return run_sweep(args, wl)
    if wl.get("kind") == "study":
        return run_study(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
