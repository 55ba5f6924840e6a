"""The paper's angle protocol on the GPU (Appendix C, "Optimization"; Section III).

For one instance and a target probability S:

  1. <H_P> (Eq. 4) of single-angle-pair G-QAOA on the pi/180 grid of
     (gamma, beta) (n <= 20; 4000 sampled angle pairs above) at every depth
     k <= p_max at once, from one cost-class evolution per angle pair
     (gqaoa_reduced_sweep, Appendix C's own simulation method), with the
     grid point of lowest <H_P> per depth from the same call;
  2. from that seed, L-BFGS-B on <H_P> with 1e-6 relative change as the
     stopping rule, the gradient from the statevector adjoint kernels
     (gqaoa_grad, the per-round gradients summed for the single angle pair;
     all 2k angles for G-QAOA with per-round angles);
  3. the solution probability P of the refined state on the statevector
     (gqaoa_evolve); the answer is the fewest rounds with P >= S.

For an unsatisfiable instance (Max-SAT, Fig. 1(b)) the target is D, the
probability of the lowest non-empty cost class (the assignments leaving the
fewest clauses unsatisfied), read the same way with GQAOA_READOUT_CLASS.

Every depth k = 1, 2, ... is refined in turn, as Appendix C optimises each
instance at each depth: L-BFGS-B starts from that depth's grid seed over the
single angle pair, or, for G-QAOA with per-round angles, from the same seed
over all 2k angles. The cost-class and statevector evaluations agree to
complex64 precision (tested), so the grid ranks candidates and the
statevector decides.
"""

from __future__ import annotations

import contextlib
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import scipy.optimize
import torch

from . import _capi as C
from . import core, instances


@dataclass
class MinRounds:
    p: int | None                 # fewest rounds reaching S (None: not within p_max)
    gammas: np.ndarray | None     # refined angles at p
    betas: np.ndarray | None
    prob: float | None            # P (or D) on the statevector at p
    energy: float | None          # <H_P> at the refined angles
    grid_prob: np.ndarray = field(default_factory=lambda: np.zeros(0))  # per depth, at the seed
    evaluations: int = 0          # statevector gradient evaluations
    launches: int = 0             # kernels launched by the library for this search
    seconds: float = 0.0


def grid_for(n: int, seed: int = 0):
    """The protocol's angle set: the pi/180 grid for n <= 20, 4000 sampled
    angle pairs above."""
    if n <= 20:
        return instances.protocol_grid()
    return instances.protocol_random_angles(4000, seed)


class _CaptureGate:
    """Protocol threads issue CUDA work side by side, but a CUDA graph is
    captured with no other protocol thread inside a CUDA call: even in
    thread-local capture mode, PyTorch's allocator and copies on other
    threads meet the open capture (an invalidated capture, failed copies).
    Work sections run concurrently; a capture waits for the running ones to
    leave and holds new ones back until it is done. Captures are rare (one
    per instance and depth), so the waits are short."""

    def __init__(self):
        self._cv = threading.Condition()
        self._active = 0
        self._capturing = False

    @contextlib.contextmanager
    def work(self):
        with self._cv:
            while self._capturing:
                self._cv.wait()
            self._active += 1
        try:
            yield
        finally:
            with self._cv:
                self._active -= 1
                if self._active == 0:
                    self._cv.notify_all()

    @contextlib.contextmanager
    def capture(self):
        with self._cv:
            while self._capturing:
                self._cv.wait()
            self._capturing = True
            while self._active > 0:
                self._cv.wait()
        try:
            yield
        finally:
            with self._cv:
                self._capturing = False
                self._cv.notify_all()


_GATE = _CaptureGate()


class _EnergyGrad:
    """<H_P> and its adjoint gradient at a fixed depth p with resident
    buffers: the angles go to the device in one copy from pinned host memory
    and the value and both gradients come back in one. An L-BFGS-B search
    makes hundreds of these small calls and each is 2p + 3 kernel launches
    on the streaming path, so after one direct call the library call is
    captured once into a CUDA graph and every further evaluation is one copy
    up, one graph launch and one copy down (the same kernels in the same
    order, so the same results)."""

    def __init__(self, prot: "Protocol", p: int):
        dev = prot.cost.device
        self.p = p
        self.d_ang = torch.empty(2 * p, dtype=torch.float64, device=dev)      # [gammas | betas]
        self.d_out = torch.empty(1 + 2 * p, dtype=torch.float64, device=dev)  # [value | dg | db]
        self.h_ang = torch.empty(2 * p, dtype=torch.float64, pin_memory=True)
        self.h_out = torch.empty(1 + 2 * p, dtype=torch.float64, pin_memory=True)
        self.a_ang = self.h_ang.numpy()
        self.a_out = self.h_out.numpy()
        self.ws = core.workspace(C.gqaoa_grad_workspace_size(prot.n, p), dev)
        ang, out = self.d_ang.data_ptr(), self.d_out.data_ptr()
        self.args = (prot.cost.data_ptr(), prot.n, prot.m, ang, ang + 8 * p, p,
                     core.objective_code("energy"), out, out + 8, out + 8 + 8 * p,
                     self.ws.data_ptr(), self.ws.numel())
        self.graph = None

    def _capture(self, stream):
        # Only the library call is captured (the two small pinned-memory
        # copies stay outside: PyTorch's pinned-memory allocator records and
        # later queries an event per copy, which must not land in a capture).
        # The capture runs on a side stream in thread-local mode, with
        # capture_begin / capture_end called directly, because the
        # torch.cuda.graph context synchronises the whole device on entry;
        # protocol searches on other host threads keep running meanwhile.
        with _GATE.capture():
            side = torch.cuda.Stream(stream.device)
            side.wait_stream(stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                g.capture_begin(capture_error_mode="thread_local")
                try:
                    C.gqaoa_grad(*self.args, side.cuda_stream)
                finally:
                    g.capture_end()
            stream.wait_stream(side)
            side.synchronize()
        self.graph = g

    def __call__(self, gammas, betas):
        p = self.p
        self.a_ang[:p] = gammas
        self.a_ang[p:] = betas
        with _GATE.work():
            st = torch.cuda.current_stream()
            self.d_ang.copy_(self.h_ang, non_blocking=True)
            if self.graph is not None:
                self.graph.replay()
            else:
                # the first call also sets the library's per-device caches up
                C.gqaoa_grad(*self.args, st.cuda_stream)
            self.h_out.copy_(self.d_out, non_blocking=True)
            st.synchronize()  # also frees the pinned buffers for the next call
        if self.graph is None:
            self._capture(st)
        return float(self.a_out[0]), self.a_out[1:1 + p].copy(), self.a_out[1 + p:].copy()


class Protocol:
    """The protocol for one instance: cost [2^n] uint8 and hist [m + 1] int64
    on the device (core.build_cost). An instance keeps per-depth device and
    pinned host buffers, so it is used by one thread at a time (different
    instances may run on different threads, as in min_rounds_many)."""

    def __init__(self, cost: torch.Tensor, hist: torch.Tensor, n: int, m: int):
        core._require_cuda(cost, hist)
        self.cost, self.hist, self.n, self.m = cost, hist, n, m
        self._ws = {}
        self._grad_calls = {}
        self.evaluations = 0
        self.launches = 0
        self._small = (1 << n) < 4096  # one CTA per state: phase tables + one or two kernels
        h = hist.cpu().numpy()
        self.min_class = int(np.nonzero(h)[0][0])  # 0 when satisfiable

    def _evolve_workspace(self, p: int) -> torch.Tensor:
        if p not in self._ws:
            self._ws[p] = core.workspace(C.gqaoa_evolve_workspace_size(self.n, p), self.cost.device)
        return self._ws[p]

    def energy_and_grad(self, gammas, betas):
        p = len(gammas)
        call = self._grad_calls.get(p)
        if call is None:
            with _GATE.work():
                call = self._grad_calls[p] = _EnergyGrad(self, p)
        self.evaluations += 1
        self.launches += 3 if self._small else 2 * p + 3
        return call(gammas, betas)

    def refine(self, gammas0, betas0, single: bool):
        """L-BFGS-B on <H_P> (relative change 1e-6). Returns (gammas, betas,
        <H_P>, evaluations)."""
        g0 = np.asarray(gammas0, np.float64)
        b0 = np.asarray(betas0, np.float64)
        p = g0.shape[0]
        if single:
            def fun(x):
                e, dg, db = self.energy_and_grad(np.full(p, x[0]), np.full(p, x[1]))
                return e, np.array([dg.sum(), db.sum()])
            x0 = np.array([g0[0], b0[0]])
        else:
            def fun(x):
                e, dg, db = self.energy_and_grad(x[:p], x[p:])
                return e, np.concatenate([dg, db])
            x0 = np.concatenate([g0, b0])
        r = scipy.optimize.minimize(fun, x0, jac=True, method="L-BFGS-B",
                                    options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))
        if single:
            return np.full(p, r.x[0]), np.full(p, r.x[1]), float(r.fun), int(r.nfev)
        return r.x[:p].copy(), r.x[p:].copy(), float(r.fun), int(r.nfev)

    def probability(self, gammas, betas, cls: int = 0) -> float:
        """Probability of cost value cls in the evolved state (statevector)."""
        with _GATE.work():
            _, out, _ = core.evolve(self.cost, self.n, self.m, gammas, betas,
                                    ws=self._evolve_workspace(len(gammas)), readout_class=cls)
            self.launches += 2 if self._small else len(gammas) + 3
            return float(out[0].item())

    def min_rounds(self, S: float = 0.5, p_max: int = 64, single: bool = True,
                   grid=None, seed: int = 0, target: str = "P", p_start: int = 1) -> MinRounds:
        """target "P": probability of a solution; "D": of a Max-SAT assignment.
        Depths p_start..p_max are searched (each depth's refinement depends
        only on its own grid seed, so a search continued at p_start = k + 1
        after depths 1..k failed returns what a search from depth 1 would)."""
        t0 = time.perf_counter()
        self.evaluations = 0
        self.launches = 0
        G, B = grid if grid is not None else grid_for(self.n, seed)
        with _GATE.work():
            out, best = core.reduced_sweep(self.hist[None], self.n, G, B, p_max)
            self.launches += 3  # phase tables, the cost-class evolution, the argmin
            bi = best[0].long()
            seed_vals = out[0, bi, torch.arange(p_max, device=out.device)].cpu().numpy()
            bi = bi.cpu().numpy()
            del out, best
        col = 0 if target == "P" else 2
        cls = 0 if target == "P" else self.min_class
        res = MinRounds(None, None, None, None, None, grid_prob=seed_vals[:, col].copy())
        for k in range(max(1, p_start), p_max + 1):
            a = int(bi[k - 1])
            g, b, e, _ = self.refine([G[a]] * k, [B[a]] * k, single=single)
            with _GATE.work():
                self._grad_calls.pop(k, None)  # this depth's checkpoints, k 2^n 8 bytes
            prob = self.probability(g, b, cls)
            if prob >= S:
                res.p, res.gammas, res.betas, res.prob, res.energy = k, g, b, prob, e
                break
        res.evaluations = self.evaluations
        res.launches = self.launches
        with _GATE.work():
            torch.cuda.current_stream().synchronize()
        res.seconds = time.perf_counter() - t0
        return res


def min_rounds_many(protocols, workers: int = 8, retry_p_max: int | None = None,
                    **kwargs) -> list:
    """Protocol.min_rounds for many instances at once: each search is a
    sequence of small GPU calls and host optimiser steps, so `workers` host
    threads, each on its own CUDA stream, keep the GPU busy while the others
    wait on the host. Instances are independent, so the results are those of
    calling min_rounds one instance after another. An instance that does not
    reach S within p_max is searched further, up to retry_p_max (if given)."""
    from concurrent.futures import ThreadPoolExecutor

    device = protocols[0].cost.device if protocols else None
    local = threading.local()  # one CUDA stream per worker thread

    def one(i):
        if not hasattr(local, "stream"):
            with _GATE.work():
                local.stream = torch.cuda.Stream(device)
        with torch.cuda.stream(local.stream):
            r = protocols[i].min_rounds(**kwargs)
            if r.p is None and retry_p_max:
                first = r
                r = protocols[i].min_rounds(**dict(kwargs, p_max=retry_p_max,
                                                   p_start=kwargs.get("p_max", 64) + 1))
                r.launches += first.launches
                r.evaluations += first.evaluations
            with _GATE.work():
                torch.cuda.current_stream().synchronize()
            return r

    with ThreadPoolExecutor(max_workers=max(1, workers)) as pool:
        return list(pool.map(one, range(len(protocols))))


def satisfiable_shapes(count: int, seed: int, n_values, d_lo: float = 2.0, d_hi: float = 4.5,
                       satisfiable: bool = True):
    """Section III's workloads: n uniform over n_values, density uniform on
    (d_lo, d_hi), m = round(n d), instances drawn until count of the wanted
    kind are found (satisfiable: h[0] > 0, the (2, 4.5) range; unsatisfiable:
    h[0] = 0, the (4.6, 8) range of the Max-SAT study), decided by the cost
    kernel. Returns [(n, m, instance seed, lits, cost, hist)]."""
    out = []
    tries = 0
    while len(out) < count:
        batch = instances.uniform_density_shapes(4 * count, seed * 1_000_003 + tries,
                                                 n_values, d_lo, d_hi)
        for i, (n, m, _) in enumerate(batch):
            iseed = (seed * 1_000_003 + tries) * 4096 + i
            lits = instances.random_3sat(n, m, iseed)
            cost, hist = core.build_cost(lits, n)
            if (int(hist[0].item()) > 0) == satisfiable:
                out.append((n, m, iseed, lits, cost, hist))
                if len(out) == count:
                    break
        tries += 1
    return out
