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

Evaluations are issued in one of two ways. Depth by depth (window = 1), each
depth's gqaoa_grad call is captured once into a CUDA graph and replayed for
every L-BFGS-B evaluation. With a depth window (window = W), W consecutive
depths are refined side by side: their L-BFGS-B searches advance in
lockstep and every wave of their gradient requests is one
gqaoa_grad_batched call, the shallower depths padded with identity rounds;
the shallowest depth of the window that reaches S is the answer, as in the
depth-by-depth scan. The searches are SciPy's L-BFGS-B routine stepped by
reverse communication from one thread, with the calls
scipy.optimize.minimize makes (so the same iterates, checked once per
process); where that check fails, each search runs minimize on a host
thread of its own.
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


# device memory the checkpoints of one refinement window may take
WINDOW_BUDGET_BYTES = 16 << 30


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
    makes hundreds of these small calls (each several kernel launches; 2p + 3
    on the streaming path above 2^16 amplitudes), so after one direct call the library call is
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


class _DepthBatch:
    """<H_P> and its adjoint gradient for several depths of one instance in
    one gqaoa_grad_batched call on the shared cost table. Depth k's angles sit
    at the end of a row of P rounds whose first P - k rounds have
    gamma = beta = 0: their phase factor is exactly 1 and their mixer term
    exactly 0, so the row evolves, reads out and differentiates the depth-k
    circuit (the padding rounds' derivatives are dropped). Buffers for up to
    rows_max rows of p_max rounds are allocated once; a wave moves its angles
    up in one copy from pinned memory and its values and gradients down in
    one."""

    def __init__(self, prot: "Protocol", rows_max: int, p_max: int):
        self.prot = prot
        dev = prot.cost.device
        n_in, n_out = 2 * rows_max * p_max, rows_max + 2 * rows_max * p_max
        with _GATE.work():
            self.h_in = torch.empty(n_in, dtype=torch.float64, pin_memory=True)
            self.h_out = torch.empty(n_out, dtype=torch.float64, pin_memory=True)
            self.d_in = torch.empty(n_in, dtype=torch.float64, device=dev)
            self.d_out = torch.empty(n_out, dtype=torch.float64, device=dev)
        self.a_in = self.h_in.numpy()
        self.a_out = self.h_out.numpy()
        self.ws = None
        self.ws_need = {}  # (rows, rounds) -> workspace bytes

    def __call__(self, rows, single: bool = False):
        """rows: list of (k, gammas, betas), the angles either k-vectors or,
        with `single`, two scalars used in all k rounds. Returns one
        (<H_P>, dL/dgamma, dL/dbeta) per row: with `single` the derivatives
        summed over the k rounds (floats, the sums of the k-vectors), else
        views of the k-vectors in the output buffer, valid until the next
        call."""
        prot = self.prot
        B = len(rows)
        P = pad_depth_rows(self.a_in, rows)
        nb = B + 2 * B * P
        with _GATE.work():
            st = torch.cuda.current_stream()
            d_in = self.d_in[:2 * B * P]
            d_in.copy_(self.h_in[:2 * B * P], non_blocking=True)
            need = self.ws_need.get((B, P))
            if need is None:
                need = self.ws_need[(B, P)] = C.gqaoa_grad_batched_workspace_size(prot.n, B, P)
            if self.ws is None or self.ws.numel() < need:
                self.ws = core.workspace(need, prot.cost.device)
            ang, out = d_in.data_ptr(), self.d_out.data_ptr()
            C.gqaoa_grad_batched(prot.cost.data_ptr(), 0, prot.n, prot.m, B, ang, ang + 8 * B * P, P,
                                 core.objective_code("energy"), out, out + 8 * B,
                                 out + 8 * (B + B * P), self.ws.data_ptr(), self.ws.numel(),
                                 st.cuda_stream)
            self.h_out[:nb].copy_(self.d_out[:nb], non_blocking=True)
            st.synchronize()
        prot.evaluations += B
        prot.launches += core.grad_launches(prot.n, P)
        return depth_row_results(self.a_out, rows, P, single)


def pad_depth_rows(buf: np.ndarray, rows) -> int:
    """Write the angles of rows (k, gammas, betas) into buf as the [2][B][P]
    block [gammas | betas] of a batched call, P the deepest k: row i's k
    angles (k-vectors, or scalars repeated in all k rounds) in its last k
    rounds, its first P - k rounds zero (identity rounds: phase factor 1,
    mixer term 0). Returns P."""
    B = len(rows)
    P = max(k for k, _, _ in rows)
    a = buf[:2 * B * P].reshape(2, B, P)
    a[:] = 0.0
    for i, (k, g, b) in enumerate(rows):
        a[0, i, P - k:] = g
        a[1, i, P - k:] = b
    return P


def depth_row_results(buf: np.ndarray, rows, P: int, single: bool):
    """Read a batched call's output [value [B] | dgamma [B][P] | dbeta [B][P]]
    from buf for rows padded by pad_depth_rows: one (value, dL/dgamma,
    dL/dbeta) per row over its own last k rounds (the padding rounds'
    derivatives dropped): with `single` summed over the k rounds (floats),
    else views of the k-vectors in buf."""
    B = len(rows)
    v = buf[:B]
    gr = buf[B:B + 2 * B * P].reshape(2, B, P)
    if single:
        return [(float(v[i]), float(gr[0, i, P - k:].sum()), float(gr[1, i, P - k:].sum()))
                for i, (k, _, _) in enumerate(rows)]
    return [(float(v[i]), gr[0, i, P - k:], gr[1, i, P - k:]) for i, (k, _, _) in enumerate(rows)]


class _Lbfgsb:
    """One L-BFGS-B search run by reverse communication: point() is the next
    x to evaluate (None once the search has ended), tell(f, g) gives the
    value and gradient there. It drives SciPy's L-BFGS-B routine (setulb,
    one step per call) with the calls scipy.optimize.minimize(method=
    "L-BFGS-B") makes for the same options and its defaults (10 corrections,
    20 line-search steps, 15000 evaluations, no bounds): an evaluation at x0
    before the first call, the last value reused when the routine asks again
    for the same x, and the iteration and evaluation limits checked at each
    new iterate. So its iterates, evaluation count and result are minimize's
    bit for bit (`lbfgsb_matches_scipy` checks this once per process), while
    many searches can be stepped from one thread."""

    def __init__(self, x0, ftol: float, gtol: float, maxiter: int, maxcor: int = 10,
                 maxls: int = 20, maxfun: int = 15000):
        from scipy.linalg.lapack import HAS_ILP64
        from scipy.optimize import _lbfgsb
        self._setulb = _lbfgsb.setulb
        it = np.int64 if HAS_ILP64 else np.int32
        self.x = np.array(x0, dtype=np.float64).ravel()
        n, m = self.x.size, maxcor
        self.m, self.maxls, self.maxiter, self.maxfun = m, maxls, maxiter, maxfun
        self.factr = ftol / np.finfo(float).eps
        self.pgtol = gtol
        self.lo = np.zeros(n)
        self.hi = np.zeros(n)
        self.nbd = np.zeros(n, dtype=it)
        self.wa = np.zeros(2 * m * n + 5 * n + 11 * m * m + 8 * m)
        self.iwa = np.zeros(3 * n, dtype=it)
        self.task = np.zeros(2, dtype=it)
        self.ln_task = np.zeros(2, dtype=it)
        self.lsave = np.zeros(4, dtype=it)
        self.isave = np.zeros(44, dtype=it)
        self.dsave = np.zeros(29)
        self.f = 0.0
        self.g = np.zeros(n)
        self.nit = 0
        self.nfev = 0
        self.last = None          # (x, f, g) of the latest evaluation
        self.want = self.x.copy()  # minimize evaluates at x0 first
        self.converged = False

    def point(self):
        return self.want

    def tell(self, f, g):
        self.nfev += 1
        self.last = (self.want, float(f), np.array(g, dtype=np.float64).ravel())
        if self.nfev > 1:
            self.f, self.g = self.last[1], self.last[2].copy()
        while True:
            self._setulb(self.m, self.x, self.lo, self.hi, self.nbd, self.f, self.g, self.factr,
                         self.pgtol, self.wa, self.iwa, self.task, self.lsave, self.isave,
                         self.dsave, self.maxls, self.ln_task)
            task = int(self.task[0])
            if task == 3:  # f and g wanted at self.x
                if np.array_equal(self.x, self.last[0]):
                    self.f, self.g = self.last[1], self.last[2].copy()
                    continue
                self.want = self.x.copy()
                return
            if task == 1:  # a new iterate
                self.nit += 1
                if self.nit >= self.maxiter:
                    self.task[0], self.task[1] = 5, 504
                elif self.nfev > self.maxfun:
                    self.task[0], self.task[1] = 5, 502
                continue
            self.converged = task == 4
            self.want = None
            return


_LBFGSB_OK = None


def lbfgsb_matches_scipy() -> bool:
    """Whether _Lbfgsb reproduces scipy.optimize.minimize(method="L-BFGS-B")
    bit for bit on this SciPy (a few seeded smooth problems of 2 and 12
    variables); False as well if SciPy's low-level routine is missing or has
    another interface. Checked once per process."""
    global _LBFGSB_OK
    if _LBFGSB_OK is not None:
        return _LBFGSB_OK
    ok = True
    try:
        rng = np.random.default_rng(7)
        for n in (2, 12):
            A = rng.normal(size=(n, n))
            H = A @ A.T + np.eye(n)
            c = rng.normal(size=n)

            def fun(x):
                r = x - c
                return float(0.5 * r @ H @ r + 0.3 * np.sin(x).sum()), H @ r + 0.3 * np.cos(x)

            x0 = rng.normal(size=n)
            ref = scipy.optimize.minimize(fun, x0, jac=True, method="L-BFGS-B",
                                          options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))
            s = _Lbfgsb(x0, 1e-6, 1e-10, 500)
            while s.point() is not None:
                s.tell(*fun(s.point()))
            ok = ok and np.array_equal(s.x, ref.x) and s.f == ref.fun and s.nfev == ref.nfev
    except Exception:  # another SciPy: the threaded lockstep is used instead
        ok = False
    _LBFGSB_OK = ok
    return ok


class _Lockstep:
    """Runs several L-BFGS-B searches side by side, one host thread each, and
    gathers every wave of their evaluation requests into one call: a wave is
    served once each search still running has asked for its next point. Each
    search waits on its own event and the serving thread on one more, so a
    wave wakes every thread once."""

    def __init__(self, keys):
        self.lock = threading.Lock()
        self.ready = threading.Event()  # the serving thread's
        self.done = {k: threading.Event() for k in keys}
        self.pending = {}
        self.results = {}
        self.live = len(self.done)
        self.error = None

    def request(self, i, x):
        ev = self.done[i]
        ev.clear()
        with self.lock:
            self.pending[i] = x
            if len(self.pending) >= self.live:
                self.ready.set()
        ev.wait()
        if self.error is not None:
            raise RuntimeError("lockstep evaluation failed") from self.error
        return self.results.pop(i)

    def finished(self):
        with self.lock:
            self.live -= 1
            if len(self.pending) >= self.live:
                self.ready.set()

    def serve(self, evaluate):
        """evaluate(dict i -> x) -> dict i -> (value, gradient); runs on the
        calling thread until every search has finished."""
        while True:
            self.ready.wait()
            with self.lock:
                self.ready.clear()
                if self.live == 0:
                    return
                if len(self.pending) < self.live:
                    continue
                batch, self.pending = self.pending, {}
            try:
                out = evaluate(batch)
            except BaseException as exc:  # wake the searches, then re-raise
                self.error = exc
                for k in batch:
                    self.done[k].set()
                raise
            self.results.update(out)
            for k in out:
                self.done[k].set()


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
        nz = np.nonzero(h)[0]
        self.min_class = int(nz[0])  # 0 when satisfiable
        # the grid search's histogram ends at the last non-empty class: the
        # cost-class kernel's work grows with the row length
        self.grid_hist = hist[:int(nz[-1]) + 1].reshape(1, -1).contiguous()

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
        self.launches += core.grad_launches(self.n, p)
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
        if lbfgsb_matches_scipy():  # minimize's search, without its per-call wrapping
            s = _Lbfgsb(x0, 1e-6, 1e-10, 500)
            while s.point() is not None:
                s.tell(*fun(s.point()))
            x, fx, nfev = s.x, s.f, s.nfev
        else:
            r = scipy.optimize.minimize(fun, x0, jac=True, method="L-BFGS-B",
                                        options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))
            x, fx, nfev = r.x, r.fun, r.nfev
        if single:
            return np.full(p, x[0]), np.full(p, x[1]), float(fx), int(nfev)
        return x[:p].copy(), x[p:].copy(), float(fx), int(nfev)

    def probability(self, gammas, betas, cls: int = 0) -> float:
        """Probability of cost value cls in the evolved state (statevector)."""
        with _GATE.work():
            _, out, _ = core.evolve(self.cost, self.n, self.m, gammas, betas,
                                    ws=self._evolve_workspace(len(gammas)), readout_class=cls)
            self.launches += 2 if self._small else len(gammas) + 3
            return float(out[0].item())

    def refine_window(self, depths, seeds, single: bool):
        """L-BFGS-B on <H_P> for several depths at once (depth k from the
        single angle pair seeds[k]): the searches run side by side and each
        wave of their gradient requests is one batched call (_DepthBatch).
        Each depth's search is the one refine() makes, so the results equal
        refine()'s up to the rounding of the batched sums. The searches are
        stepped from the calling thread (_Lbfgsb) where that reproduces
        SciPy's minimize bit for bit, else each runs minimize on a host
        thread of its own (_Lockstep). Returns {k: (gammas, betas, <H_P>)}."""
        batch = _DepthBatch(self, len(depths), max(depths))
        results, errors = {}, []

        def rows_of(wave):
            if single:
                return [(k, x[0], x[1]) for k, x in wave.items()]
            return [(k, x[:k], x[k:]) for k, x in wave.items()]

        def evaluate(wave):
            out = batch(rows_of(wave), single)
            res = {}
            for k, (e, dg, db) in zip(wave, out):
                res[k] = (e, np.array([dg, db]) if single else np.concatenate([dg, db]))
            return res

        def x0_of(k):
            g0, b0 = seeds[k]
            return np.array([g0, b0]) if single else np.concatenate([np.full(k, g0), np.full(k, b0)])

        def keep(k, x, fun):
            if single:
                results[k] = (np.full(k, x[0]), np.full(k, x[1]), float(fun))
            else:
                results[k] = (x[:k].copy(), x[k:].copy(), float(fun))

        if lbfgsb_matches_scipy():
            # every search stepped from this thread: one batched call per wave
            searches = {k: _Lbfgsb(x0_of(k), 1e-6, 1e-10, 500) for k in depths}
            while True:
                wave = {k: s.point() for k, s in searches.items() if s.point() is not None}
                if not wave:
                    break
                for k, fg in evaluate(wave).items():
                    searches[k].tell(*fg)
            for k, s in searches.items():
                keep(k, s.x, s.f)
            return results

        # the same searches by scipy.optimize.minimize, one host thread each
        steps = _Lockstep(depths)

        def search(k):
            try:
                r = scipy.optimize.minimize(lambda x: steps.request(k, x), x0_of(k), jac=True,
                                            method="L-BFGS-B",
                                            options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))
                keep(k, r.x, r.fun)
            except BaseException as exc:
                errors.append(exc)
            finally:
                steps.finished()

        stream = torch.cuda.current_stream()
        threads = [threading.Thread(target=search, args=(k,)) for k in depths]
        for t in threads:
            t.start()
        try:
            with torch.cuda.stream(stream):
                steps.serve(evaluate)
        finally:
            for t in threads:
                t.join()
        if errors:
            raise errors[0]
        return results

    def probabilities(self, rows, cls: int = 0):
        """Probability of cost value cls after each (gammas, betas) of rows
        (several depths at once, padded as in _DepthBatch; statevector)."""
        P = max(len(g) for g, _ in rows)
        G = np.zeros((len(rows), P))
        Bt = np.zeros((len(rows), P))
        for i, (g, b) in enumerate(rows):
            G[i, P - len(g):] = g
            Bt[i, P - len(b):] = b
        with _GATE.work():
            _, out, _ = core.evolve_batched(self.cost, self.n, self.m, G, Bt, shared_cost=True,
                                            readout_class=cls)
            self.launches += 2 if self._small else P + 3
            return out[:, 0].cpu().numpy()

    def min_rounds(self, S: float = 0.5, p_max: int = 64, single: bool = True,
                   grid=None, seed: int = 0, target: str = "P", p_start: int = 1,
                   window: int = 1) -> MinRounds:
        """target "P": probability of a solution; "D": of a Max-SAT assignment.
        Depths p_start..p_max are searched (each depth's refinement depends
        only on its own grid seed, so a search continued at p_start = k + 1
        after depths 1..k failed returns what a search from depth 1 would).
        window > 1 refines that many consecutive depths at once
        (refine_window, with batched gradient calls) and accepts the
        shallowest of them that reaches S; its checkpoints are kept within
        WINDOW_BUDGET_BYTES by narrowing the window for large states."""
        t0 = time.perf_counter()
        self.evaluations = 0
        self.launches = 0
        G, B = grid if grid is not None else grid_for(self.n, seed)
        with _GATE.work():
            out, best = core.reduced_sweep(self.grid_hist, self.n, G, B, p_max)
            self.launches += 4  # phase tables, minima reset, the cost-class evolution, argmin
            bi = best[0].long()
            seed_vals = out[0, bi, torch.arange(p_max, device=out.device)].cpu().numpy()
            bi = bi.cpu().numpy()
            del out, best
        col = 0 if target == "P" else 2
        cls = 0 if target == "P" else self.min_class
        res = MinRounds(None, None, None, None, None, grid_prob=seed_vals[:, col].copy())
        k0 = max(1, p_start)
        while window > 1 and k0 <= p_max:
            W = window
            while W > 1 and W * (k0 + W - 1) * (8 << self.n) > WINDOW_BUDGET_BYTES:
                W -= 1
            depths = list(range(k0, min(p_max, k0 + W - 1) + 1))
            seeds = {k: (G[int(bi[k - 1])], B[int(bi[k - 1])]) for k in depths}
            ref = self.refine_window(depths, seeds, single)
            probs = self.probabilities([(ref[k][0], ref[k][1]) for k in depths], cls)
            for k, prob in zip(depths, probs):
                if prob >= S:
                    g, b, e = ref[k]
                    res.p, res.gammas, res.betas, res.prob, res.energy = k, g, b, float(prob), e
                    break
            if res.p is not None:
                break
            k0 = depths[-1] + 1
        for k in range(k0, p_max + 1) if window <= 1 else ():
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
