"""Batched G-QAOA angle optimisation on the GPU.

Appendix C optimises the angles with a gradient method from grid or random
seeds. Here every step is one call of the batched adjoint kernels
(gqaoa_grad_batched: forward rounds with checkpoints, backward rounds) and
one Adam kernel (gqaoa_adam_f64) over all instances' angles; Python only
sequences the calls. Angles live on the device as theta[2, B, p]
(gammas, betas), contiguous per half.
"""

from __future__ import annotations

import time

import numpy as np
import torch

from . import _capi as C
from . import core


class AngleOptimizer:
    """Adam over the 2p angles of B equal-n instances (cost [B, 2^n] uint8)."""

    def __init__(self, cost: torch.Tensor, n: int, m: int, p: int, objective: str = "p0"):
        if cost.dim() != 2:
            raise ValueError("cost must be [B, 2^n]")
        self.cost = cost
        self.n, self.m, self.p = n, m, p
        self.B = cost.shape[0]
        self.objective = objective
        self.sign = -1.0 if objective == "p0" else 1.0  # maximise P, minimise <H>
        dev = cost.device
        self.theta = torch.zeros((2, self.B, p), dtype=torch.float64, device=dev)
        self.grad = torch.zeros_like(self.theta)
        self.m1 = torch.zeros_like(self.theta)
        self.m2 = torch.zeros_like(self.theta)
        self.value = torch.zeros(self.B, dtype=torch.float64, device=dev)
        self.ws = core.workspace(C.gqaoa_grad_batched_workspace_size(n, self.B, p), dev)
        self.t = 0
        self.launches = 0        # kernels launched by the library for this optimizer
        self.amp_evaluations = 0  # instances x 2^n x gradient evaluations

    def reset(self, gammas, betas):
        self.theta[0].copy_(torch.as_tensor(gammas, dtype=torch.float64))
        self.theta[1].copy_(torch.as_tensor(betas, dtype=torch.float64))
        self.m1.zero_()
        self.m2.zero_()
        self.t = 0

    def evaluate(self) -> torch.Tensor:
        """Objective and gradient at the current angles (value [B] on the device)."""
        s = torch.cuda.current_stream().cuda_stream
        C.gqaoa_grad_batched(self.cost.data_ptr(), 1 << self.n, self.n, self.m, self.B,
                             self.theta[0].data_ptr(), self.theta[1].data_ptr(), self.p,
                             core.objective_code(self.objective), self.value.data_ptr(),
                             self.grad[0].data_ptr(), self.grad[1].data_ptr(), self.ws.data_ptr(),
                             self.ws.numel(), s)
        self.launches += core.grad_launches(self.n, self.p)
        self.amp_evaluations += self.B << self.n
        return self.value

    def step(self, lr: float = 0.05, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        """One Adam step; returns the objective at the angles before the step."""
        v = self.evaluate()
        self.t += 1
        C.gqaoa_adam_f64(self.theta.data_ptr(), self.grad.data_ptr(), self.m1.data_ptr(),
                         self.m2.data_ptr(), self.theta.numel(), lr, beta1, beta2, eps, self.t,
                         self.sign, torch.cuda.current_stream().cuda_stream)
        self.launches += 1
        return v

    def run(self, steps: int, lr: float = 0.05, target: torch.Tensor | None = None):
        """Adam for `steps` steps. Returns a dict with the value history [steps+1, B]
        (host), wall-clock seconds at each evaluation, and, when `target` [B] is
        given, the first evaluation index at which each instance reached it
        (-1 if never)."""
        hist = []
        wall = []
        t0 = time.perf_counter()
        for _ in range(steps):
            v = self.step(lr)
            hist.append(v.clone())
            torch.cuda.synchronize()
            wall.append(time.perf_counter() - t0)
        v = self.evaluate().clone()
        torch.cuda.synchronize()
        hist.append(v)
        wall.append(time.perf_counter() - t0)
        H = torch.stack(hist).cpu().numpy()
        out = {"values": H, "wall": np.array(wall)}
        if target is not None:
            tgt = target.cpu().numpy() if isinstance(target, torch.Tensor) else np.asarray(target)
            ok = (H >= tgt[None, :]) if self.sign < 0 else (H <= tgt[None, :])
            first = np.where(ok.any(0), ok.argmax(0), -1)
            out["first_hit"] = first
        return out

    def angles(self):
        return self.theta[0].clone(), self.theta[1].clone()


def canonicalize(gammas: np.ndarray, betas: np.ndarray) -> np.ndarray:
    """Labels [B, 2p] in [0, 2 pi): angles are 2 pi periodic (C is an integer
    and H_M a projector) and (gamma, beta) -> (-gamma, -beta) conjugates the
    state without changing P or <H>; the representative with gamma_1 <= pi is
    kept."""
    g = np.mod(np.asarray(gammas, dtype=np.float64), 2 * np.pi)
    b = np.mod(np.asarray(betas, dtype=np.float64), 2 * np.pi)
    flip = g[:, 0] > np.pi
    g[flip] = np.mod(2 * np.pi - g[flip], 2 * np.pi)
    b[flip] = np.mod(2 * np.pi - b[flip], 2 * np.pi)
    return np.concatenate([g, b], axis=1)


def single_angle_grid_start(cost: torch.Tensor, n: int, m: int, p: int, grid: int = 16,
                            objective: str = "p0"):
    """Best single angle pair (Eq. 5) on a grid x grid lattice of [0, 2pi) x [0, pi)
    per instance (cost [B, 2^n]). P(C=0) of every lattice point comes from one
    persistent sweep (gqaoa_sweep) when n allows, else from batched evolution with
    the instance's cost table shared by the lattice. Returns gammas [B], betas [B]."""
    B = cost.shape[0]
    gs = (np.arange(grid) + 0.5) * (2 * np.pi / grid)
    bs = (np.arange(grid) + 0.5) * (np.pi / grid)
    G = np.repeat(gs, grid)
    Bt = np.tile(bs, grid)
    A = grid * grid
    if objective == "p0" and C.GQAOA_SWEEP_MIN_N <= n <= C.GQAOA_SWEEP_L2_MAX_N:
        gd = torch.as_tensor(G, device=cost.device)
        bd = torch.as_tensor(Bt, device=cost.device)
        out = torch.empty((B, A, 1), dtype=torch.float64, device=cost.device)
        ws = core.workspace(C.gqaoa_sweep_workspace_size(n, A, 0), cost.device)
        r = np.array([p], dtype=np.int32)
        C.gqaoa_sweep(cost.data_ptr(), n, m, B, gd.data_ptr(), bd.data_ptr(), A, p, r.ctypes.data, 1,
                      0, out.data_ptr(), ws.data_ptr(), ws.numel(),
                      torch.cuda.current_stream().cuda_stream)
        k = torch.argmax(out[:, :, 0], dim=1).cpu().numpy()
        return G[k], Bt[k]
    Gm = np.repeat(G[:, None], p, 1)
    Bm = np.repeat(Bt[:, None], p, 1)
    best_g = np.zeros(B)
    best_b = np.zeros(B)
    gd = torch.as_tensor(Gm, device=cost.device)
    bd = torch.as_tensor(Bm, device=cost.device)
    state = torch.empty((A, 1 << n), dtype=torch.complex64, device=cost.device)
    ws = core.workspace(C.gqaoa_evolve_batched_workspace_size(n, A, p), cost.device)
    for i in range(B):
        _, out, _ = core.evolve_batched(cost[i], n, m, gd, bd, shared_cost=True, state=state, ws=ws)
        col = out[:, 0] if objective == "p0" else -out[:, 1]
        k = int(torch.argmax(col).item())
        best_g[i], best_b[i] = G[k], Bt[k]
    return best_g, best_b
