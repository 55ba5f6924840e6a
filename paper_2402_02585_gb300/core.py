"""PyTorch-facing wrappers of the C ABI (argument marshalling only).

Every function here allocates its outputs and workspace with torch on the
current CUDA device, passes raw pointers and the current stream to
libgqaoa.so, and returns torch tensors. All arithmetic happens in the CUDA
kernels behind the C ABI; there is no CPU fallback.

Conventions follow include/gqaoa.h: cost tables are uint8 [2^n], states are
complex64 [2^n] (torch.complex64 has the interleaved (re, im) float layout
the kernels use), angles are float64 on the device.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _capi as C

OBJECTIVES = {"p0": C.GQAOA_OBJ_P0, "energy": C.GQAOA_OBJ_ENERGY}


def objective_code(objective) -> int:
    """"p0", "energy", ("class", c) (the probability of cost value c; the
    lowest non-empty class gives the Max-SAT probability D) or a raw code."""
    if isinstance(objective, tuple) and objective[0] == "class":
        return C.GQAOA_OBJ_CLASS(objective[1])
    if isinstance(objective, int):
        return objective
    return OBJECTIVES[objective]


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensor must live on a CUDA device")


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Device scratch of at least nbytes (256-byte aligned by the allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def _angles(x, device) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=device).contiguous()


def build_cost(lits, n: int, device=None, with_hist: bool = True):
    """C(z) (uint8 [2^n]) and h[c] (int64 [m+1]) of a 3-SAT instance.

    lits: int32 [m, 3] DIMACS literals on the host (numpy or CPU tensor).
    """
    lits = np.ascontiguousarray(np.asarray(lits, dtype=np.int32).reshape(-1, 3))
    m = lits.shape[0]
    device = torch.device(device or "cuda")
    cost = torch.empty(1 << n, dtype=torch.uint8, device=device)
    hist = torch.empty(m + 1, dtype=torch.int64, device=device) if with_hist else None
    C.gqaoa_build_cost(lits.ctypes.data if m else None, n, m, _ptr(cost), _ptr(hist), _stream())
    return cost, hist


def evolve(cost: torch.Tensor, n: int, m: int, gammas, betas, state: torch.Tensor | None = None,
           state_in: bool = False, trace: bool = False, ws: torch.Tensor | None = None,
           readout_class: int = 0):
    """psi_p of Eq. 3. Returns (state complex64 [2^n], out float64 [3], trace or None);
    out[0] is the probability of cost value readout_class (default 0: P(C=0))."""
    _require_cuda(cost)
    device = cost.device
    g = _angles(gammas, device)
    b = _angles(betas, device)
    p = g.numel()
    if state is None:
        if state_in:
            raise ValueError("state_in needs a state")
        state = torch.empty(1 << n, dtype=torch.complex64, device=device)
    out = torch.empty(3, dtype=torch.float64, device=device)
    tr = torch.empty(p, dtype=torch.float64, device=device) if trace else None
    need = C.gqaoa_evolve_workspace_size(n, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    flags = (C.GQAOA_STATE_IN if state_in else 0) | C.GQAOA_READOUT_CLASS(readout_class)
    C.gqaoa_evolve(_ptr(cost), n, m, _ptr(g), _ptr(b), p, _ptr(state), _ptr(out), _ptr(tr),
                   _ptr(ws), ws.numel(), flags, _stream())
    return state, out, tr


def evolve_batched(cost: torch.Tensor, n: int, m: int, gammas, betas, shared_cost: bool = False,
                   state: torch.Tensor | None = None, state_in: bool = False, trace: bool = False,
                   ws: torch.Tensor | None = None, readout_class: int = 0):
    """Batched Eq. 3. gammas, betas [B, p]; cost [B, 2^n] or [2^n] if shared_cost.
    Returns (state [B, 2^n], out [B, 3], trace [B, p] or None); out[:, 0] is the
    probability of cost value readout_class (default 0: P(C=0))."""
    _require_cuda(cost)
    device = cost.device
    g = _angles(gammas, device)
    b = _angles(betas, device)
    B, p = g.shape
    if state is None:
        state = torch.empty((B, 1 << n), dtype=torch.complex64, device=device)
    out = torch.empty((B, 3), dtype=torch.float64, device=device)
    tr = torch.empty((B, p), dtype=torch.float64, device=device) if trace else None
    need = C.gqaoa_evolve_batched_workspace_size(n, B, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    stride = 0 if shared_cost else (1 << n)
    flags = (C.GQAOA_STATE_IN if state_in else 0) | C.GQAOA_READOUT_CLASS(readout_class)
    C.gqaoa_evolve_batched(_ptr(cost), stride, n, m, B, _ptr(g), _ptr(b), p, _ptr(state), _ptr(out),
                           _ptr(tr), _ptr(ws), ws.numel(), flags, _stream())
    return state, out, tr


def prob(state: torch.Tensor, cost: torch.Tensor, n: int, ws: torch.Tensor | None = None):
    """[P(C=0), <H_P>, norm] of a state (float64 [3] on the device)."""
    _require_cuda(state, cost)
    out = torch.empty(3, dtype=torch.float64, device=state.device)
    need = C.gqaoa_prob_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, state.device)
    C.gqaoa_prob(_ptr(state), _ptr(cost), n, _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def sample(state: torch.Tensor, n: int, seed: int, shots: int, ws: torch.Tensor | None = None,
           out: torch.Tensor | None = None):
    """Shots z ~ |psi(z)|^2 (int64 [shots] on the device)."""
    _require_cuda(state)
    if out is None:
        out = torch.empty(int(shots), dtype=torch.int64, device=state.device)
    need = C.gqaoa_sample_workspace_size(n, int(shots))
    if ws is None or ws.numel() < need:
        ws = workspace(need, state.device)
    C.gqaoa_sample(_ptr(state), n, int(seed) & 0xFFFFFFFFFFFFFFFF, int(shots), _ptr(out), _ptr(ws),
                   ws.numel(), _stream())
    return out


def evolve_sample(cost: torch.Tensor, n: int, m: int, gammas, betas, seed: int, shots: int,
                  state: torch.Tensor | None = None, state_in: bool = False, trace: bool = False,
                  ws: torch.Tensor | None = None, readout_class: int = 0):
    """Eq. 3 then Section IV's shots in one call (gqaoa_evolve_sample): returns
    (out float64 [3], trace or None, shots int64 [shots]); `state` is working
    memory and does not hold psi_p afterwards."""
    _require_cuda(cost)
    device = cost.device
    g = _angles(gammas, device)
    b = _angles(betas, device)
    p = g.numel()
    if state is None:
        if state_in:
            raise ValueError("state_in needs a state")
        state = torch.empty(1 << n, dtype=torch.complex64, device=device)
    out = torch.empty(3, dtype=torch.float64, device=device)
    tr = torch.empty(p, dtype=torch.float64, device=device) if trace else None
    shot_idx = torch.empty(int(shots), dtype=torch.int64, device=device)
    need = C.gqaoa_evolve_sample_workspace_size(n, p, int(shots))
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    flags = (C.GQAOA_STATE_IN if state_in else 0) | C.GQAOA_READOUT_CLASS(readout_class)
    C.gqaoa_evolve_sample(_ptr(cost), n, m, _ptr(g), _ptr(b), p, _ptr(state), _ptr(out), _ptr(tr),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, int(shots), _ptr(shot_idx), _ptr(ws),
                          ws.numel(), flags, _stream())
    return out, tr, shot_idx


def grad(cost: torch.Tensor, n: int, m: int, gammas, betas, objective: str = "p0",
         ws: torch.Tensor | None = None):
    """(L, dL/dgamma [p], dL/dbeta [p]) on the device, by the adjoint kernels."""
    _require_cuda(cost)
    device = cost.device
    g = _angles(gammas, device)
    b = _angles(betas, device)
    p = g.numel()
    value = torch.empty(1, dtype=torch.float64, device=device)
    dg = torch.empty(p, dtype=torch.float64, device=device)
    db = torch.empty(p, dtype=torch.float64, device=device)
    need = C.gqaoa_grad_workspace_size(n, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    C.gqaoa_grad(_ptr(cost), n, m, _ptr(g), _ptr(b), p, objective_code(objective), _ptr(value), _ptr(dg),
                 _ptr(db), _ptr(ws), ws.numel(), _stream())
    return value[0], dg, db


def grad_launches(n: int, p: int, streaming: bool = False) -> int:
    """Kernels one gqaoa_grad(_batched) call launches, following the
    library's choice of path: phase tables, the mixer coefficients'
    conversion, the cluster-resident adjoint and its closing kernel for
    10 <= n <= 16; otherwise (or with GQAOA_GRAD_STREAMING) phase tables plus
    a one-CTA forward and adjoint below 4096 amplitudes, else phase tables,
    p forward rounds, lambda init, p adjoint rounds and the finalize."""
    if 10 <= n <= 16 and not streaming:
        return 4
    if (1 << n) < 4096:
        return 3
    return 2 * p + 3


def grad_hbm_bytes(n: int, p: int, streaming: bool = False) -> int:
    """Algorithmic HBM bytes per amplitude of one gqaoa_grad(_batched)
    evaluation, following the library's choice of path: with the state on
    chip (the cluster-resident adjoint for 10 <= n <= 16, the one-CTA kernels
    below 4096 amplitudes) the cost byte once and each round's checkpoint
    written forward and read backward, 1 + 16 p; on the streaming passes the
    forward rounds (9 B, then 17 B per round), lambda's initialisation (17 B)
    and the backward rounds (25 B per round)."""
    if (10 <= n <= 16 and not streaming) or (1 << n) < 4096:
        return 1 + 16 * p
    return 9 + 17 * (p - 1) + 17 + 25 * p


def grad_batched(cost: torch.Tensor, n: int, m: int, gammas, betas, objective: str = "p0",
                 shared_cost: bool = False, ws: torch.Tensor | None = None):
    """Batched adjoint: value [B], dgamma [B, p], dbeta [B, p]."""
    _require_cuda(cost)
    device = cost.device
    g = _angles(gammas, device)
    b = _angles(betas, device)
    B, p = g.shape
    value = torch.empty(B, dtype=torch.float64, device=device)
    dg = torch.empty((B, p), dtype=torch.float64, device=device)
    db = torch.empty((B, p), dtype=torch.float64, device=device)
    need = C.gqaoa_grad_batched_workspace_size(n, B, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    stride = 0 if shared_cost else (1 << n)
    C.gqaoa_grad_batched(_ptr(cost), stride, n, m, B, _ptr(g), _ptr(b), p, objective_code(objective),
                         _ptr(value), _ptr(dg), _ptr(db), _ptr(ws), ws.numel(), _stream())
    return value, dg, db


def reduced_sweep(hist: torch.Tensor, n: int, gammas, betas, p: int, best: bool = True,
                  ws: torch.Tensor | None = None):
    """Cost-class model (Appendix C) over angle points: hist [B, stride] (int64,
    each row summing to 2^n; stride m + 1, or less when the classes past it
    are empty), gammas/betas [A] single angle pairs. Returns out [B, A, p, 3]
    (P, <H_P>, Max-SAT weight D after every round, FP32; a view of the
    library's round-major [B, p, 3, A] buffer) and, with best=True,
    best [B, p] (the angle point of smallest <H_P> per round)."""
    _require_cuda(hist)
    device = hist.device
    hist = hist.reshape(-1, hist.shape[-1]).contiguous()
    B, stride = hist.shape
    g = _angles(gammas, device).reshape(-1)
    b = _angles(betas, device).reshape(-1)
    A = g.numel()
    out = torch.empty((B, p, 3, A), dtype=torch.float32, device=device)  # round-major
    bst = torch.empty((B, p), dtype=torch.int32, device=device) if best else None
    need = C.gqaoa_reduced_sweep_workspace_size(stride, B, A, p)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    C.gqaoa_reduced_sweep(_ptr(hist), stride, n, B, _ptr(g), _ptr(b), A, p, _ptr(out), _ptr(bst),
                          _ptr(ws), ws.numel(), _stream())
    return out.permute(0, 3, 1, 2), bst


def fairness(shots: torch.Tensor, runs: int, cost: torch.Tensor, n: int, target: int,
             targets: int, chi2_crit: float, min_draws: int, ws: torch.Tensor | None = None):
    """Section IV's fair-sampling metrics per run (gqaoa_fairness): shots
    [runs * shots_per_run] (run r = shots r, r + runs, ...), the target cost
    class and its size. Returns (to_all [runs], to_reject [runs]) int64."""
    _require_cuda(shots, cost)
    device = shots.device
    per_run = shots.numel() // runs
    to_all = torch.empty(runs, dtype=torch.int64, device=device)
    to_rej = torch.empty(runs, dtype=torch.int64, device=device)
    need = C.gqaoa_fairness_workspace_size(n, runs, targets)
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    C.gqaoa_fairness(_ptr(shots), runs, per_run, _ptr(cost), n, target, targets, float(chi2_crit),
                     int(min_draws), _ptr(to_all), _ptr(to_rej), _ptr(ws), ws.numel(), _stream())
    return to_all, to_rej


class GQAOAObjective(torch.autograd.Function):
    """L(gamma, beta) = P(C=0) or <H_P> of Eq. 3, differentiable in the angles.

    forward runs the adjoint kernels once (forward passes with checkpoints,
    then the backward passes) and keeps the gradient; backward scales it by
    the incoming gradient. Works for one instance (angles [p]) or a batch of
    equal-n instances (angles [B, p], cost [B, 2^n])."""

    @staticmethod
    def forward(ctx, gammas, betas, cost, n, m, objective="p0"):
        if gammas.dim() == 1:
            v, dg, db = grad(cost, n, m, gammas.detach(), betas.detach(), objective)
        else:
            v, dg, db = grad_batched(cost, n, m, gammas.detach(), betas.detach(), objective)
        ctx.save_for_backward(dg, db)
        return v.to(gammas.dtype)

    @staticmethod
    def backward(ctx, gout):
        dg, db = ctx.saved_tensors
        if dg.dim() == 2:
            gout = gout.reshape(-1, 1)
        return (gout * dg).to(dg.dtype), (gout * db).to(db.dtype), None, None, None, None


def objective(gammas, betas, cost, n, m, objective="p0"):
    return GQAOAObjective.apply(gammas, betas, cost, n, m, objective)
