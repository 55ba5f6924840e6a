"""The paper's angle protocol (Appendix C, "Optimization"), FP64 numpy/scipy on
the cost-class model.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Appendix C minimises the cost function <H_P> (Eq. 4) of single-angle-pair
G-QAOA in three steps: evaluate it on a uniform (beta, gamma) grid of spacing
pi/180 (n <= 20; 4000 sampled angle pairs above), start L-BFGS-B from the
best grid point with a stopping criterion of 1e-6 relative change of the cost
between iterations, and, for G-QAOA with per-round angles, start the same
L-BFGS-B from the same seed over all 2p angles. Section III then reports, per
instance, the fewest rounds p whose optimised state has solution
probability of at least S (50 %; 25 % and 75 % in Appendix C).

Every evaluation here is the exact (m+1)-dimensional model of
oracle.reduced, whose forward pass and adjoint gradient are pinned against
the statevector oracle. Grid values for all prefix depths come from one
evolution per angle pair (the trace after every round).
"""

from __future__ import annotations

import numpy as np
import scipy.optimize

from . import reduced


def grid_readouts(hist, gammas, betas, p: int):
    """E[a][k], P[a][k], D[a][k] after rounds k = 1..p for every single angle
    pair (gammas[a], betas[a]) (the cost-class recurrence of oracle.reduced,
    evaluated for all angle pairs at once)."""
    h = np.asarray(hist, dtype=np.float64)
    N = h.sum()
    c = np.arange(h.shape[0], dtype=np.float64)
    cs = reduced.min_class(hist)
    G = np.asarray(gammas, np.float64)[:, None]
    B = np.asarray(betas, np.float64)[:, None]
    T = np.exp(-1j * G * c[None, :])
    alpha = np.exp(-1j * B) - 1.0
    f = np.full((G.shape[0], h.shape[0]), 1.0 / np.sqrt(N), dtype=np.complex128)
    E = np.empty((G.shape[0], p))
    P = np.empty((G.shape[0], p))
    D = np.empty((G.shape[0], p))
    for k in range(p):
        g = T * f
        S = g @ h
        f = g + alpha * (S[:, None] / N)
        w = np.abs(f) ** 2 * h[None, :]
        E[:, k] = w @ c
        P[:, k] = w[:, 0]
        D[:, k] = w[:, cs]
    return E, P, D


def refine(hist, gammas0, betas0, single: bool):
    """L-BFGS-B on <H_P> from the given angles (relative cost change 1e-6).
    single: one (gamma, beta) for all rounds, gradient = sum over rounds of
    the per-round adjoint gradient; else all 2p angles. Returns
    (gammas [p], betas [p], <H_P>, function evaluations)."""
    g0 = np.asarray(gammas0, np.float64)
    b0 = np.asarray(betas0, np.float64)
    p = g0.shape[0]
    if single:
        def fun(x):
            L, dg, db = reduced.grad(hist, [x[0]] * p, [x[1]] * p, reduced.OBJ_ENERGY)
            return L, np.array([dg.sum(), db.sum()])
        x0 = np.array([g0[0], b0[0]])
    else:
        def fun(x):
            L, dg, db = reduced.grad(hist, x[:p], x[p:], reduced.OBJ_ENERGY)
            return L, np.concatenate([dg, db])
        x0 = np.concatenate([g0, b0])
    r = scipy.optimize.minimize(fun, x0, jac=True, method="L-BFGS-B",
                                options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))
    if single:
        return np.full(p, r.x[0]), np.full(p, r.x[1]), float(r.fun), int(r.nfev)
    return r.x[:p].copy(), r.x[p:].copy(), float(r.fun), int(r.nfev)


def min_rounds(hist, gammas, betas, S: float = 0.5, p_max: int = 64, single: bool = True,
               target: str = "P"):
    """Fewest rounds k <= p_max whose <H_P>-optimised state reaches
    probability S of a solution (target "P") or of a Max-SAT assignment
    (target "D"). Every depth k = 1, 2, ... is optimised in turn, as
    Appendix C does for each instance and depth: the seed is the grid point
    of lowest <H_P> after k rounds, L-BFGS-B starts from it over the single
    angle pair (single) or over all 2k per-round angles (not single: the
    same seed, every angle free), and the depth is accepted when the
    optimised state reaches S. Returns (k or None, gammas, betas,
    probability, <H_P>)."""
    E, _, _ = grid_readouts(hist, gammas, betas, p_max)
    G = np.asarray(gammas, np.float64)
    B = np.asarray(betas, np.float64)
    for k in range(1, p_max + 1):
        a = int(np.argmin(E[:, k - 1]))
        g, b, e, _ = refine(hist, [G[a]] * k, [B[a]] * k, single=single)
        r = reduced.readouts_trace(hist, g, b)[-1]
        val = r[0] if target == "P" else r[2]
        if val >= S:
            return k, g, b, float(val), float(e)
    return None, None, None, None, None
