"""Exact (m+1)-dimensional cost-class model of G-QAOA (Appendix C), FP64 numpy.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Appendix C notes that G-QAOA is invariant under relabelling the states inside
one energy manifold, so starting from |+> the state stays a function of the
cost value: psi_k(z) = f_k(C(z)). With h[c] the manifold sizes and N = 2^n,
one round of Eq. 3 becomes

    g_k(c) = e^{-i gamma_k c} f_{k-1}(c)                 (phase, Eq. 3)
    S_k    = sum_c h[c] g_k(c)                            (= sum_z chi_k(z))
    f_k(c) = g_k(c) + (e^{-i beta_k} - 1) S_k / N         (mixer, Eq. 2)

from f_0(c) = N^{-1/2}. Then P = h[0] |f_p(0)|^2 and <H_P> = sum_c c h[c] |f_p(c)|^2.

The adjoint gradient below differentiates the same recurrence. For an
objective L = <psi_p|O|psi_p> with O diagonal in the cost value
(O = projector on C=0 for P, O = diag(c) for <H_P>), lambda_p = O f_p and for
k = p..1:

    dL/dbeta_k  = 2 Re[ -i e^{-i beta_k} (S_k / N) conj(sum_c h[c] lambda_k(c)) ]
    mu_k        = lambda_k + (e^{+i beta_k} - 1) (sum_c h[c] lambda_k(c)) / N
    dL/dgamma_k = 2 Re[ sum_c h[c] conj(mu_k(c)) (-i c) g_k(c) ]
    lambda_{k-1} = e^{+i gamma_k c} mu_k

(the chain rule for L = <f, O f> in the h-weighted inner product; mu_k is the
adjoint after undoing the mixer, lambda_{k-1} after undoing the phase).

Pins: equality with the full statevector oracle at small n (every amplitude),
central finite differences of its own forward pass and of the statevector
oracle, and the special cases pinned for the statevector oracle.
"""

from __future__ import annotations

import numpy as np

OBJ_P0 = 0
OBJ_ENERGY = 1


def evolve(hist, gammas, betas, trace: bool = False):
    """f_p(c) as complex128 [m+1]; with trace=True also P after each round."""
    h = np.asarray(hist, dtype=np.float64)
    N = h.sum()
    c = np.arange(h.shape[0], dtype=np.float64)
    f = np.full(h.shape[0], 1.0 / np.sqrt(N), dtype=np.complex128)
    tr = []
    for g, b in zip(np.asarray(gammas, np.float64), np.asarray(betas, np.float64)):
        gk = np.exp(-1j * g * c) * f
        S = np.sum(h * gk)
        f = gk + (np.exp(-1j * b) - 1.0) * S / N
        if trace:
            tr.append(h[0] * abs(f[0]) ** 2)
    return (f, np.array(tr)) if trace else f


def min_class(hist) -> int:
    """The lowest cost value with a non-empty manifold: the number of clauses
    a Max-SAT assignment leaves unsatisfied (0 for a satisfiable instance)."""
    h = np.asarray(hist)
    nz = np.nonzero(h)[0]
    return int(nz[0])


def readouts_trace(hist, gammas, betas):
    """[p][3]: after every round k, P(C=0), <H_P> and D = sum over the lowest
    non-empty class c* of |psi_k|^2 = h[c*] |f_k(c*)|^2 (the probability of
    measuring a Max-SAT assignment; D = P when the instance is satisfiable)."""
    h = np.asarray(hist, dtype=np.float64)
    N = h.sum()
    c = np.arange(h.shape[0], dtype=np.float64)
    cs = min_class(hist)
    f = np.full(h.shape[0], 1.0 / np.sqrt(N), dtype=np.complex128)
    out = []
    for g, b in zip(np.asarray(gammas, np.float64), np.asarray(betas, np.float64)):
        gk = np.exp(-1j * g * c) * f
        S = np.sum(h * gk)
        f = gk + (np.exp(-1j * b) - 1.0) * S / N
        w = h * np.abs(f) ** 2
        out.append((w[0], np.sum(c * w), w[cs]))
    return np.array(out).reshape(-1, 3)


def readout(hist, f):
    """[P(C=0), <H_P>, norm] of the class-amplitude vector f."""
    h = np.asarray(hist, dtype=np.float64)
    c = np.arange(h.shape[0], dtype=np.float64)
    w = h * np.abs(f) ** 2
    return np.array([w[0], np.sum(c * w), np.sum(w)])


def amplitudes(f, cost):
    """psi_p(z) = f_p(C(z)) for the given cost values."""
    return np.asarray(f)[np.asarray(cost, dtype=np.int64)]


def grad(hist, gammas, betas, objective: int = OBJ_P0, target: int = 0):
    """(L, dL/dgamma [p], dL/dbeta [p]) by the adjoint recurrence above.
    OBJ_P0 projects on cost value `target` (0: P(C=0); the lowest non-empty
    class: the Max-SAT probability D)."""
    h = np.asarray(hist, dtype=np.float64)
    N = h.sum()
    c = np.arange(h.shape[0], dtype=np.float64)
    gammas = np.asarray(gammas, np.float64)
    betas = np.asarray(betas, np.float64)
    p = gammas.shape[0]
    f = np.full(h.shape[0], 1.0 / np.sqrt(N), dtype=np.complex128)
    gs, Ss = [], []
    for k in range(p):
        gk = np.exp(-1j * gammas[k] * c) * f
        S = np.sum(h * gk)
        f = gk + (np.exp(-1j * betas[k]) - 1.0) * S / N
        gs.append(gk)
        Ss.append(S)
    if objective == OBJ_P0:
        O = (c == target).astype(np.float64)
    elif objective == OBJ_ENERGY:
        O = c
    else:
        raise ValueError("objective")
    L = float(np.sum(h * O * np.abs(f) ** 2))
    lam = O * f
    dg = np.zeros(p)
    db = np.zeros(p)
    for k in range(p - 1, -1, -1):
        lam_sum = np.sum(h * lam)
        db[k] = 2.0 * np.real(-1j * np.exp(-1j * betas[k]) * (Ss[k] / N) * np.conj(lam_sum))
        mu = lam + (np.exp(1j * betas[k]) - 1.0) * lam_sum / N
        dg[k] = 2.0 * np.real(np.sum(h * np.conj(mu) * (-1j * c) * gs[k]))
        lam = np.exp(1j * gammas[k] * c) * mu
    return L, dg, db


def objective_value(hist, gammas, betas, objective: int = OBJ_P0, target: int = 0) -> float:
    f = evolve(hist, gammas, betas)
    if objective == OBJ_P0:
        return float(np.asarray(hist, np.float64)[target] * abs(f[target]) ** 2)
    return float(readout(hist, f)[1])


def fd_grad(hist, gammas, betas, objective: int = OBJ_P0, step: float = 1e-4, target: int = 0):
    """Central finite differences of objective_value (FP64)."""
    gammas = np.array(gammas, np.float64)
    betas = np.array(betas, np.float64)
    p = gammas.shape[0]
    dg = np.zeros(p)
    db = np.zeros(p)
    for k in range(p):
        for arr, out in ((gammas, dg), (betas, db)):
            old = arr[k]
            arr[k] = old + step
            up = objective_value(hist, gammas, betas, objective, target)
            arr[k] = old - step
            dn = objective_value(hist, gammas, betas, objective, target)
            arr[k] = old
            out[k] = (up - dn) / (2 * step)
    return dg, db
