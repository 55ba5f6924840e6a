"""Seeded synthetic inputs: random 3-SAT instances and random angle schedules.

This module draws inputs only. It holds none of the method's arithmetic (no
clause evaluation, no cost table, no evolution), so both the CUDA path and the
CPU oracle can be fed from it without sharing any computation.

Instance recipe (Section III and Appendix C of arXiv:2402.02585):
  * each clause takes 3 distinct variables, uniformly at random among the n;
  * each literal is negated with probability 1/2;
  * m = round(d * n) clauses, rounded half up;
  * the paper keeps one copy of any repeated clause; here a repeated clause
    (same literal set, order ignored) is redrawn, so the instance keeps
    exactly m distinct clauses.

Literals use the DIMACS convention: +(v+1) is variable v, -(v+1) its negation.

Every draw comes from the raw 64-bit output of numpy's PCG64 (stable across
numpy versions and machines) mapped to ranges with integer arithmetic, so an
instance is identical on every host.
"""

from __future__ import annotations

import math

import numpy as np

_STREAM_CLAUSES = 0
_STREAM_ANGLES = 1
_STREAM_SHAPE = 2
_STREAM_PROTOCOL = 5
_STREAM_SHOTS = 6


def _raw(seed: int, stream: int) -> np.random.PCG64:
    return np.random.PCG64([int(seed), int(stream)])


def _below(bg: np.random.PCG64, bound: np.ndarray) -> np.ndarray:
    """Integers in [0, bound) from 64-bit words by the multiply-high map."""
    bound = np.asarray(bound, dtype=np.uint64)
    x = bg.random_raw(bound.size).astype(np.uint64).reshape(bound.shape)
    # (x * bound) >> 64 without 128-bit ints: split x into 32-bit halves.
    x_hi = x >> np.uint64(32)
    x_lo = x & np.uint64(0xFFFFFFFF)
    b = bound
    lo_prod = (x_lo * b) >> np.uint64(32)
    return ((x_hi * b + lo_prod) >> np.uint64(32)).astype(np.int64)


def _unit(bg: np.random.PCG64, size: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    x = bg.random_raw(size).astype(np.uint64)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def clause_count(n: int, d: float) -> int:
    """m = round(d * n), half up (Appendix C leaves the rounding open)."""
    return int(math.floor(d * n + 0.5))


def _draw_clauses(bg: np.random.PCG64, n: int, k: int) -> np.ndarray:
    a = _below(bg, np.full(k, n))
    b = _below(bg, np.full(k, n - 1))
    b = b + (b >= a)
    c = _below(bg, np.full(k, n - 2))
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    c = c + (c >= lo)
    c = c + (c >= hi)
    var = np.stack([a, b, c], axis=1)
    neg = _below(bg, np.full((k, 3), 2)).astype(bool)
    lits = (var + 1) * np.where(neg, -1, 1)
    return lits.astype(np.int32)


def _key(clause: np.ndarray) -> tuple:
    return tuple(sorted(int(x) for x in clause))


def random_3sat(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct random 3-literal clauses over n variables, int32 [m, 3]."""
    if n < 3:
        raise ValueError("3-SAT needs n >= 3")
    if m < 0 or m > 8 * math.comb(n, 3):
        raise ValueError(f"cannot draw {m} distinct clauses over {n} variables")
    bg = _raw(seed, _STREAM_CLAUSES)
    lits = _draw_clauses(bg, n, m)
    seen: dict[tuple, int] = {}
    for i in range(m):
        while True:
            k = _key(lits[i])
            if k not in seen:
                seen[k] = i
                break
            lits[i] = _draw_clauses(bg, n, 1)[0]
    return lits


def random_angles(p: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """gamma_k, beta_k uniform in [0, pi), k = 1..p (float64 [p] each)."""
    u = _unit(_raw(seed, _STREAM_ANGLES), 2 * p)
    return np.pi * u[:p], np.pi * u[p:]


def protocol_grid(step_deg: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """The angle grid of the paper's protocol (Appendix C: spacing pi/180):
    gamma = i pi/180, i = 0..180, times beta = j pi/180, j = 0..359
    (gamma-major). The conjugation (gamma, beta) -> (2 pi - gamma, 2 pi - beta)
    leaves P and <H_P> unchanged, so gamma in [0, pi] covers the torus.
    step_deg > 1 thins both axes (for small tests)."""
    gi = np.arange(0, 181, step_deg) * (np.pi / 180)
    bj = np.arange(0, 360, step_deg) * (np.pi / 180)
    return np.repeat(gi, bj.size), np.tile(bj, gi.size)


def protocol_random_angles(count: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """count angle pairs uniform on [0, pi) x [0, 2 pi) (the protocol's sampled
    alternative to the grid above n = 20)."""
    u = _unit(_raw(seed, _STREAM_PROTOCOL), 2 * count)
    return np.pi * u[:count], 2 * np.pi * u[count:]


def synthetic_shots(n: int, count: int, seed: int, hot=None, hot_fraction: float = 0.0):
    """count measurement outcomes z in [0, 2^n) (uint64): uniform, except that
    a hot_fraction of them is drawn uniformly from the `hot` assignments
    (e.g. the solutions), so shot streams with many solution hits are cheap."""
    bg = _raw(seed, _STREAM_SHOTS)
    z = _below(bg, np.full(count, 1 << n)).astype(np.uint64)
    if hot is not None and hot_fraction > 0:
        hot = np.asarray(hot, dtype=np.uint64)
        u = _unit(bg, count)
        pick = _below(bg, np.full(count, hot.size))
        sel = u < hot_fraction
        z[sel] = hot[pick[sel]]
    return z


def sweep_shapes(count: int, seed: int, n_values=range(12, 21),
                 d_values=(3.0, 4.2, 5.0)) -> list[tuple[int, int, float]]:
    """(n, m, d) per instance of the batched sweep: n and d uniform over the sets."""
    n_values = list(n_values)
    d_values = list(d_values)
    bg = _raw(seed, _STREAM_SHAPE)
    ni = _below(bg, np.full(count, len(n_values)))
    di = _below(bg, np.full(count, len(d_values)))
    out = []
    for i in range(count):
        n = n_values[ni[i]]
        d = d_values[di[i]]
        out.append((n, clause_count(n, d), d))
    return out


def uniform_density_shapes(count: int, seed: int, n_values, d_lo: float, d_hi: float):
    """(n, m, d) per instance with n uniform over n_values and d uniform on [d_lo, d_hi]."""
    n_values = list(n_values)
    bg = _raw(seed, _STREAM_SHAPE)
    ni = _below(bg, np.full(count, len(n_values)))
    du = _unit(bg, count)
    out = []
    for i in range(count):
        n = n_values[ni[i]]
        d = d_lo + (d_hi - d_lo) * du[i]
        out.append((n, clause_count(n, d), d))
    return out


def random_state(n: int, seed: int) -> np.ndarray:
    """A normalised random complex128 state of 2^n amplitudes (Gaussian entries)."""
    u = _unit(_raw(seed, 3), 2 * (1 << n))
    # Box-Muller on pairs of uniforms.
    u1 = np.maximum(u[0::2], 1e-300)
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)
    return z / np.linalg.norm(z)


def mlp_dims(p: int = 16, d_in: int = 130, d_hidden: int = 256) -> tuple[int, int, int]:
    """(d_in, d_hidden, d_out) of the angle proposer: d_out = 2p (p gammas, p betas)."""
    return d_in, d_hidden, 2 * p


def mlp_param_count(d_in: int, d_h: int, d_out: int) -> int:
    return d_h * d_in + d_h + d_h * d_h + d_h + d_out * d_h + d_out


def random_mlp_params(d_in: int, d_h: int, d_out: int, seed: int) -> np.ndarray:
    """Flat float32 parameters [W1 (d_h x d_in), b1, W2 (d_h x d_h), b2, W3 (d_out x d_h), b3],
    weights uniform in +-sqrt(1/fan_in) (the usual fully-connected initialisation), biases 0."""
    bg = _raw(seed, 4)
    out = []
    for fan_out, fan_in in ((d_h, d_in), (d_h, d_h), (d_out, d_h)):
        lim = np.sqrt(1.0 / fan_in)
        w = (2.0 * _unit(bg, fan_out * fan_in) - 1.0) * lim
        out.append(w.astype(np.float32))
        out.append(np.zeros(fan_out, dtype=np.float32))
    return np.concatenate(out)
