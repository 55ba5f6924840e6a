"""Full-statevector FP64 oracle: ctypes wrapper of gqaoa_oracle.c.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

The C file is compiled here with gcc (-O2 -fopenmp) into oracle/_build/ on
first use; `build()` does it eagerly.

Functions and what pins them (tests/test_oracle_*.py):
  cost_table    brute-force Python loop of Appendix B's rule; sum h = 2^n;
                sum c h[c] = m 2^{n-3}; Section IV footnote instances.
  evolve        p=1 closed form; Grover's textbook sin^2((2k+1)theta) at
                gamma = beta = pi (Appendix A); gamma = 0 or beta = 0 leave
                P = h[0]/2^n; norm conservation; a dense-matrix brute force
                (expm of H_M and H_P) at tiny n; Table I noiseless values.
  readout       brute force; the uniform state gives P = h[0]/2^n and
                <H> = m/8.
  sample        numpy.searchsorted on the same CDF; chi-square goodness of fit.
  philox        published known-answer vectors of Philox4x32-10.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gqaoa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gqaoa_oracle.c into a shared library (plain gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_cost_at.argtypes = [P, ctypes.c_int, ctypes.c_uint64]
            lib.oracle_cost_at.restype = ctypes.c_int
            lib.oracle_cost_table.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
            lib.oracle_cost_table.restype = ctypes.c_int
            lib.oracle_plus_state.argtypes = [ctypes.c_int, P]
            lib.oracle_apply_phase.argtypes = [P, ctypes.c_int, ctypes.c_double, P]
            lib.oracle_apply_mixer.argtypes = [ctypes.c_int, ctypes.c_double, P]
            lib.oracle_readout.argtypes = [P, P, ctypes.c_int, P]
            lib.oracle_evolve.argtypes = [P, ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int, P]
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_shot_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_shot_uniform.restype = ctypes.c_double
            lib.oracle_sample.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, P, P]
            lib.oracle_sample.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def cost_at(lits: np.ndarray, z: int) -> int:
    lits = np.ascontiguousarray(lits, dtype=np.int32)
    return int(_load().oracle_cost_at(_ptr(lits), lits.shape[0], int(z)))


def cost_table(lits: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """C(z) (uint8 [2^n]) and h[c] (uint64 [m+1])."""
    lits = np.ascontiguousarray(lits, dtype=np.int32).reshape(-1, 3)
    m = lits.shape[0]
    cost = np.empty(1 << n, dtype=np.uint8)
    hist = np.zeros(m + 1, dtype=np.uint64)
    rc = _load().oracle_cost_table(_ptr(lits), n, m, _ptr(cost), _ptr(hist))
    if rc != 0:
        raise ValueError("oracle_cost_table: bad instance")
    return cost, hist


def histogram(lits: np.ndarray, n: int) -> np.ndarray:
    """h[c] only (the cost table is not kept)."""
    lits = np.ascontiguousarray(lits, dtype=np.int32).reshape(-1, 3)
    m = lits.shape[0]
    hist = np.zeros(m + 1, dtype=np.uint64)
    rc = _load().oracle_cost_table(_ptr(lits), n, m, None, _ptr(hist))
    if rc != 0:
        raise ValueError("oracle_cost_table: bad instance")
    return hist


def plus_state(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().oracle_plus_state(n, _ptr(psi))
    return psi


def evolve(cost: np.ndarray, n: int, gammas, betas, psi0: np.ndarray | None = None,
           trace: bool = False):
    """psi_p of Eq. 3 (complex128 [2^n]); with trace=True also P after each round."""
    gammas = np.ascontiguousarray(gammas, dtype=np.float64)
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    p = gammas.shape[0]
    assert betas.shape[0] == p
    cost = np.ascontiguousarray(cost, dtype=np.uint8)
    if psi0 is None:
        psi = np.empty(1 << n, dtype=np.complex128)
        from_plus = 1
    else:
        psi = np.array(psi0, dtype=np.complex128, copy=True)
        from_plus = 0
    tr = np.zeros(p, dtype=np.float64) if trace else None
    _load().oracle_evolve(_ptr(cost), n, _ptr(gammas), _ptr(betas), p, _ptr(psi), from_plus,
                          _ptr(tr))
    return (psi, tr) if trace else psi


def apply_phase(cost, n, gamma, psi):
    _load().oracle_apply_phase(_ptr(cost), n, float(gamma), _ptr(psi))


def apply_mixer(n, beta, psi):
    _load().oracle_apply_mixer(n, float(beta), _ptr(psi))


def readout(psi: np.ndarray, cost: np.ndarray, n: int) -> np.ndarray:
    """[P(C=0), <H_P>, norm] of a state."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    cost = np.ascontiguousarray(cost, dtype=np.uint8)
    out = np.zeros(3, dtype=np.float64)
    _load().oracle_readout(_ptr(psi), _ptr(cost), n, _ptr(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def shot_uniform(seed: int, shot: int) -> float:
    return float(_load().oracle_shot_uniform(int(seed), int(shot)))


def sample(psi: np.ndarray, n: int, seed: int, shots: int, return_cdf: bool = False):
    """uint32 [shots]: shot s = smallest z with CDF(z) > u_s * CDF(N-1)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(shots, dtype=np.uint32)
    cdf = np.empty(1 << n, dtype=np.float64) if return_cdf else None
    rc = _load().oracle_sample(_ptr(psi), n, int(seed), int(shots), _ptr(out), _ptr(cdf))
    if rc != 0:
        raise ValueError("oracle_sample: zero-norm state")
    return (out, cdf) if return_cdf else out
