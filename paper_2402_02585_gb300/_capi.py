"""ctypes binding of libgqaoa.so: the C ABI of include/gqaoa.h, same names.

Arguments are plain integers (device or host addresses, sizes); every call
returns the C status and a nonzero status raises GQAOAError. No computation
happens here. If the library is missing the import of a function fails
loudly: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

GQAOA_OK = 0
GQAOA_EINVAL = -1
GQAOA_ERANGE = -2
GQAOA_ECUDA = -3
GQAOA_ETIMEOUT = -4
GQAOA_ENOMEM = -5
GQAOA_STATE_IN = 1
GQAOA_OBJ_P0 = 0
GQAOA_OBJ_ENERGY = 1
GQAOA_GRAD_STREAMING = 1 << 16  # OR-ed into a gradient objective: the streaming passes


def GQAOA_OBJ_CLASS(c: int) -> int:
    """Objective: the probability of cost value c (0..255)."""
    return 256 + (int(c) & 0xFF)


def GQAOA_READOUT_CLASS(c: int) -> int:
    """gqaoa_evolve flag: out[0] is the probability of cost value c."""
    return (int(c) & 0xFF) << 8

GQAOA_MAX_N = 34
GQAOA_MAX_M = 255
GQAOA_SWEEP_MIN_N = 9
GQAOA_SWEEP_MAX_N = 19
GQAOA_SWEEP_L2 = 1
GQAOA_SWEEP_L2_MIN_N = 20
GQAOA_SWEEP_L2_MAX_N = 24
GQAOA_NOALLOC_MAX_P = 256
GQAOA_NOALLOC_SCRATCH_BYTES = 1 << 20


class GQAOAError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_SZP = ctypes.POINTER(ctypes.c_size_t)
_U = ctypes.c_uint
_D = ctypes.c_double

# name -> argtypes (all return int status unless noted)
SIGNATURES = {
    "gqaoa_build_cost": [_P, _I, _I, _P, _P, _P],
    "gqaoa_evolve_workspace_size": [_I, _I, _SZP],
    "gqaoa_evolve": [_P, _I, _I, _P, _P, _I, _P, _P, _P, _P, _SZ, _U, _P],
    "gqaoa_evolve_batched_workspace_size": [_I, _I, _I, _SZP],
    "gqaoa_evolve_batched": [_P, _I64, _I, _I, _I, _P, _P, _I, _P, _P, _P, _P, _SZ, _U, _P],
    "gqaoa_prob_workspace_size": [_I, _SZP],
    "gqaoa_prob": [_P, _P, _I, _P, _P, _SZ, _P],
    "gqaoa_sample_workspace_size": [_I, _I64, _SZP],
    "gqaoa_sample": [_P, _I, _U64, _I64, _P, _P, _SZ, _P],
    "gqaoa_evolve_sample_workspace_size": [_I, _I, _I64, _SZP],
    "gqaoa_evolve_sample": [_P, _I, _I, _P, _P, _I, _P, _P, _P, _U64, _I64, _P, _P, _SZ, _U, _P],
    "gqaoa_grad_workspace_size": [_I, _I, _SZP],
    "gqaoa_grad": [_P, _I, _I, _P, _P, _I, _I, _P, _P, _P, _P, _SZ, _P],
    "gqaoa_grad_batched_workspace_size": [_I, _I, _I, _SZP],
    "gqaoa_grad_batched": [_P, _I64, _I, _I, _I, _P, _P, _I, _I, _P, _P, _P, _P, _SZ, _P],
    "gqaoa_batched_geometry": [_I, _I, _I, _P, _P],
    "gqaoa_evolve_noalloc": [_P, _I, _I, _P, _P, _I, _P, _P, _P, _U, _P],
    "gqaoa_sweep_workspace_size": [_I, _I, _I, _SZP],
    "gqaoa_reduced_sweep_workspace_size": [_I, _I, _I, _I, _SZP],
    "gqaoa_fairness_workspace_size": [_I, _I64, _I, _SZP],
    "gqaoa_fairness": [_P, _I64, _I64, _P, _I, _I, _I, _D, _I64, _P, _P, _P, _SZ, _P],
    "gqaoa_reduced_sweep": [_P, _I, _I, _I, _P, _P, _I, _I, _P, _P, _P, _SZ, _P],
    "gqaoa_sweep": [_P, _I, _I, _I, _P, _P, _I, _I, _P, _I, _I, _P, _P, _SZ, _P],
    "gqaoa_mlp_param_count": [_I, _I, _I, _SZP],
    "gqaoa_mlp_workspace_size": [_I, _I, _I, _I, _SZP],
    "gqaoa_mlp_forward": [_P, _I, _I, _I, _P, _I, _P, _P, _SZ, _P],
    "gqaoa_mlp_backward": [_P, _I, _I, _I, _P, _P, _I, _P, _P, _P, _SZ, _P],
    "gqaoa_mlp_features": [_P, _I, _P, _P, _I, _I, _P, _P],
    "gqaoa_adam_f32": [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I, _D, _P],
    "gqaoa_adam_f64": [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I, _D, _P],
    "gqaoa_version": [],
    "gqaoa_strerror": [_I],
}


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgqaoa.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing; run paper_2402_02585_gb300.build")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, argtypes in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = argtypes
            fn.restype = ctypes.c_char_p if name == "gqaoa_strerror" else ctypes.c_int
        _lib = lib
        return lib


def strerror(status: int) -> str:
    return load().gqaoa_strerror(int(status)).decode()


def _call(name: str, *args) -> None:
    lib = _lib if _lib is not None else load()  # no lock once loaded
    rc = getattr(lib, name)(*args)
    if rc != GQAOA_OK:
        raise GQAOAError(name, rc, strerror(rc))


def _size(name: str, *args) -> int:
    out = ctypes.c_size_t(0)
    _call(name, *args, ctypes.byref(out))
    return int(out.value)


def gqaoa_version() -> int:
    return int(load().gqaoa_version())


def gqaoa_build_cost(lits, n, m, cost, hist, stream):
    _call("gqaoa_build_cost", lits, n, m, cost, hist, stream)


def gqaoa_evolve_workspace_size(n, p) -> int:
    return _size("gqaoa_evolve_workspace_size", n, p)


def gqaoa_evolve(cost, n, m, gammas, betas, p, state, out, trace, ws, ws_bytes, flags, stream):
    _call("gqaoa_evolve", cost, n, m, gammas, betas, p, state, out, trace, ws, ws_bytes, flags,
          stream)


def gqaoa_evolve_batched_workspace_size(n, batch, p) -> int:
    return _size("gqaoa_evolve_batched_workspace_size", n, batch, p)


def gqaoa_evolve_batched(cost, cost_stride, n, m, batch, gammas, betas, p, state, out, trace, ws,
                         ws_bytes, flags, stream):
    _call("gqaoa_evolve_batched", cost, cost_stride, n, m, batch, gammas, betas, p, state, out,
          trace, ws, ws_bytes, flags, stream)


def gqaoa_prob_workspace_size(n) -> int:
    return _size("gqaoa_prob_workspace_size", n)


def gqaoa_prob(state, cost, n, out, ws, ws_bytes, stream):
    _call("gqaoa_prob", state, cost, n, out, ws, ws_bytes, stream)


def gqaoa_sample_workspace_size(n, shots) -> int:
    return _size("gqaoa_sample_workspace_size", n, shots)


def gqaoa_sample(state, n, seed, shots, out_idx, ws, ws_bytes, stream):
    _call("gqaoa_sample", state, n, seed, shots, out_idx, ws, ws_bytes, stream)


def gqaoa_evolve_sample_workspace_size(n, p, shots) -> int:
    return _size("gqaoa_evolve_sample_workspace_size", n, p, shots)


def gqaoa_evolve_sample(cost, n, m, gammas, betas, p, state, out, trace, seed, shots, out_idx, ws,
                        ws_bytes, flags, stream):
    _call("gqaoa_evolve_sample", cost, n, m, gammas, betas, p, state, out, trace, seed, shots,
          out_idx, ws, ws_bytes, flags, stream)


def gqaoa_grad_workspace_size(n, p) -> int:
    return _size("gqaoa_grad_workspace_size", n, p)


def gqaoa_grad(cost, n, m, gammas, betas, p, objective, value, dgamma, dbeta, ws, ws_bytes, stream):
    _call("gqaoa_grad", cost, n, m, gammas, betas, p, objective, value, dgamma, dbeta, ws, ws_bytes,
          stream)


def gqaoa_grad_batched_workspace_size(n, batch, p) -> int:
    return _size("gqaoa_grad_batched_workspace_size", n, batch, p)


def gqaoa_grad_batched(cost, cost_stride, n, m, batch, gammas, betas, p, objective, value, dgamma,
                       dbeta, ws, ws_bytes, stream):
    _call("gqaoa_grad_batched", cost, cost_stride, n, m, batch, gammas, betas, p, objective, value,
          dgamma, dbeta, ws, ws_bytes, stream)


def gqaoa_sweep_workspace_size(n, angles, amps_per_thread=0) -> int:
    return _size("gqaoa_sweep_workspace_size", n, angles, amps_per_thread)


def gqaoa_sweep(cost, n, m, batch, gammas, betas, angles, p, rounds, nrounds, amps_per_thread,
                out, ws, ws_bytes, stream):
    _call("gqaoa_sweep", cost, n, m, batch, gammas, betas, angles, p, rounds, nrounds,
          amps_per_thread, out, ws, ws_bytes, stream)


def gqaoa_reduced_sweep_workspace_size(hist_stride, batch, angles, p) -> int:
    return _size("gqaoa_reduced_sweep_workspace_size", hist_stride, batch, angles, p)


def gqaoa_reduced_sweep(hist, hist_stride, n, batch, gammas, betas, angles, p, out, best, ws,
                        ws_bytes, stream):
    _call("gqaoa_reduced_sweep", hist, hist_stride, n, batch, gammas, betas, angles, p, out, best,
          ws, ws_bytes, stream)


def gqaoa_fairness_workspace_size(n, runs, targets) -> int:
    return _size("gqaoa_fairness_workspace_size", n, runs, targets)


def gqaoa_fairness(shots, runs, shots_per_run, cost, n, target, targets, chi2_crit, min_draws,
                   to_all, to_reject, ws, ws_bytes, stream):
    _call("gqaoa_fairness", shots, runs, shots_per_run, cost, n, target, targets, chi2_crit,
          min_draws, to_all, to_reject, ws, ws_bytes, stream)


def gqaoa_mlp_param_count(d_in, d_h, d_out) -> int:
    return _size("gqaoa_mlp_param_count", d_in, d_h, d_out)


def gqaoa_mlp_workspace_size(batch, d_in, d_h, d_out) -> int:
    return _size("gqaoa_mlp_workspace_size", batch, d_in, d_h, d_out)


def gqaoa_mlp_forward(params, d_in, d_h, d_out, x, batch, angles, ws, ws_bytes, stream):
    _call("gqaoa_mlp_forward", params, d_in, d_h, d_out, x, batch, angles, ws, ws_bytes, stream)


def gqaoa_mlp_backward(params, d_in, d_h, d_out, x, labels, batch, grads, loss, ws, ws_bytes,
                       stream):
    _call("gqaoa_mlp_backward", params, d_in, d_h, d_out, x, labels, batch, grads, loss, ws,
          ws_bytes, stream)


def gqaoa_mlp_features(hist, hist_stride, ns, ms, batch, d_in, x, stream):
    _call("gqaoa_mlp_features", hist, hist_stride, ns, ms, batch, d_in, x, stream)


def gqaoa_adam_f32(params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale, stream):
    _call("gqaoa_adam_f32", params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale,
          stream)


def gqaoa_adam_f64(params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale, stream):
    _call("gqaoa_adam_f64", params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale,
          stream)


def gqaoa_evolve_noalloc(cost, n, m, gammas, betas, p, state, out, trace, flags, stream):
    """gqaoa_evolve with the library's fixed static scratch instead of a
    caller workspace (for callers that cannot allocate device memory)."""
    _call("gqaoa_evolve_noalloc", cost, n, m, gammas, betas, p, state, out, trace, flags, stream)


def gqaoa_batched_geometry(n, batch, adjoint) -> tuple[int, int]:
    """(CTAs per instance, reduction records per instance) of the batched
    streaming passes (adjoint: the gradient's backward rounds)."""
    cpi = ctypes.c_int(0)
    rec = ctypes.c_int(0)
    _call("gqaoa_batched_geometry", n, batch, int(bool(adjoint)), ctypes.byref(cpi),
          ctypes.byref(rec))
    return int(cpi.value), int(rec.value)
