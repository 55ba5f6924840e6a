"""Index-by-index comparison of two shot streams drawn from the same state.

Both samplers invert the same cumulative distribution with the same
uniforms, so a shot can only differ where its target u_s * total lies within
the two CDFs' rounding of a boundary between amplitudes. `eps` bounds that
rounding (absolute, in units of the state's squared norm); every differing
shot must sit that close to each boundary between the two indices.
"""

import numpy as np

from oracle import statevector as sv


def compare_same_state(got, ref, cdf, seed: int, eps: float, label: str = ""):
    """got, ref: shot indices (GPU, oracle) for shots 0..len-1; cdf: the
    oracle's CDF of the state. Returns (differing shots, shots whose target
    lies within eps of a CDF boundary) and asserts that every differing shot
    is one of the latter."""
    got = np.asarray(got, dtype=np.int64)
    ref = np.asarray(ref, dtype=np.int64)
    assert got.shape == ref.shape
    assert got.min() >= 0 and got.max() < cdf.shape[0]
    total = cdf[-1]
    diff = np.flatnonzero(got != ref)
    u = np.array([sv.shot_uniform(seed, s) for s in range(len(ref))])
    t = u * total
    lo_edge = np.where(ref > 0, cdf[np.maximum(ref - 1, 0)], 0.0)
    near = int(np.sum((t - lo_edge <= eps) | (cdf[ref] - t <= eps)))
    for s in diff:
        a, b = sorted((int(got[s]), int(ref[s])))
        # every boundary cdf[a] .. cdf[b - 1] between the two picks is within eps
        assert abs(cdf[a] - t[s]) <= eps and abs(cdf[b - 1] - t[s]) <= eps, (
            label, int(s), int(got[s]), int(ref[s]), float(cdf[a] - t[s]), float(cdf[b - 1] - t[s]))
    print(f"{label}: {len(diff)} of {len(ref)} shots differ; {near} targets lie within "
          f"{eps:.1e} of a CDF boundary")
    return len(diff), near
