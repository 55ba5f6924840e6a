"""Host logic of the protocol's batched depth windows (pad_depth_rows,
depth_row_results): depth k's angles in the last k rounds of a P-round row,
the leading P - k rounds identity (gamma = beta = 0: phase factor 1, mixer
term 0). Pinned with the oracle's cost-class adjoint: a padded row has the
unpadded circuit's objective, and its derivatives over the last k rounds are
the unpadded circuit's derivatives."""

import numpy as np

from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import instances
from paper_2402_02585_gb300.protocol import depth_row_results, pad_depth_rows


def _rows():
    rng = np.random.default_rng(3)
    return [(3, rng.uniform(0, 3, 3), rng.uniform(0, 3, 3)), (1, 0.7, 1.9),
            (5, rng.uniform(0, 3, 5), rng.uniform(0, 3, 5)), (2, 2.2, 0.4)]


def test_padding_layout():
    rows = _rows()
    buf = np.full(2 * 8 * 8, np.nan)
    P = pad_depth_rows(buf, rows)
    assert P == 5
    a = buf[:2 * len(rows) * P].reshape(2, len(rows), P)
    for i, (k, g, b) in enumerate(rows):
        assert np.all(a[:, i, :P - k] == 0.0)
        assert np.array_equal(a[0, i, P - k:], np.broadcast_to(g, (k,)))
        assert np.array_equal(a[1, i, P - k:], np.broadcast_to(b, (k,)))
    assert np.all(np.isnan(buf[2 * len(rows) * P:]))  # nothing written past the block


def test_padded_rows_are_the_unpadded_circuits():
    n, m = 8, 34
    hist = sv.histogram(instances.random_3sat(n, m, 11), n)
    rows = _rows()
    buf = np.zeros(2 * len(rows) * 5)
    P = pad_depth_rows(buf, rows)
    a = buf[:2 * len(rows) * P].reshape(2, len(rows), P)
    B = len(rows)
    out = np.zeros(B + 2 * B * P)
    direct = []
    for i, (k, g, b) in enumerate(rows):
        L, dg, db = reduced.grad(hist, a[0, i], a[1, i], reduced.OBJ_ENERGY)
        out[i] = L
        out[B + i * P:B + (i + 1) * P] = dg
        out[B + B * P + i * P:B + B * P + (i + 1) * P] = db
        direct.append(reduced.grad(hist, np.broadcast_to(g, (k,)).copy(),
                                   np.broadcast_to(b, (k,)).copy(), reduced.OBJ_ENERGY))
    per_round = depth_row_results(out, rows, P, single=False)
    summed = depth_row_results(out, rows, P, single=True)
    for (k, _, _), (L0, dg0, db0), (L, dg, db), (Ls, sg, sb) in zip(rows, direct, per_round, summed):
        assert abs(L - L0) < 1e-12 * m and Ls == L
        assert np.allclose(dg, dg0, atol=1e-12 * m) and np.allclose(db, db0, atol=1e-12 * m)
        assert len(dg) == k and sg == float(np.sum(dg)) and sb == float(np.sum(db))
