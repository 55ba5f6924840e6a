"""The protocol's lockstep driver (host logic, no GPU): several L-BFGS-B
searches on host threads whose evaluation requests are served in waves must
end exactly where the same searches run one by one end, and every wave must
hold one request from each search still running."""

import threading

import numpy as np
import scipy.optimize

from paper_2402_02585_gb300.protocol import _Lockstep


def _fun(k, x):
    # a smooth, slightly rugged landscape per search k
    v = (x[0] - 0.3 * k) ** 2 + 3.0 * (x[1] + 0.1 * k) ** 2 + 0.1 * np.sin(5.0 * x[0] + k)
    g = np.array([2.0 * (x[0] - 0.3 * k) + 0.5 * np.cos(5.0 * x[0] + k), 6.0 * (x[1] + 0.1 * k)])
    return v, g


def _minimize(f, x0):
    return scipy.optimize.minimize(f, x0, jac=True, method="L-BFGS-B",
                                   options=dict(ftol=1e-6, gtol=1e-10, maxiter=500))


def test_lockstep_equals_independent_searches():
    ks = list(range(1, 9))
    x0 = {k: np.array([0.1 * k, 1.0 - 0.05 * k]) for k in ks}
    alone = {k: _minimize(lambda x, k=k: _fun(k, x), x0[k]) for k in ks}

    steps = _Lockstep(ks)
    waves, got = [], {}

    def search(k):
        try:
            got[k] = _minimize(lambda x: steps.request(k, x), x0[k])
        finally:
            steps.finished()

    def evaluate(batch):
        waves.append(sorted(batch))
        return {k: _fun(k, x) for k, x in batch.items()}

    threads = [threading.Thread(target=search, args=(k,)) for k in ks]
    for t in threads:
        t.start()
    steps.serve(evaluate)
    for t in threads:
        t.join()
    for k in ks:
        assert np.array_equal(got[k].x, alone[k].x) and got[k].fun == alone[k].fun
        assert got[k].nfev == alone[k].nfev
    # wave w holds exactly the searches that needed more than w evaluations
    for w, wave in enumerate(waves):
        assert wave == [k for k in ks if alone[k].nfev > w]
    assert len(waves) == max(alone[k].nfev for k in ks)


def test_lockstep_error_reaches_the_searches():
    steps = _Lockstep([0, 1])
    seen = []

    def search(k):
        try:
            steps.request(k, np.zeros(2))
        except RuntimeError as exc:
            seen.append(exc)
        finally:
            steps.finished()

    def evaluate(batch):
        raise ValueError("evaluation failed")

    threads = [threading.Thread(target=search, args=(k,)) for k in (0, 1)]
    for t in threads:
        t.start()
    try:
        steps.serve(evaluate)
    except ValueError:
        pass
    for t in threads:
        t.join(timeout=10)
    assert len(seen) == 2 and all(isinstance(e.__cause__, ValueError) for e in seen)
