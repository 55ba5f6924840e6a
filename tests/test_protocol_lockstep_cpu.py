"""The protocol's lockstep drivers (host logic, no GPU): several L-BFGS-B
searches whose evaluation requests are served in waves must end exactly where
the same searches run one by one by scipy.optimize.minimize end, and every
wave must hold one request from each search still running. Two drivers: the
reverse-communication one (_Lbfgsb, all searches stepped from one thread) and
the threaded one (_Lockstep, one host thread per search), its fallback."""

import threading

import numpy as np
import scipy.optimize

from paper_2402_02585_gb300.protocol import _Lbfgsb, _Lockstep, lbfgsb_matches_scipy


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


def _fun_n(k, x):
    # a coupled, rugged landscape in len(x) variables (the all-angles search)
    n = x.size
    c = np.linspace(-0.5, 0.5, n) + 0.05 * k
    w = 1.0 + np.arange(n) / n
    v = float(np.sum(w * (x - c) ** 2) + 0.2 * np.sum(np.sin(3.0 * x) * np.cos(x[::-1])))
    g = 2.0 * w * (x - c) + 0.2 * (3.0 * np.cos(3.0 * x) * np.cos(x[::-1])
                                   - (np.sin(3.0 * x) * np.sin(x[::-1]))[::-1])
    return v, g


def test_reverse_communication_equals_minimize():
    assert lbfgsb_matches_scipy()
    cases = [(k, _fun, np.array([0.1 * k, 1.0 - 0.05 * k])) for k in range(1, 9)]
    cases += [(k, _fun_n, np.full(2 * k, 0.3)) for k in (2, 5, 11)]
    searches = {}
    for k, f, x0 in cases:
        searches[(k, f.__name__)] = (_Lbfgsb(x0, 1e-6, 1e-10, 500), f, x0)
    waves = []
    while True:
        wave = {key: s.point() for key, (s, _, _) in searches.items() if s.point() is not None}
        if not wave:
            break
        waves.append(sorted(wave))
        for key, x in wave.items():
            s, f, _ = searches[key]
            s.tell(*f(key[0], x))
    for key, (s, f, x0) in searches.items():
        r = _minimize(lambda x: f(key[0], x), x0)
        assert np.array_equal(s.x, r.x) and s.f == r.fun, key
        assert s.nfev == r.nfev and s.nit == r.nit and s.converged == r.success, key
    # wave w holds exactly the searches that needed more than w evaluations
    for w, wave in enumerate(waves):
        assert wave == sorted(key for key, (s, _, _) in searches.items() if s.nfev > w)


def test_reverse_communication_iteration_limit():
    # maxiter stops the search where minimize stops it
    x0 = np.full(6, 0.3)
    s = _Lbfgsb(x0, 1e-12, 1e-14, 3)
    while s.point() is not None:
        s.tell(*_fun_n(1, s.point()))
    r = scipy.optimize.minimize(lambda x: _fun_n(1, x), x0, jac=True, method="L-BFGS-B",
                                options=dict(ftol=1e-12, gtol=1e-14, maxiter=3))
    assert s.nit == r.nit == 3 and np.array_equal(s.x, r.x) and not s.converged
