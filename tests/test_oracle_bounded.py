"""Pins of the oracle's bounded-variable LPs (max c^T x, A x <= b, l <= x <= u): the change of
variables x = l + z against direct vertex enumeration of the bounded polytope (finite bounds)
and against scipy's HiGHS (finite and infinite upper bounds)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import brute


def _pack(lps):
    return synth.pack([(A, b, c) for A, b, c, _, _ in lps])


def _bounds(lps):
    return (np.concatenate([l for *_, l, _ in lps]), np.concatenate([u for *_, _, u in lps]))


def test_bounded_matches_vertex_enumeration():
    rng = np.random.default_rng(21)
    lps = []
    for _ in range(150):
        m = int(rng.integers(1, 4)); n = int(rng.integers(1, 4))
        A = rng.normal(size=(m, n)); b = rng.normal(size=m) + 0.5; c = rng.normal(size=n)
        l = rng.uniform(-2, 0.5, size=n); u = l + rng.uniform(-0.2, 3, size=n)     # some empty boxes
        lps.append((A, b, c, l, u))
    sb = _pack(lps)
    l, u = _bounds(lps)
    r = oracle.solve_bounded_batch(sb, l, u)
    seen = set()
    for k, (A, b, c, lk, uk) in enumerate(lps):
        st, ob, _ = brute.solve_box(A, b, c, lk, uk)
        seen.add(st)
        assert r["status"][k] == st, k
        if st == 0:
            assert abs(r["obj"][k] - ob) <= 1e-9 * (1 + abs(ob))
            x = r["x"][sb.c_off[k]:sb.c_off[k] + len(c)]
            assert np.all(x >= lk - 1e-9) and np.all(x <= uk + 1e-9) and np.all(A @ x <= b + 1e-9)
            assert abs(float(c @ x) - ob) <= 1e-9 * (1 + abs(ob))
    assert seen == {0, 1}


def test_bounded_matches_highs():
    sp = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(22)
    lps = []
    for k in range(60):
        m, n = 12, 10
        A = rng.uniform(-1, 1, size=(m, n)); b = rng.uniform(0.5, 5, size=m); c = rng.normal(size=n)
        l = rng.uniform(-3, 0, size=n); u = l + rng.uniform(0.5, 4, size=n)
        if k % 3 == 0:
            u[rng.integers(0, n)] = np.inf
        lps.append((A, b, c, l, u))
    sb = _pack(lps)
    l, u = _bounds(lps)
    r = oracle.solve_bounded_batch(sb, l, u)
    for k, (A, b, c, lk, uk) in enumerate(lps):
        h = sp.linprog(-c, A_ub=A, b_ub=b, bounds=list(zip(lk, [None if np.isinf(v) else v for v in uk])),
                       method="highs")
        want = {0: 0, 2: 1, 3: 2}[h.status]
        assert r["status"][k] == want, k
        if want == 0:
            assert abs(r["obj"][k] + h.fun) <= 1e-8 * (1 + abs(h.fun))
