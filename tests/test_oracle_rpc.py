"""Pins of the oracle's "random positive coefficient" pivot rule (RPC, Section 4.2).

* the counter-based generator against the published SplitMix64 outputs
  (tests/golden/splitmix64_seed0.json);
* statuses and optima under RPC against brute-force enumeration (a pivot rule changes
  the path, never the optimum or the status);
* the first entering variable is uniform over the eligible ones (chi-square);
* RPC takes more pivots than the most-negative rule on type-1 LPs (the paper's
  observation that LPC converges in fewer iterations, Section 5).
"""
import json
import os

import numpy as np

import oracle
import synth
from oracle import brute, certify

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_outputs():
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.json")) as f:
        g = json.load(f)
    assert oracle.splitmix64(g["state"], len(g["outputs_hex"])) == [int(h, 16) for h in g["outputs_hex"]]


def test_rpc_matches_brute_force_on_tiny_lps():
    rng = np.random.default_rng(11)
    seen = set()
    for k in range(300):
        m = int(rng.integers(1, 5)); n = int(rng.integers(1, 5))
        A = rng.integers(-3, 4, size=(m, n)).astype(float)
        b = rng.integers(-3, 6, size=m).astype(float)
        c = rng.integers(-2, 4, size=n).astype(float)
        st, ob, _ = brute.solve(A, b, c)
        r = oracle.solve_one(A, b, c, rule=oracle.RPC, seed=3, lp=k)
        seen.add(st)
        assert r["status"] == st, (A, b, c)
        if st == 0:
            assert abs(r["obj"] - ob) <= 1e-9 * (1 + abs(ob))
            assert certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)
    assert seen == {0, 1, 2}


def test_rpc_first_choice_is_uniform():
    """With c > 0 every structural is eligible at the first pivot; over many LP indices
    the variable that enters first must be uniform (chi-square, 7 degrees of freedom,
    p > 0.001), and the most-negative rule must not be what RPC picks."""
    n = 8
    A = np.full((1, n), 1.0)
    b = np.array([1.0])
    c = np.linspace(1.0, 2.0, n)          # LPC always takes the last column first
    counts = np.zeros(n)
    trials = 4000
    for k in range(trials):
        r = oracle.solve_one(A, b, c, max_iter=1, rule=oracle.RPC, seed=5, lp=k)
        assert r["status"] == oracle.ITER_LIMIT or r["status"] == oracle.OPTIMAL
        counts[r["basis"][0]] += 1
    chi2 = float(((counts - trials / n) ** 2 / (trials / n)).sum())
    assert chi2 < 24.3, counts
    lpc = oracle.solve_one(A, b, c, max_iter=1)
    assert lpc["basis"][0] == n - 1


def test_rpc_takes_more_pivots_than_lpc():
    sb = synth.type1(300, 40, 40, seed=9)
    lpc = oracle.solve_batch(sb)
    rpc = oracle.solve_batch(sb, rule=oracle.RPC, seed=1)
    assert np.array_equal(lpc["status"], rpc["status"]) and np.all(lpc["status"] == 0)
    np.testing.assert_allclose(rpc["obj"], lpc["obj"], rtol=1e-12)
    assert rpc["iters"].mean() > 1.3 * lpc["iters"].mean()


def test_rpc_depends_on_seed_and_lp_index_only():
    sb = synth.type1(40, 12, 12, seed=4)
    a = oracle.solve_batch(sb, rule=oracle.RPC, seed=2)
    b = oracle.solve_batch(sb.subset(np.arange(20, 40)), rule=oracle.RPC, seed=2, first_lp=20)
    assert np.array_equal(a["iters"][20:], b["iters"]) and np.array_equal(a["basis"][20 * 12:], b["basis"])
    c = oracle.solve_batch(sb, rule=oracle.RPC, seed=3)
    assert not np.array_equal(a["basis"], c["basis"])
