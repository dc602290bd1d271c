"""Pins of the oracle's steepest-edge pricing (entering column maximizing r_j^2 / gamma_j with
gamma_j = 1 + sum_i t_ij^2; not in the paper, which compares only LPC and RPC in Section 4.2).

* a one-row LP worked by hand (tests/golden/steepest_edge_one_row.json) where the two rules
  take different first columns and different pivot counts;
* the entering variable of every pivot maximizes r_j^2 / gamma_j over the eligible columns,
  with the tableau of each intermediate basis rebuilt independently here (numpy solve of
  B^{-1} [A | I] and c_B^T B^{-1} [A | I] - [c | 0]);
* statuses and optima under the rule against brute-force vertex enumeration (a pricing rule
  changes the path, never the optimum or the status), one- and two-phase;
* fewer pivots than the largest-coefficient rule on type-1 LPs, as steepest edge is known for.
"""
import json
import os

import numpy as np

import oracle
import synth
from oracle import brute, certify

HERE = os.path.dirname(os.path.abspath(__file__))


def test_steepest_edge_worked_example():
    with open(os.path.join(HERE, "golden", "steepest_edge_one_row.json")) as f:
        g = json.load(f)
    A, b, c = (np.array(g[k], dtype=float) for k in ("A", "b", "c"))
    lpc = oracle.solve_one(A, b, c)
    se = oracle.solve_one(A, b, c, rule=oracle.SE)
    assert lpc["iters"] == g["pivots_largest_coefficient"]
    assert se["iters"] == g["pivots_steepest_edge"]
    for r in (lpc, se):
        assert r["status"] == oracle.OPTIMAL
        assert abs(r["obj"] - g["optimum"]) <= 1e-12 * g["optimum"]
        assert np.allclose(r["x"], g["x"], rtol=1e-12, atol=1e-12)
        assert np.allclose(r["y"], g["y"], rtol=1e-12, atol=1e-12)
    # The first entering column under each rule.
    first_lpc = oracle.solve_one(A, b, c, max_iter=1)
    first_se = oracle.solve_one(A, b, c, max_iter=1, rule=oracle.SE)
    assert first_lpc["basis"][0] == 0 and first_se["basis"][0] == 1


def _tableau(A, b, c, basis):
    """B^{-1} [A | I], B^{-1} b and the reduced costs of every variable for a basis given as
    variable indices (0..n-1 structurals, n..n+m-1 slacks)."""
    m, n = A.shape
    full = np.hstack([A, np.eye(m)])
    cf = np.concatenate([c, np.zeros(m)])
    B = full[:, basis]
    T = np.linalg.solve(B, full)
    r = cf[basis] @ T - cf
    return T, np.linalg.solve(B, b), r


def test_each_entering_column_maximizes_the_score():
    rng = np.random.default_rng(31)
    checked = 0
    for trial in range(25):
        m, n = int(rng.integers(3, 8)), int(rng.integers(3, 8))
        A = rng.uniform(0.1, 1.0, (m, n))
        b = rng.uniform(1.0, 10.0, m)
        c = rng.uniform(0.0, 1.0, n)
        full = oracle.solve_one(A, b, c, rule=oracle.SE)
        assert full["status"] == oracle.OPTIMAL
        prev = list(range(n, n + m))               # the slack basis
        for k in range(1, full["iters"] + 1):
            cur = oracle.solve_one(A, b, c, max_iter=k, rule=oracle.SE)["basis"].tolist()
            entered = [v for v in cur if v not in prev]
            assert len(entered) == 1
            T, _, r = _tableau(A, b, c, prev)
            nonbasic = [j for j in range(n + m) if j not in prev]
            elig = [j for j in nonbasic if r[j] < -oracle.EPS_D]
            score = {j: r[j] ** 2 / (1.0 + np.sum(T[:, j] ** 2)) for j in elig}
            best = max(score.values())
            assert score[entered[0]] >= best * (1 - 1e-9), (trial, k, score, entered)
            ranked = sorted(score.values())          # where the best is clear, it is the only choice
            if len(ranked) == 1 or ranked[-2] < best * (1 - 1e-6):
                assert entered[0] == max(score, key=score.get)
            prev = cur
            checked += 1
    assert checked > 40


def test_steepest_edge_matches_brute_force_on_tiny_lps():
    rng = np.random.default_rng(12)
    seen = set()
    for k in range(300):
        m = int(rng.integers(1, 5)); n = int(rng.integers(1, 5))
        A = rng.integers(-3, 4, size=(m, n)).astype(float)
        b = rng.integers(-3, 6, size=m).astype(float)
        c = rng.integers(-2, 4, size=n).astype(float)
        st, ob, _ = brute.solve(A, b, c)
        r = oracle.solve_one(A, b, c, rule=oracle.SE)
        seen.add(st)
        assert r["status"] == st, (A, b, c)
        if st == 0:
            assert abs(r["obj"] - ob) <= 1e-9 * (1 + abs(ob))
            assert certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)
    assert seen == {0, 1, 2}


def test_steepest_edge_takes_fewer_pivots_than_lpc():
    sb = synth.type1(300, 40, 40, seed=9)
    lpc = oracle.solve_batch(sb)
    se = oracle.solve_batch(sb, rule=oracle.SE)
    assert (se["status"] == 0).all() and (lpc["status"] == 0).all()
    assert np.max(np.abs(se["obj"] - lpc["obj"]) / (1 + np.abs(lpc["obj"]))) <= 1e-12
    assert se["iters"].mean() < 0.95 * lpc["iters"].mean()


def test_steepest_edge_two_phase_statuses():
    sb = synth.type2(120, 24, 20, seed=4, frac_infeasible=0.1, frac_unbounded=0.1)
    lpc = oracle.solve_batch(sb)
    se = oracle.solve_batch(sb, rule=oracle.SE)
    assert (se["status"] == lpc["status"]).all()
    assert set(np.unique(se["status"])) == {0, 1, 2}
    ok = lpc["status"] == 0
    assert np.max(np.abs(se["obj"][ok] - lpc["obj"][ok]) / (1 + np.abs(lpc["obj"][ok]))) <= 1e-9
