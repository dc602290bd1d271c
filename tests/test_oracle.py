"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-derived LPs (tests/golden/handworked_lps.json, every vertex listed);
* brute-force vertex / extreme-ray enumeration on tiny LPs (all statuses);
* LP duality certificates: KKT + strong duality for optimal results, Farkas
  vectors for infeasible ones, rays for unbounded ones;
* duals and primal values recomputed from the final basis by a linear solve;
* an independent LP solver (scipy's HiGHS) on moderate sizes;
* the type-1 fact that A > 0, b > 0 makes every LP bounded and optimal;
* Beale's classic cycling example (terminates at the enumerated optimum).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute, certify

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    with open(os.path.join(HERE, "golden", "handworked_lps.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_handworked(case):
    A = np.array(case["A"], dtype=float)
    r = oracle.solve_one(A, case["b"], case["c"])
    assert r["status"] == case["status"]
    if case["status"] == 0:
        assert abs(r["obj"] - case["obj"]) <= 1e-12 * (1 + abs(case["obj"]))
        if "x" in case:
            np.testing.assert_allclose(r["x"], case["x"], atol=1e-12)
        if "y" in case:
            np.testing.assert_allclose(r["y"], case["y"], atol=1e-12)
        assert certify.is_optimal_pair(A, case["b"], case["c"], r["x"], r["y"], tol=1e-12)
    elif case["status"] == 1:
        assert certify.is_farkas(A, case["b"], r["cert"][:A.shape[0]])
    elif case["status"] == 2:
        assert certify.is_ray(A, case["c"], r["cert"][:A.shape[1]])


def _tiny_lps(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        m = int(rng.integers(1, 5)); n = int(rng.integers(1, 5))
        A = rng.integers(-3, 4, size=(m, n)).astype(float)
        b = rng.integers(-3, 6, size=m).astype(float)
        c = rng.integers(-2, 4, size=n).astype(float)
        yield A, b, c


def test_brute_force_tiny_integer_lps():
    """Integer data gives many ties and degenerate vertices; statuses and optima must
    match exhaustive enumeration."""
    seen = set()
    for A, b, c in _tiny_lps(1, 400):
        st, ob, _ = brute.solve(A, b, c)
        r = oracle.solve_one(A, b, c)
        seen.add(st)
        assert r["status"] == st, (A, b, c)
        if st == 0:
            assert abs(r["obj"] - ob) <= 1e-9 * (1 + abs(ob))
            assert certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)
    assert seen == {0, 1, 2}


def test_brute_force_tiny_continuous_lps():
    rng = np.random.default_rng(7)
    for _ in range(150):
        m = int(rng.integers(1, 6)); n = int(rng.integers(1, 6))
        A = rng.normal(size=(m, n)); b = rng.normal(size=m) + 0.5; c = rng.normal(size=n)
        st, ob, _ = brute.solve(A, b, c)
        r = oracle.solve_one(A, b, c)
        assert r["status"] == st
        if st == 0:
            assert abs(r["obj"] - ob) <= 1e-9 * (1 + abs(ob))


def test_certificates_of_every_status():
    for A, b, c in _tiny_lps(3, 300):
        m, n = A.shape
        r = oracle.solve_one(A, b, c)
        if r["status"] == 0:
            assert certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)
        elif r["status"] == 1:
            assert certify.is_farkas(A, b, r["cert"][:m])
        elif r["status"] == 2:
            assert certify.is_ray(A, c, r["cert"][:n])


def test_type1_always_optimal_and_kkt():
    """A > 0 and b > 0 bound every LP and make the origin feasible, so all are optimal."""
    bt = synth.type1(64, 16, 16, seed=0)
    r = oracle.solve_batch(bt)
    assert np.all(r["status"] == 0)
    for k in range(bt.count):
        A, b, c = bt.lp(k)
        x = r["x"][bt.c_off[k]:bt.c_off[k] + 16]
        y = r["y"][bt.b_off[k]:bt.b_off[k] + 16]
        assert certify.is_optimal_pair(A, b, c, x, y, tol=1e-10)
        assert abs(r["obj"][k] - c @ x) <= 1e-12 * (1 + abs(r["obj"][k]))


def test_duals_and_primal_match_basis_solves():
    bt = synth.type1(16, 30, 24, seed=11)
    r = oracle.solve_batch(bt)
    for k in range(bt.count):
        A, b, c = bt.lp(k)
        basis = r["basis"][bt.b_off[k]:bt.b_off[k] + 30]
        y = r["y"][bt.b_off[k]:bt.b_off[k] + 30]
        x = r["x"][bt.c_off[k]:bt.c_off[k] + 24]
        np.testing.assert_allclose(y, certify.duals_from_basis(A, c, basis), atol=1e-10)
        np.testing.assert_allclose(x, certify.primal_from_basis(A, b, basis), atol=1e-10)


def test_type2_statuses_by_construction_and_certificates():
    bt = synth.type2(80, 24, 24, seed=2, frac_infeasible=0.15, frac_unbounded=0.15)
    assert set(np.unique(bt.kind)) == {0, 1, 2}
    for k in range(bt.count):
        A, b, c = bt.lp(k)
        r = oracle.solve_one(A, b, c)
        want = {0: 0, 1: 1, 2: 2}[int(bt.kind[k])]
        assert r["status"] == want
        if want == 0:
            assert certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)
        elif want == 1:
            assert certify.is_farkas(A, b, r["cert"][:24])
        else:
            assert certify.is_ray(A, c, r["cert"][:24])


def test_independent_solver_highs():
    sp = pytest.importorskip("scipy.optimize")
    for bt in (synth.type1(20, 40, 40, seed=5), synth.type2(20, 30, 30, seed=6)):
        r = oracle.solve_batch(bt)
        for k in range(bt.count):
            A, b, c = bt.lp(k)
            h = sp.linprog(-c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
            st = {0: 0, 2: 1, 3: 2}[h.status]
            assert r["status"][k] == st
            if st == 0:
                assert abs(r["obj"][k] - (-h.fun)) <= 1e-9 * (1 + abs(h.fun))


def test_beale_cycling_example_terminates():
    """Beale's LP cycles under Dantzig's rule with naive tie-breaking; the oracle must
    still reach the optimum found by enumeration."""
    A = np.array([[0.25, -8, -1, 9], [0.5, -12, -0.5, 3], [0, 0, 1, 0]])
    b = np.array([0.0, 0.0, 1.0])
    c = np.array([0.75, -20, 0.5, -6])
    st, ob, _ = brute.solve(A, b, c)
    r = oracle.solve_one(A, b, c)
    assert st == 0 and r["status"] == 0
    assert abs(r["obj"] - ob) <= 1e-12


def test_iteration_cap():
    bt = synth.type1(1, 30, 30, seed=9)
    A, b, c = bt.lp(0)
    full = oracle.solve_one(A, b, c)
    assert full["status"] == 0 and full["iters"] > 2
    capped = oracle.solve_one(A, b, c, max_iter=2)
    assert capped["status"] == 3 and capped["iters"] == 2


def test_nondegenerate_helper_rejects_degenerate_case():
    case = [c for c in _golden() if c["name"] == "degenerate_corner"][0]
    A = np.array(case["A"], dtype=float)
    r = oracle.solve_one(A, case["b"], case["c"])
    assert not certify.nondegenerate(A, case["b"], case["c"], r["x"], r["y"], r["basis"])
    u = [c for c in _golden() if c["name"] == "two_var_unique"][0]
    A = np.array(u["A"], dtype=float)
    r = oracle.solve_one(A, u["b"], u["c"])
    assert certify.nondegenerate(A, u["b"], u["c"], r["x"], r["y"], r["basis"])
