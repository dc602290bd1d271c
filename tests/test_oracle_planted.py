"""Planted mistakes: each mutation below is a plausible slip in the oracle's C source
(a dropped term, a flipped sign, a wrong index or row).  A mutated copy is compiled
on the CPU and the pins of test_oracle.py must reject it, which shows the pins
constrain every part of the oracle that they are meant to pin."""
import functools
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth
from oracle import brute, certify

SRC = os.path.join(os.path.dirname(oracle.__file__), "simplex_oracle.c")

MUTATIONS = {
    "pivot_row_not_divided": ("pr[j] = pr[j] / pe;", "pr[j] = pr[j];"),
    "row_update_sign": ("ri[j] = ri[j] - f * pr[j];", "ri[j] = ri[j] + f * pr[j];"),
    "ratio_test_takes_max": ("ratio < br ||", "ratio > br ||"),
    "phase1_row_sign": ("TE(&t, m + 1, j) -= TE(&t, i, j);", "TE(&t, m + 1, j) += TE(&t, i, j);"),
    "duals_from_wrong_row": ("y[i] = TE(&t, m, n + i);", "y[i] = TE(&t, m + 1, n + i);"),
    "negated_slack_sign": ("TE(&t, i, n + i) = s;", "TE(&t, i, n + i) = 1.0;"),
    "column_index_reversed": ("s * A[(size_t)i * n + j]", "s * A[(size_t)i * n + (n - 1 - j)]"),
    "objective_row_sign": ("TE(&t, m, j) = -c[j];", "TE(&t, m, j) = c[j];"),
    "ratio_uses_wrong_column": ("TE(t, i, t->ncol) / a", "TE(t, i, e) / a"),
}


@functools.lru_cache(maxsize=1)
def _cases():
    """Tiny integer LPs (all statuses, many ties) and small type-2 LPs, each with its
    brute-force status and optimum."""
    rng = np.random.default_rng(1)
    lps = []
    for _ in range(120):
        m = int(rng.integers(1, 5)); n = int(rng.integers(1, 5))
        lps.append((rng.integers(-3, 4, size=(m, n)).astype(float),
                    rng.integers(-3, 6, size=m).astype(float),
                    rng.integers(-2, 4, size=n).astype(float)))
    bt = synth.type2(10, 6, 5, seed=2, frac_infeasible=0.3, frac_unbounded=0.3)
    lps += [bt.lp(k) for k in range(bt.count)]
    return [(A, b, c) + tuple(brute.solve(A, b, c)[:2]) for A, b, c in lps]


def _pins_hold(lib) -> bool:
    for A, b, c, st, ob in _cases():
        r = oracle.solve_one(A, b, c, lib=lib)
        if r["status"] != st:
            return False
        if st == 0 and (abs(r["obj"] - ob) > 1e-9 * (1 + abs(ob))
                        or not certify.is_optimal_pair(A, b, c, r["x"], r["y"], tol=1e-9)):
            return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "mutated.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutated.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(mutated), "-lm"])
    assert not _pins_hold(oracle.load_variant(str(so)))


def test_unmutated_oracle_passes_the_same_pins():
    assert _pins_hold(None)
