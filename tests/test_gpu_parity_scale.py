"""GPU parity at the workloads' own sizes, and of the passes that the smaller tests reach
only by chance (liblpb.so through the C ABI, against the FP64 oracle).

* Two-phase LPs of m = n = 200 (infeasible slack basis, ~5% infeasible and ~5% unbounded
  LPs mixed in; Section 3's two-phase method): 2,000 LPs of the 10,000-LP batch through
  the default plan, FP32 tableau + FP64 refinement and plain FP64.
* The warm FP64 re-solve of LPs that fail the FP32 certificate: LPs built so that the FP32
  tableau cannot tell two objective coefficients apart, which makes it stop at a basis
  that the FP64 certificate rejects.
* Type-1 LPs of m = n = 300 (the largest size of the size sweep).
* A mixed-size batch solved with the size hints forced to the largest size, so that every
  LP goes through the single pass planned for uniform batches.

Statuses must match exactly, objectives to 1e-9 (FP64) / 1e-8 (FP32 + refinement)
relative, x* and y to the same norm-wise relative tolerances where the oracle certifies
the optimum unique, and every optimal (x, y) must pass an FP64 KKT check.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


@pytest.fixture(scope="module")
def type2_200():
    sb = synth.type2(10_000, 200, 200, seed=2, first=0, stop=2000)
    return sb, oracle.solve_batch(sb)


@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp64", 1e-9)])
def test_two_phase_m200_2000_lps(solver, type2_200, prec, rtol):
    """2,000 two-phase LPs of m = n = 200 (seed 2), default plan (Phase-I pass, L2-slot
    tableau placement, FP64 re-solve of certificate failures)."""
    sb, ref = type2_200
    got = host(solver.solve(to_device(sb), prec=prec))
    _, n_unique = compare(sb, got, ref=ref, obj_rtol=rtol)
    st = ref["status"]
    assert (st == 1).sum() > 40 and (st == 2).sum() > 40 and (st == 0).sum() > 1600
    assert n_unique > 1000
    assert np.all(np.isneginf(got["obj"][st == 1])) and np.all(np.isposinf(got["obj"][st == 2]))


def _near_tie_lps(count, m, n, seed):
    """Type-1 LPs with one extra column: a copy of the column with the largest objective
    coefficient among those basic at the optimum, its coefficient larger by a factor
    1 + 3e-8 (well above the certificate's dual tolerance of about 2e-9).  FP32 rounds the two
    coefficients to the same value as a rule, so the FP32 tableau ties them and keeps the
    lower index; the FP64 certificate then sees a reduced cost of about -3e-8 c_j."""
    base = synth.type1(count, m, n, seed=seed)
    ref = oracle.solve_batch(base)
    lps, dup = [], []
    for k in range(count):
        A, b, c = base.lp(k)
        basic = [int(v) for v in ref["basis"][base.b_off[k]:base.b_off[k] + m] if v < n]
        j = max(basic, key=lambda v: c[v])
        A2 = np.hstack([A, A[:, j:j + 1]])
        c2 = np.concatenate([c, [c[j] * (1.0 + 3e-8)]])
        lps.append((A2, b, c2))
        dup.append(j)
    return synth.pack(lps), np.array(dup)


def test_fp64_resolve_of_certificate_failures(solver):
    sb, dup = _near_tie_lps(200, 30, 30, seed=41)
    ref = oracle.solve_batch(sb)
    got = host(solver.solve(to_device(sb), prec="fp32_refine"))
    resolved = solver.stats()["resolved_fp64"]
    assert resolved >= 50, resolved                 # most LPs went through the FP64 re-solve
    compare(sb, got, ref=ref, obj_rtol=1e-8)
    # The optimum is unique in x: the copy carries the whole value, the original column none.
    for k in range(sb.count):
        x = got["x"][sb.c_off[k]:sb.c_off[k] + 31]
        xr = ref["x"][sb.c_off[k]:sb.c_off[k] + 31]
        assert xr[dup[k]] == 0.0 and xr[30] > 0.0
        assert x[dup[k]] == 0.0, k
        assert abs(x[30] - xr[30]) <= 1e-8 * (1 + abs(xr[30])), k


@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp64", 1e-9)])
def test_type1_m300_sample(solver, prec, rtol):
    """64 LPs of m = n = 300 (beyond every register template: tableau kernel, rows split
    between shared memory and an L2 slot)."""
    sb = synth.type1(2000, 300, 300, seed=3, first=0, stop=64)
    got = host(solver.solve(to_device(sb), prec=prec))
    _, n_unique = compare(sb, got, obj_rtol=rtol)
    assert np.all(got["status"] == 0) and n_unique > 30


@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp32", 1e-5)])
def test_size_hints_forced_to_max(solver, prec, rtol):
    """A wrong size hint costs speed, not correctness: a mixed-size batch of type-1 and
    two-phase LPs declared as if every LP had the largest size."""
    t1 = synth.mixed_sizes(300, seed=17, lo=3, hi=90)
    t2 = synth.type2(100, 40, 36, seed=18, frac_infeasible=0.1, frac_unbounded=0.1)
    sb = synth.pack([t1.lp(k) for k in range(t1.count)] + [t2.lp(k) for k in range(t2.count)])
    ref = oracle.solve_batch(sb)
    plain = to_device(sb)
    hinted = to_device(sb)
    hinted.min_m, hinted.min_n = hinted.max_m, hinted.max_n
    a = host(solver.solve(plain, prec=prec))
    b = host(solver.solve(hinted, prec=prec))
    assert np.array_equal(a["status"], b["status"])
    for got in (a, b):
        compare(sb, got, ref=ref, obj_rtol=rtol, kkt_tol=1e-8 if prec != "fp32" else 1e-4,
                check_unique=prec != "fp32")
