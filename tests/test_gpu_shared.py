"""lpb_solve_shared: the support function of one polytope in many directions (Section 6's
application), through the C ABI.  Every direction is checked against the oracle solving
the LP (A, b, C[k]) on its own: statuses exactly, objectives to 1e-9 (FP64) or 1e-8 (FP32
with FP64 refinement), and the GPU's (x, y) by KKT in FP64."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import certify

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _check(A, b, C, res, rtol, kkt=1e-8):
    torch.cuda.synchronize()
    count, n = C.shape
    m = A.shape[0]
    sb = synth.pack([(A, b, C[k]) for k in range(count)])
    ref = oracle.solve_batch(sb)
    st = res.status.cpu().numpy()
    assert np.array_equal(st, ref["status"]), (st[:20], ref["status"][:20])
    obj = res.obj.cpu().numpy()
    x = res.x.cpu().numpy().reshape(count, n)
    y = res.y.cpu().numpy().reshape(count, m)
    for k in np.nonzero(ref["status"] == 0)[0]:
        assert abs(obj[k] - ref["obj"][k]) <= rtol * (1 + abs(ref["obj"][k])), k
        assert certify.is_optimal_pair(A, b, C[k], x[k], y[k], tol=kkt), k
    return ref


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-9), ("fp32_refine", 1e-8)])
@pytest.mark.parametrize("m,n", [(40, 30), (100, 100), (150, 140)])
def test_shared_type1_polytope(solver, prec, rtol, m, n):
    lp = synth.type1(1, m, n, seed=m + n)
    A, b, _ = lp.lp(0)
    C = np.random.default_rng(m).normal(size=(300, n))        # directions of every sign
    res = solver.solve_shared(torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"),
                              torch.tensor(C, device="cuda"), prec=prec)
    ref = _check(A, b, C, res, rtol)
    assert np.all(ref["status"] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_shared_phase1_polytope(solver, prec):
    """b has negative entries: every direction needs Phase I."""
    t2 = synth.type2(1, 24, 20, seed=3, frac_infeasible=0.0, frac_unbounded=0.0)
    A, b, _ = t2.lp(0)
    assert (b < 0).any()
    C = np.random.default_rng(4).uniform(0, 1, size=(200, 20))
    res = solver.solve_shared(torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"),
                              torch.tensor(C, device="cuda"), prec=prec)
    _check(A, b, C, res, 1e-9 if prec == "fp64" else 1e-8)


def test_shared_unbounded_and_infeasible_regions(solver):
    rng = np.random.default_rng(5)
    A = rng.uniform(0.1, 1, size=(12, 10)); A[:, 3] = 0.0       # x_3 is free above: unbounded when C[k, 3] > 0
    b = rng.uniform(1, 10, size=12)
    C = rng.normal(size=(120, 10))
    res = solver.solve_shared(torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"),
                              torch.tensor(C, device="cuda"), prec="fp32_refine")
    ref = _check(A, b, C, res, 1e-8)
    assert set(np.unique(ref["status"])) == {0, 2}
    Ai = np.vstack([A[:2], -A[:1]]); bi = np.array([b[0], b[1], -(b[0] + 1.0)])   # a^T x <= b0 and a^T x >= b0 + 1
    res = solver.solve_shared(torch.tensor(Ai, device="cuda"), torch.tensor(bi, device="cuda"),
                              torch.tensor(C[:50], device="cuda"), prec="fp64")
    ref = _check(Ai, bi, C[:50], res, 1e-9)
    assert np.all(ref["status"] == 1)


def test_shared_matches_an_explicit_batch(solver):
    """The same LPs written out as an ordinary packed batch: identical results in FP64;
    in FP32 with refinement the warm starts may end at another optimal basis, so the
    statuses must match and the objectives agree to 1e-8."""
    from paper_1609_08114_gb300 import LPBatch
    lp = synth.type1(1, 60, 50, seed=9)
    A, b, _ = lp.lp(0)
    C = np.random.default_rng(9).uniform(0, 1, size=(256, 50))
    sb = synth.pack([(A, b, C[k]) for k in range(256)])
    batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cuda")
    args = (torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"), torch.tensor(C, device="cuda"))
    res = solver.solve_shared(*args, prec="fp64")
    ref = solver.solve(batch, prec="fp64")
    torch.cuda.synchronize()
    assert torch.equal(res.status, ref.status) and torch.equal(res.obj, ref.obj) and torch.equal(res.x, ref.x)
    assert torch.equal(res.y, ref.y)
    res = solver.solve_shared(*args, prec="fp32_refine")
    ref = solver.solve(batch, prec="fp32_refine")
    torch.cuda.synchronize()
    assert torch.equal(res.status, ref.status)
    rel = ((res.obj - ref.obj).abs() / (1 + ref.obj.abs())).max().item()
    assert rel <= 1e-8


def test_shared_warm_starts_cut_pivots(solver):
    """Slowly turning directions: each objective starts from its neighbour's optimal basis,
    so the pivots per objective fall far below a cold start's, with the same optima."""
    lp = synth.type1(1, 80, 80, seed=12)
    A, b, _ = lp.lp(0)
    rng = np.random.default_rng(12)
    c0, d = rng.uniform(0, 1, size=80), rng.normal(size=80)
    C = c0[None, :] + 1e-3 * np.arange(2048)[:, None] * d[None, :]
    args = (torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda"), torch.tensor(C, device="cuda"))
    warm = solver.solve_shared(*args, prec="fp32_refine")
    cold = solver.solve_shared(*args, prec="fp64")          # the FP64 path starts every LP from the slack basis
    torch.cuda.synchronize()
    assert torch.equal(warm.status, cold.status)
    rel = ((warm.obj - cold.obj).abs() / (1 + cold.obj.abs())).max().item()
    assert rel <= 1e-8
    ok = cold.status == 0
    assert warm.iters[ok].float().mean().item() < 0.5 * cold.iters[ok].float().mean().item()
    _check(A, b, C[:300], solver.solve_shared(args[0], args[1], args[2][:300].contiguous(), prec="fp32_refine"),
           1e-8)
