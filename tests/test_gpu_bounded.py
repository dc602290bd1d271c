"""lpb_solve_bounded: max c^T x, A x <= b, l <= x <= u through the C ABI, against the oracle
(its own change of variables, pinned by vertex enumeration and HiGHS): statuses exactly,
objectives to 1e-9 (FP64) or 1e-8 (FP32 with FP64 refinement), x inside its bounds."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _problem(count, m, n, seed, empty=0.0, free_cols=0.0):
    rng = np.random.default_rng(seed)
    lps, ls, us = [], [], []
    for k in range(count):
        A = rng.uniform(0.1, 1, size=(m, n))
        b = rng.uniform(1, 10, size=m)
        c = rng.normal(size=n)
        l = rng.uniform(-1, 0, size=n)
        u = l + rng.uniform(0.5, 2, size=n)
        u[rng.uniform(size=n) < 0.2] = np.inf
        if rng.uniform() < empty:                  # an empty box: infeasible
            u[0] = l[0] - 0.5
        if rng.uniform() < free_cols:              # a column free above with c_j > 0: unbounded
            A[:, 1] = -A[:, 1]
            u[1] = np.inf
            c[1] = abs(c[1]) + 0.1
        lps.append((A, b, c)); ls.append(l); us.append(u)
    return synth.pack(lps), np.concatenate(ls), np.concatenate(us)


def _solve(solver, sb, l, u, prec):
    from paper_1609_08114_gb300 import LPBatch
    batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cuda")
    r = solver.solve_bounded(batch, torch.tensor(l, device="cuda"), torch.tensor(u, device="cuda"), prec=prec)
    torch.cuda.synchronize()
    return {k: getattr(r, k).cpu().numpy() for k in ("status", "obj", "x", "y")}


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-9), ("fp32_refine", 1e-8)])
@pytest.mark.parametrize("m,n", [(30, 20), (60, 60)])
def test_bounded_parity(solver, prec, rtol, m, n):
    sb, l, u = _problem(300, m, n, seed=m * 7 + n, empty=0.05, free_cols=0.05)
    got = _solve(solver, sb, l, u, prec)
    ref = oracle.solve_bounded_batch(sb, l, u)
    assert np.array_equal(got["status"], ref["status"])
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    for k in np.nonzero(ref["status"] == 0)[0]:
        A, b, c = sb.lp(int(k))
        x = got["x"][sb.c_off[k]:sb.c_off[k] + n]
        lk, uk = l[sb.c_off[k]:sb.c_off[k] + n], u[sb.c_off[k]:sb.c_off[k] + n]
        assert abs(got["obj"][k] - ref["obj"][k]) <= rtol * (1 + abs(ref["obj"][k])), k
        assert np.all(x >= lk - 1e-8) and np.all(x <= uk + 1e-8) and np.all(A @ x <= b + 1e-8 * (1 + np.abs(b)))
        assert abs(float(c @ x) - got["obj"][k]) <= 1e-8 * (1 + abs(got["obj"][k]))


def test_bounded_rejects_fp32_and_basis(solver):
    from paper_1609_08114_gb300 import LPBatch, LPBError
    sb, l, u = _problem(4, 5, 4, seed=1)
    batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cuda", dtype=torch.float32)
    with pytest.raises(ValueError):
        solver.solve_bounded(batch, torch.tensor(l, device="cuda"), torch.tensor(u, device="cuda"))
    b64 = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cuda")
    res = solver.alloc_result(b64)                 # a result with a basis array is refused
    with pytest.raises(LPBError):
        solver.solve_bounded(b64, torch.tensor(l, device="cuda"), torch.tensor(u, device="cuda"), out=res)
