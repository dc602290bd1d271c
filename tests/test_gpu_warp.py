"""GPU parity of the one-warp-per-LP kernel with the FP32 tableau in shared memory
(LPB_KERNEL_WARP, liblpb.so through the C ABI) against the FP64 oracle.

The kernel runs Section 3.1's Steps 1-3 in one warp per LP (FP64 input, m, n <= 127) and
fuses the FP64 refinement and certificate; LPs it cannot finish go to the shared-memory
kernel (some b_i < 0: Phase I) or to the FP64 re-solve (unbounded or capped in FP32, a
failed certificate, more basic structurals than its refinement holds).  Statuses must
match exactly; objectives within 1e-8 relative after refinement (1e-4 in plain FP32);
x* and y to the same tolerance where the oracle certifies the optimum unique; the GPU's
own (x, y) must pass an FP64 KKT check.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu

WARP = 5


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _check(solver, sb, prec, ref=None, **kw):
    got = host(solver.solve(to_device(sb), prec=prec, kernel=WARP, **kw))
    rtol = 1e-8 if prec == "fp32_refine" else 1e-4
    compare(sb, got, ref=ref, obj_rtol=rtol, kkt_tol=1e-8 if prec != "fp32" else 1e-3,
            check_unique=prec != "fp32")
    assert solver.sync_error() == 0
    return got


@pytest.mark.parametrize("m,n", [(33, 33), (40, 70), (70, 40), (64, 64), (100, 100), (127, 127), (127, 32),
                                 (32, 127), (1, 40), (40, 1), (2, 99), (99, 3), (127, 100), (110, 96), (101, 100)])
@pytest.mark.parametrize("prec", ["fp32_refine", "fp32"])
def test_shapes(solver, m, n, prec):
    """Shapes at and near the kernel's limits: odd and even n (16-byte or single loads in
    the build), row counts that leave a partial last slot of the sweep, one row or column,
    and LPs above 7,000 entries with even n in the wide templates, whose rows arrive in
    rounds of bulk copies with different last rounds (127 x 100, 110 x 96, 101 x 100)."""
    sb = synth.type1(120, m, n, seed=100 + m + 3 * n)
    got = _check(solver, sb, prec)
    assert np.all(got["status"] == 0)


def test_full_workload_sample(solver):
    """300 LPs of the m = n = 100 workload through the warp kernel."""
    sb = synth.type1(50000, 100, 100, seed=1, first=2000, stop=2300)
    _check(solver, sb, "fp32_refine")


def test_degenerate_integer_data(solver):
    """Small-integer data: ties in both ratio tests and degenerate pivots (the lowest-index
    tie rules and Bland's fallback), in a warp-kernel size."""
    rng = np.random.default_rng(41)
    lps = []
    for _ in range(150):
        m, n = int(rng.integers(32, 60)), int(rng.integers(32, 60))
        A = rng.integers(0, 4, size=(m, n)).astype(float)
        b = rng.integers(0, 5, size=m).astype(float)       # zeros: degenerate vertices
        c = rng.integers(0, 4, size=n).astype(float)
        lps.append((A, b, c))
    sb = synth.pack(lps)
    ref = oracle.solve_batch(sb)
    assert (ref["status"] == 2).sum() > 0 or (ref["status"] == 0).sum() > 0
    for prec in ("fp32_refine", "fp32"):
        got = host(solver.solve(to_device(sb), prec=prec, kernel=WARP))
        assert np.array_equal(got["status"], ref["status"])
        opt = ref["status"] == 0
        rel = np.abs(got["obj"][opt] - ref["obj"][opt]) / (1 + np.abs(ref["obj"][opt]))
        assert rel.max() <= (1e-8 if prec == "fp32_refine" else 1e-4)


def test_unbounded_and_phase_one(solver):
    """Unbounded LPs with b >= 0 (a column of A with no positive entry and c_j > 0): the
    FP32 ratio test finds no row, the LP goes to the FP64 re-solve; two-phase LPs (some
    b_i < 0) go to the Phase-I pass; the rest are solved in place."""
    base = synth.type1(90, 50, 45, seed=77)
    lps = []
    for k in range(base.count):
        A, b, c = base.lp(k)
        A = A.copy()
        if k % 3 == 1:
            A[:, k % 45] = -A[:, k % 45]
        lps.append((A, b, c))
    two = synth.type2(60, 48, 40, seed=78, frac_infeasible=0.2, frac_unbounded=0.2)
    sb = synth.pack(lps + [two.lp(k) for k in range(two.count)])
    ref = oracle.solve_batch(sb)
    assert (ref["status"] == 2).sum() >= 30 and (ref["status"] == 1).sum() >= 5
    _check(solver, sb, "fp32_refine", ref=ref)
    _check(solver, sb, "fp32", ref=ref)


def test_random_rule(solver):
    """The random positive-coefficient rule (Section 4.2) in the warp kernel: the same
    counter-based keys as the oracle's; the optimum is unique, so objectives match."""
    sb = synth.type1(200, 60, 60, seed=22)
    ref = oracle.solve_batch(sb, rule=oracle.RPC, seed=7)
    got = host(solver.solve(to_device(sb), prec="fp32_refine", kernel=WARP, pivot_rule="rpc", seed=7))
    compare(sb, got, ref=ref, obj_rtol=1e-8)


def test_iteration_cap(solver):
    """A pivot cap below what the LPs need: plain FP32 stops with ITER_LIMIT after exactly
    the cap; with refinement the capped LPs go to the FP64 re-solve, which reports
    ITER_LIMIT too."""
    sb = synth.type1(40, 50, 50, seed=9)
    got = host(solver.solve(to_device(sb), prec="fp32", kernel=WARP, max_iter=2))
    assert np.all(got["status"] == 3) and np.all(got["iters"] == 2)
    got = host(solver.solve(to_device(sb), prec="fp32_refine", kernel=WARP, max_iter=2))
    assert np.all(got["status"] == 3)


def test_many_basic_structurals_go_to_the_fp64_resolve(solver):
    """LPs whose optimal basis holds more basic structurals than the on-chip refinement
    takes (24): those go to the FP64 re-solve, with oracle parity."""
    rng = np.random.default_rng(5)
    lps = []
    for _ in range(40):
        m = n = 60
        A = np.eye(m) + 0.01 * rng.random((m, n))       # near-diagonal: every column enters
        b = 1.0 + rng.random(m)
        c = 1.0 + rng.random(n)
        lps.append((A, b, c))
    sb = synth.pack(lps)
    ref = oracle.solve_batch(sb)
    assert np.all(ref["status"] == 0)
    assert min(int((ref["basis"][sb.b_off[k]:sb.b_off[k] + 60] < 60).sum()) for k in range(40)) > 24
    got = _check(solver, sb, "fp32_refine", ref=ref)
    assert solver.stats()["resolved_fp64"] == 40
    assert np.all(got["status"] == 0)


def test_planner_picks_it_for_mid_sizes(solver):
    """The default plan for uniform FP64 batches (the size hint min = max given): the warp
    kernel up to m n = 10,000 and, beyond, where an SM holds four of its regions and one
    register-kernel CTA (110 x 100), the register kernel otherwise (100 x 110, 127 x 127);
    parity every way."""
    for (m, n) in ((64, 64), (100, 100), (110, 100), (100, 110), (127, 127)):
        sb = synth.type1(200, m, n, seed=3)
        dev = to_device(sb)
        dev.min_m, dev.min_n = dev.max_m, dev.max_n
        got = host(solver.solve(dev, prec="fp32_refine"))
        compare(sb, got, obj_rtol=1e-8)


def test_mixed_batch_class(solver):
    """A mixed-size batch (m, n ~ U{3..127}): the size classes up to 63 x 63 and 127 x 103
    run on the warp kernel by default, the smallest and the largest on the register
    templates."""
    sb = synth.mixed_sizes(400, seed=12, lo=3, hi=127)
    got = host(solver.solve(to_device(sb), prec="fp32_refine"))
    compare(sb, got, obj_rtol=1e-8)


def test_shared_constraints(solver):
    """lpb_solve_shared with the warp kernel asked for: every LP shares A and b (no warm
    starts on this kernel); each direction against the oracle."""
    rng = np.random.default_rng(8)
    m, n, k = 48, 40, 64
    A = 0.1 + 0.9 * rng.random((m, n))
    b = 1 + 9 * rng.random(m)
    C = rng.random((k, n))
    r = solver.solve_shared(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(C).cuda(),
                            prec="fp32_refine", kernel=WARP)
    torch.cuda.synchronize()
    sb = synth.pack([(A, b, C[j]) for j in range(k)])
    ref = oracle.solve_batch(sb)
    assert np.array_equal(r.status.cpu().numpy(), ref["status"])
    rel = np.abs(r.obj.cpu().numpy() - ref["obj"]) / (1 + np.abs(ref["obj"]))
    assert rel.max() <= 1e-8


def test_fp32_input_is_refused(solver):
    """The warp kernel reads FP64 input only: asking for it with FP32 data is refused."""
    from paper_1609_08114_gb300 import LPBError
    sb = synth.type1(10, 40, 40, seed=1)
    with pytest.raises(LPBError):
        solver.solve(to_device(sb, dtype=torch.float32), prec="fp32_refine", kernel=WARP)
