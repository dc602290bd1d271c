"""GPU parity of steepest-edge pricing (entering column with the largest r_j^2 / gamma_j,
gamma_j = 1 + sum_i t_ij^2; not one of the paper's Section 4.2 rules).

In FP64 the weights are summed in the oracle's row order and the scores compared exactly
(after an FP32 prefilter that keeps every candidate within 1e-5 of the best), so the GPU
follows the oracle's pivot path up to rare near-ties that round differently: statuses
and objectives must match and the pivot counts agree.  The FP32 + FP64-refine form must
give the oracle's statuses and objectives to 1e-8, on the shared-memory / L2-slot kernel
and on the register kernel (its 8-warp templates; a 4-warp register request is refused).
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


def _run(solver, sb, prec, **kw):
    return host(solver.solve(to_device(sb), prec=prec, pivot_rule="steepest", **kw))


@pytest.mark.parametrize("kernel", [1, 2])
def test_steepest_fp64_follows_the_oracle(solver, kernel):
    sb = synth.type1(300, 30, 30, seed=41)
    got = _run(solver, sb, "fp64", kernel=kernel)
    ref = oracle.solve_batch(sb, rule=oracle.SE)
    compare(sb, got, ref=ref, obj_rtol=1e-9)
    assert np.mean(got["iters"] == ref["iters"]) >= 0.97
    lpc = oracle.solve_batch(sb)
    assert ref["iters"].mean() < lpc["iters"].mean()


def test_steepest_fp64_two_phase(solver):
    sb = synth.type2(160, 30, 24, seed=8, frac_infeasible=0.1, frac_unbounded=0.1)
    got = _run(solver, sb, "fp64")
    ref = oracle.solve_batch(sb, rule=oracle.SE)
    compare(sb, got, ref=ref, obj_rtol=1e-9)
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    assert np.mean(got["iters"] == ref["iters"]) >= 0.95


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_steepest_fp32_refine(solver, kernel):
    sb = synth.type1(400, 60, 60, seed=42)
    got = _run(solver, sb, "fp32_refine", kernel=kernel)
    ref = oracle.solve_batch(sb, rule=oracle.SE)
    compare(sb, got, ref=ref, obj_rtol=1e-8)


def test_steepest_fp32_refine_two_phase_mixed_sizes(solver):
    sb = synth.type2(200, 40, 36, seed=9, frac_infeasible=0.1, frac_unbounded=0.1)
    got = _run(solver, sb, "fp32_refine")
    ref = oracle.solve_batch(sb, rule=oracle.SE)
    compare(sb, got, ref=ref, obj_rtol=1e-8)


def test_steepest_takes_fewer_pivots_on_the_gpu(solver):
    sb = synth.type1(2000, 50, 50, seed=43)
    dev = to_device(sb)
    lpc = solver.solve(dev, prec="fp64")
    se = solver.solve(dev, prec="fp64", pivot_rule="steepest")
    torch.cuda.synchronize()
    assert bool((se.status == 0).all()) and bool((lpc.status == 0).all())
    assert se.iters.float().mean().item() < 0.95 * lpc.iters.float().mean().item()
    assert torch.allclose(se.obj, lpc.obj, rtol=1e-10, atol=0)


def test_steepest_register_kernel_takes_fewer_pivots(solver):
    sb = synth.type1(2000, 50, 50, seed=44)
    dev = to_device(sb)
    lpc = solver.solve(dev, prec="fp32_refine", kernel=3)
    se = solver.solve(dev, prec="fp32_refine", kernel=3, pivot_rule="steepest")
    torch.cuda.synchronize()
    assert bool((se.status == 0).all()) and bool((lpc.status == 0).all())
    assert se.iters.float().mean().item() < 0.95 * lpc.iters.float().mean().item()
    assert torch.allclose(se.obj, lpc.obj, rtol=1e-9, atol=0)


def test_steepest_shared_constraints_warm_start(solver):
    """One polytope, many directions, on the register kernel's warm starts: the objectives
    equal those of an explicit batch solved by the oracle."""
    rng = np.random.default_rng(45)
    m, n, k = 40, 40, 300
    A = rng.uniform(0.1, 1.0, (m, n)); b = rng.uniform(1.0, 10.0, m)
    C = rng.uniform(0.0, 1.0, (k, n))
    dev = torch.device("cuda", 0)
    r = solver.solve_shared(torch.tensor(A, device=dev), torch.tensor(b, device=dev),
                            torch.tensor(C, device=dev), prec="fp32_refine", pivot_rule="steepest")
    torch.cuda.synchronize()
    ref = np.array([oracle.solve_one(A, b, C[i], rule=oracle.SE)["obj"] for i in range(k)])
    got = r.obj.cpu().numpy()
    assert bool((r.status == 0).all())
    assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) <= 1e-8


def test_steepest_refuses_the_four_warp_register_kernel(solver):
    from paper_1609_08114_gb300 import LPBError
    sb = synth.type1(4, 10, 10, seed=1)
    with pytest.raises(LPBError):
        solver.solve(to_device(sb), prec="fp32_refine", pivot_rule="steepest", kernel=3, reg_warps=4)
