"""GPU parity of the "random positive coefficient" pivot rule (RPC, Section 4.2).

The random draw is a counter-based function of (seed, LP index, pivot, variable) shared
by the oracle and the kernels, so in FP64 the GPU follows the oracle's pivot path: the
statuses and objectives must match and the pivot counts must agree (up to rare
near-ties that round differently).  The FP32 + FP64-refine form must give the oracle's
statuses and objectives to 1e-8.  And RPC takes more pivots than the most-negative
rule on the GPU too, as the paper observed.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu

SEED = 0x5EED


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _run(solver, sb, prec, **kw):
    return host(solver.solve(to_device(sb), prec=prec, pivot_rule="rpc", seed=SEED, **kw))


@pytest.mark.parametrize("kernel", [1, 2])
def test_rpc_fp64_follows_the_oracle(solver, kernel):
    sb = synth.type1(300, 30, 30, seed=21)
    got = _run(solver, sb, "fp64", kernel=kernel)
    ref = oracle.solve_batch(sb, rule=oracle.RPC, seed=SEED)
    compare(sb, got, ref=ref, obj_rtol=1e-9)
    assert np.mean(got["iters"] == ref["iters"]) >= 0.99
    lpc = oracle.solve_batch(sb)
    assert ref["iters"].mean() > 1.3 * lpc["iters"].mean()


def test_rpc_fp64_two_phase(solver):
    sb = synth.type2(160, 30, 24, seed=7, frac_infeasible=0.1, frac_unbounded=0.1)
    got = _run(solver, sb, "fp64")
    ref = oracle.solve_batch(sb, rule=oracle.RPC, seed=SEED)
    compare(sb, got, ref=ref, obj_rtol=1e-9)
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    assert np.mean(got["iters"] == ref["iters"]) >= 0.97


@pytest.mark.parametrize("kernel", [0, 1, 3])
def test_rpc_fp32_refine(solver, kernel):
    sb = synth.type1(400, 60, 60, seed=22)
    got = _run(solver, sb, "fp32_refine", kernel=kernel)
    ref = oracle.solve_batch(sb, rule=oracle.RPC, seed=SEED)
    compare(sb, got, ref=ref, obj_rtol=1e-8)


def test_rpc_takes_more_pivots_on_the_gpu(solver):
    sb = synth.type1(2000, 50, 50, seed=23)
    dev = to_device(sb)
    lpc = solver.solve(dev, prec="fp32_refine")
    torch.cuda.synchronize()
    it_lpc = lpc.iters.float().mean().item()
    rpc = solver.solve(dev, prec="fp32_refine", pivot_rule="rpc", seed=SEED)
    torch.cuda.synchronize()
    assert bool((rpc.status == 0).all()) and rpc.iters.float().mean().item() > 1.3 * it_lpc


def test_rpc_rejects_unknown_rule(solver):
    from paper_1609_08114_gb300 import LPBError
    sb = synth.type1(4, 5, 5, seed=1)
    with pytest.raises(LPBError):
        solver.solve(to_device(sb), prec="fp64", pivot_rule=7)
