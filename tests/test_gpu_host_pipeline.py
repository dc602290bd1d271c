"""lpb_solve_host, the CUDA-streams pipeline of Section 4.5 (copy chunk i+1 in and chunk
i-1's results out while chunk i is solved), through the C ABI.

Each chunk is solved by the same kernels as lpb_solve with the same batch bounds, so the
results must equal those of one lpb_solve of the whole batch bit for bit, for any chunk
size, precision and pivot rule (the random rule keys LPs by their batch index)."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _batch():
    t1 = synth.type1(700, 40, 36, seed=31)
    t2 = synth.type2(150, 30, 28, seed=32, frac_infeasible=0.1, frac_unbounded=0.1)
    return synth.pack([t1.lp(k) for k in range(t1.count)] + [t2.lp(k) for k in range(t2.count)])


def _host_batch(sb, pinned=True):
    from paper_1609_08114_gb300 import LPBatch
    hb = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cpu")
    return hb.pin_memory() if pinned else hb


def _host_result(res):
    torch.cuda.synchronize()
    return {k: getattr(res, k).numpy().copy() for k in ("status", "iters", "obj", "x", "y", "basis")}


@pytest.mark.parametrize("prec,chunk,rule", [("fp32_refine", 256, "lpc"), ("fp32_refine", 333, "rpc"),
                                             ("fp64", 100, "lpc"), ("fp64", 5000, "rpc"),
                                             ("fp32_refine", 1, "lpc")])
def test_host_pipeline_equals_device_solve(solver, prec, chunk, rule):
    sb = _batch()
    if chunk == 1:
        sb = sb.subset(np.arange(40))
    ref = host(solver.solve(to_device(sb), prec=prec, pivot_rule=rule, seed=9))
    got = _host_result(solver.solve_host(_host_batch(sb), prec=prec, chunk=chunk, pivot_rule=rule, seed=9))
    for k in ("status", "iters", "basis"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("obj", "x", "y"):
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    if rule == "lpc":
        compare(sb, got, obj_rtol=1e-9 if prec == "fp64" else 1e-8, check_unique=False)


def test_host_pipeline_pageable_memory(solver):
    sb = _batch().subset(np.arange(300))
    ref = host(solver.solve(to_device(sb), prec="fp32_refine"))
    got = _host_result(solver.solve_host(_host_batch(sb, pinned=False), prec="fp32_refine", chunk=128))
    assert np.array_equal(got["status"], ref["status"]) and np.array_equal(got["obj"], ref["obj"], equal_nan=True)


def test_host_pipeline_rejects_unordered_offsets(solver):
    from paper_1609_08114_gb300 import LPBError
    sb = synth.type1(8, 5, 5, seed=2)
    hb = _host_batch(sb)
    hb.a_off[0], hb.a_off[1] = hb.a_off[1].item(), hb.a_off[0].item()
    with pytest.raises(LPBError):
        solver.solve_host(hb, prec="fp64", chunk=4)


def test_host_pipeline_repeated_calls_reuse_buffers(solver):
    """Back-to-back calls on one stream share the workspace and the handle's streams."""
    sb = _batch()
    hb = _host_batch(sb)
    outs = [solver.solve_host(hb, prec="fp32_refine", chunk=200) for _ in range(3)]
    res = [_host_result(o) for o in outs]
    for r in res[1:]:
        assert np.array_equal(r["obj"], res[0]["obj"], equal_nan=True) and np.array_equal(r["x"], res[0]["x"])
