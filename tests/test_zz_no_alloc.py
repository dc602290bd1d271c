"""lpb_solve_noalloc: the solve for callers that cannot allocate device memory (a plug-in
whose host framework owns the device memory pool, a loop where cudaMalloc/cudaFree may not
run because they can synchronise the device).  Its scratch is a fixed array inside the
library instead of a caller workspace.

Called through the C ABI, twice in a row (the second call reuses the array the first one
left behind), it must give the same results as lpb_solve with a caller workspace, within
the tolerances the other parity tests use; a batch whose scratch exceeds the array must be
refused before anything runs; and the device error word that these calls keep in the same
array reads 0 after a clean call (lpb_noalloc_sync_error).  This file is collected last so that a failure here leaves
every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from lp_helpers import host, to_device

pytestmark = pytest.mark.gpu


def _noalloc(solver, batch, prec, out):
    from paper_1609_08114_gb300 import _lib
    opt = solver.options(prec)
    cb, cr = batch.cstruct(), out.cstruct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return solver.lib.lpb_solve_noalloc(ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(cr), stream)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-9), ("fp32_refine", 1e-8)])
def test_noalloc_matches_workspace_solve_twice(prec, rtol):
    from paper_1609_08114_gb300 import Solver, _lib
    solver = Solver(0)
    t1 = synth.type1(400, 60, 50, seed=21)
    t2 = synth.type2(200, 40, 36, seed=22, frac_infeasible=0.1, frac_unbounded=0.1)
    sb = synth.pack([t1.lp(k) for k in range(t1.count)] + [t2.lp(k) for k in range(t2.count)])
    batch = to_device(sb)
    want = host(solver.solve(batch, prec=prec))
    for call in range(2):
        out = solver.alloc_result(batch)
        for t in (out.status, out.iters, out.basis):
            t.fill_(-7)
        for t in (out.obj, out.x, out.y):
            t.fill_(float("nan"))
        assert _noalloc(solver, batch, prec, out) == _lib.OK
        got = host(out)
        assert np.array_equal(got["status"], want["status"]), call
        opt = want["status"] == 0
        rel = np.abs(got["obj"][opt] - want["obj"][opt]) / (1 + np.abs(want["obj"][opt]))
        assert rel.max() <= rtol, call
        assert np.all(np.abs(got["x"] - want["x"]) <= 1e-7 * (1 + np.abs(want["x"]))), call
        assert np.all(np.abs(got["y"] - want["y"]) <= 1e-7 * (1 + np.abs(want["y"]))), call
        word = ctypes.c_uint32(0xFFFFFFFF)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert solver.lib.lpb_noalloc_sync_error(stream, ctypes.byref(word)) == _lib.OK, call
        assert word.value == 0, call                    # a clean call leaves no fault bit


def test_noalloc_refuses_batches_beyond_its_scratch():
    from paper_1609_08114_gb300 import Solver, _lib
    solver = Solver(0)
    sb = synth.type1(2, 3, 3, seed=1)
    # Size bounds of 2000 force per-CTA tableau slots far beyond the fixed array.
    batch = to_device(sb, max_m=2000, max_n=2000)
    out = solver.alloc_result(batch)
    out.status.fill_(-7)
    assert _noalloc(solver, batch, "fp64", out) == _lib.ENOMEM
    torch.cuda.synchronize()
    assert np.all(out.status.cpu().numpy() == -7)      # nothing was launched
