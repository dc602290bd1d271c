"""GPU parity of the batched simplex (liblpb.so through the C ABI) against the FP64 oracle.

Statuses must match exactly; objectives within 1e-9 relative in FP64 and 1e-8 after
FP32 + FP64 refinement; x* and y to the same relative tolerances (norm-wise) where the oracle
certifies the optimum unique;
and the GPU's own (x, y) must satisfy KKT in FP64 on every optimal LP.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def run(solver, sb, prec, dtype=torch.float64, **kw):
    res = solver.solve(to_device(sb, dtype=dtype), prec=prec, **kw)
    return host(res)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-9), ("fp32_refine", 1e-8)])
def test_type1_m16_full_batch(solver, prec, rtol):
    """1,000 LPs of m = n = 16 (A ~ U[0.1,1], b ~ U[1,10], c ~ U[0,1], seed 0)."""
    sb = synth.type1(1000, 16, 16, seed=0)
    got = run(solver, sb, prec)
    ref, n_unique = compare(sb, got, obj_rtol=rtol)
    assert np.all(got["status"] == 0) and n_unique > 900


@pytest.mark.parametrize("prec,rtol,kernel,threads", [
    ("fp64", 1e-9, 1, 0), ("fp64", 1e-9, 2, 0),                 # shared-memory, L2-slot tableau
    ("fp32_refine", 1e-8, 1, 0), ("fp32_refine", 1e-8, 2, 0),
    ("fp32_refine", 1e-8, 3, 128), ("fp32_refine", 1e-8, 3, 256),  # register tableau, 4 or 8 warps
    ("fp32", 1e-5, 3, 0)])
def test_type1_m100_sample(solver, prec, rtol, kernel, threads):
    """300 LPs of the m = n = 100 workload through every kernel class."""
    sb = synth.type1(50000, 100, 100, seed=1, first=1000, stop=1300)
    got = run(solver, sb, prec, kernel=kernel, threads=threads)
    compare(sb, got, obj_rtol=rtol, kkt_tol=1e-8 if prec != "fp32" else 1e-4,
            check_unique=prec != "fp32")


@pytest.mark.parametrize("m,n", [(1, 1), (5, 5), (7, 7), (12, 15), (16, 16), (31, 7), (9, 31), (31, 31)])
@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp32", 1e-5)])
def test_one_warp_templates(solver, m, n, prec, rtol):
    """Tiny LPs at and near the 8-, 16- and 32-column limits: the default plan (several LPs
    per warp up to m, n <= 15, one warp per LP up to 31) and the one-warp templates, against
    the oracle and against the 8-warp templates."""
    sb = synth.type1(300, m, n, seed=7 * m + n)
    wide = run(solver, sb, prec, reg_warps=8)
    for kw in ({}, {"reg_warps": 1}):
        got = run(solver, sb, prec, **kw)
        compare(sb, got, obj_rtol=rtol, kkt_tol=1e-8 if prec != "fp32" else 1e-4, check_unique=prec != "fp32")
        assert np.array_equal(got["status"], wide["status"])
        assert np.allclose(got["obj"], wide["obj"], rtol=rtol, atol=0)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 7), (7, 2), (5, 5), (7, 7), (8, 8), (7, 8), (8, 3), (12, 15), (15, 15),
                                 (15, 9), (16, 16), (16, 3), (20, 31), (31, 7), (31, 31)])
@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp32", 1e-5)])
def test_several_lps_per_warp(solver, m, n, prec, rtol):
    """Several tiny LPs per warp (four of m, n <= 7, two of m, n <= 15, one of m, n <= 31 in
    one warp), at and near every segment limit and with a ragged last group (1001 LPs),
    against the oracle."""
    from paper_1609_08114_gb300 import KERNEL_PACK
    sb = synth.type1(1001, m, n, seed=31 * m + n)
    got = run(solver, sb, prec, kernel=KERNEL_PACK)
    compare(sb, got, obj_rtol=rtol, kkt_tol=1e-8 if prec != "fp32" else 1e-4, check_unique=prec != "fp32")
    assert solver.stats()["deferred"] == 0
    auto = run(solver, sb, prec)                   # the default plan takes the same kernel
    assert np.array_equal(auto["status"], got["status"]) and np.array_equal(auto["obj"], got["obj"])


def test_several_lps_per_warp_all_statuses(solver):
    """Mixed tiny LPs with Phase I (deferred to the tableau kernel), infeasible and unbounded
    LPs (confirmed by the FP64 re-solve), integer data with ties and degenerate vertices,
    and the random pivot rule."""
    from paper_1609_08114_gb300 import KERNEL_PACK
    t2 = synth.type2(200, 12, 10, seed=14, frac_infeasible=0.15, frac_unbounded=0.15)
    lps = [t2.lp(k) for k in range(t2.count)] + _tiny_integer_lps(9, 400)
    lps += [synth.mixed_sizes(300, seed=15, lo=1, hi=15).lp(k) for k in range(300)]
    sb = synth.pack(lps)
    ref = oracle.solve_batch(sb)
    for kw in ({"kernel": KERNEL_PACK}, {}):
        got = run(solver, sb, "fp32_refine", **kw)
        compare(sb, got, ref=ref, obj_rtol=1e-8, check_unique=False)
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    got = run(solver, sb, "fp32_refine", kernel=KERNEL_PACK, pivot_rule="rpc", seed=5)
    compare(sb, got, ref=ref, obj_rtol=1e-8, check_unique=False)


def test_one_warp_templates_mixed_and_two_phase(solver):
    """Tiny LPs of mixed sizes with infeasible and unbounded ones (Phase-I LPs leave the
    register kernel for the tableau kernel)."""
    sb = synth.type2(400, 24, 20, seed=12, frac_infeasible=0.1, frac_unbounded=0.1)
    got = run(solver, sb, "fp32_refine")
    compare(sb, got, obj_rtol=1e-8)
    sb = synth.mixed_sizes(500, seed=13, lo=1, hi=31)
    got = run(solver, sb, "fp32_refine")
    compare(sb, got, obj_rtol=1e-8)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 5), (16, 16), (31, 20), (20, 31), (40, 63), (63, 63),
                                 (100, 100), (127, 103), (120, 127)])
def test_register_kernel_shapes(solver, m, n):
    """Every register-tableau configuration at and near its size limits (ragged tiles)."""
    sb = synth.type1(120, m, n, seed=m * 1000 + n)
    got = run(solver, sb, "fp32_refine", kernel=3)
    compare(sb, got, obj_rtol=1e-8)
    assert solver.stats()["deferred"] == 0


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-9), ("fp32_refine", 1e-8)])
def test_type2_two_phase(solver, prec, rtol):
    """Infeasible initial basis: Phase I, with infeasible and unbounded LPs mixed in."""
    sb = synth.type2(240, 48, 40, seed=2, frac_infeasible=0.1, frac_unbounded=0.1)
    got = run(solver, sb, prec)
    ref, _ = compare(sb, got, obj_rtol=rtol)
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    assert np.all(np.isinf(got["obj"][got["status"] == 1]) & (got["obj"][got["status"] == 1] < 0))
    assert np.all(np.isinf(got["obj"][got["status"] == 2]) & (got["obj"][got["status"] == 2] > 0))


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine", "fp32"])
def test_handworked_golden(solver, prec):
    cases = json.load(open(os.path.join(HERE, "golden", "handworked_lps.json")))["cases"]
    sb = synth.pack([(np.array(c["A"], float), np.array(c["b"], float), np.array(c["c"], float)) for c in cases])
    got = run(solver, sb, prec)
    for k, c in enumerate(cases):
        assert got["status"][k] == c["status"], c["name"]
        if c["status"] == 0:
            assert abs(got["obj"][k] - c["obj"]) <= (1e-12 if prec != "fp32" else 1e-5) * (1 + abs(c["obj"])), c["name"]


def _tiny_integer_lps(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(1, 6)); n = int(rng.integers(1, 6))
        out.append((rng.integers(-3, 4, size=(m, n)).astype(float), rng.integers(-3, 6, size=m).astype(float),
                    rng.integers(-2, 4, size=n).astype(float)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_tiny_degenerate_lps_all_statuses(solver, prec):
    """Integer data: ties, degenerate vertices, redundant rows, all three statuses."""
    sb = synth.pack(_tiny_integer_lps(5, 600))
    got = run(solver, sb, prec)
    ref, _ = compare(sb, got, obj_rtol=1e-9, check_unique=False)
    assert set(np.unique(ref["status"])) == {0, 1, 2}


def test_mixed_sizes_small(solver):
    sb = synth.mixed_sizes(120, seed=4, lo=1, hi=64)
    for prec in ("fp64", "fp32_refine"):
        got = run(solver, sb, prec)
        compare(sb, got, obj_rtol=1e-9 if prec == "fp64" else 1e-8)


def test_fp32_input_dtype(solver):
    sb = synth.type1(200, 30, 20, seed=8)
    got = run(solver, sb, "fp32_refine", dtype=torch.float32)
    sb32 = synth.pack([tuple(a.astype(np.float32).astype(np.float64) for a in sb.lp(k)) for k in range(sb.count)])
    compare(sb32, got, obj_rtol=1e-8)


def test_edge_cases(solver):
    from paper_1609_08114_gb300 import LPBatch
    # empty batch
    empty = synth.pack([])
    lb = LPBatch.from_packed(empty.m, empty.n, empty.A, empty.b, empty.c, device="cuda", max_m=4, max_n=4)
    r = solver.solve(lb, prec="fp64")
    assert r.status.numel() == 0
    # m = 1 / n = 1 and a size above the declared bound
    lps = [(np.array([[2.0]]), np.array([7.0]), np.array([3.0])),
           (np.ones((1, 9)), np.array([4.0]), np.arange(9.0)),
           (np.ones((9, 1)), np.arange(1.0, 10.0), np.array([1.0]))]
    sb = synth.pack(lps)
    got = host(solver.solve(to_device(sb, max_m=9, max_n=9), prec="fp64"))
    compare(sb, got)
    big = synth.pack(lps + [(np.ones((12, 3)), np.ones(12), np.ones(3))])
    got = host(solver.solve(to_device(big, max_m=9, max_n=9), prec="fp64"))
    assert list(got["status"]) == [0, 0, 0, 5]
    # NaN in the data -> numeric status, others unaffected
    A, b, c = lps[1]
    A = A.copy(); A[0, 3] = np.nan
    got = host(solver.solve(to_device(synth.pack([lps[0], (A, b, c), lps[2]])), prec="fp64"))
    assert list(got["status"]) == [0, 4, 0]
    # iteration cap
    sb = synth.type1(4, 30, 30, seed=9)
    got = host(solver.solve(to_device(sb), prec="fp64", max_iter=2))
    assert np.all(got["status"] == 3) and np.all(got["iters"] == 2)
    assert solver.sync_error() == 0


def test_full_size_sampled_parity(solver):
    """The 50,000 x (m = n = 100) batch in the benchmark's launch configuration; the oracle
    checks a sample of 400 LPs spread over the batch."""
    sb = synth.type1(50000, 100, 100, seed=1)
    dev = to_device(sb)
    idx = np.unique(np.linspace(0, 49999, 400).astype(int))
    for prec, rtol in (("fp32_refine", 1e-8), ("fp64", 1e-9)):
        got = host(solver.solve(dev, prec=prec))
        assert np.all(got["status"] == 0)
        sub = sb.subset(idx)
        sel = {k: v for k, v in got.items()}
        sel["status"] = got["status"][idx]; sel["obj"] = got["obj"][idx]; sel["iters"] = got["iters"][idx]
        sel["x"] = np.concatenate([got["x"][sb.c_off[k]:sb.c_off[k] + 100] for k in idx])
        sel["y"] = np.concatenate([got["y"][sb.b_off[k]:sb.b_off[k] + 100] for k in idx])
        sel["basis"] = np.concatenate([got["basis"][sb.b_off[k]:sb.b_off[k] + 100] for k in idx])
        compare(sub, sel, obj_rtol=rtol)


@pytest.mark.parametrize("prec,rtol", [("fp32_refine", 1e-8), ("fp64", 1e-9)])
def test_mixed_sizes_up_to_256(solver, prec, rtol):
    """The mixed-size workload's distribution (m, n ~ U{8..256}): the batch is split into size
    classes (register templates and the tableau kernel for the rest)."""
    sb = synth.mixed_sizes(20000, seed=4, first=0, stop=160)
    got = run(solver, sb, prec)
    compare(sb, got, obj_rtol=rtol)


def test_cuda_graph_replay_matches_eager(solver):
    """A whole solve is a fixed sequence of memsets and kernels with device-side work-list
    lengths, so it can be captured once and replayed."""
    sb = synth.mixed_sizes(300, seed=12, lo=4, hi=150)
    dev = to_device(sb)
    eager = host(solver.solve(dev, prec="fp32_refine"))
    out = solver.alloc_result(dev)
    solver.solve(dev, prec="fp32_refine", out=out)          # sizes the workspace before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            solver.solve(dev, prec="fp32_refine", out=out)
    for t in (out.status, out.iters):
        t.fill_(-9)
    out.obj.fill_(float("nan"))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    rep = host(out)
    assert np.array_equal(rep["status"], eager["status"])
    assert np.array_equal(rep["obj"], eager["obj"])
    assert np.array_equal(rep["x"], eager["x"])
