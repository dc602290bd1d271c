"""GPU hyperbox support functions (Section 6, Eq. 8) through the C ABI: bit-exact against
the oracle's fixed-order, per-operation-rounded sum."""
import numpy as np
import pytest
import torch

import synth
from oracle import hyperbox as ohb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    from paper_1609_08114_gb300 import Solver
    return Solver(0)


def _run(solver, c, l, u, want_x=True):
    tc = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    tl = torch.from_numpy(np.ascontiguousarray(l)).cuda()
    tu = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    out = solver.hyperbox(tc, tl, tu, want_x=want_x)
    torch.cuda.synchronize()
    if want_x:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy(), None


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 5, 28, 32, 33, 70])
@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("count", [1, 31, 257, 5000])
def test_bit_exact(solver, dtype, n, shared, count):
    c, l, u = synth.hyperbox(count, n, seed=n + count, shared_box=shared, dtype=dtype)
    obj, x = _run(solver, c, l, u)
    ref, h = ohb.support(c, l, u)
    assert obj.dtype == dtype
    assert np.array_equal(obj.view(np.uint32 if dtype == np.float32 else np.uint64),
                          ref.view(np.uint32 if dtype == np.float32 else np.uint64))
    assert np.array_equal(x, h)


def test_zero_and_negative_zero_directions(solver):
    c = np.array([[0.0, -0.0, 0.0], [-0.0, -0.0, -0.0], [1.0, -2.0, 0.0]])
    l = np.full((3, 3), -4.0); u = np.full((3, 3), 3.0)
    obj, x = _run(solver, c, l, u)
    ref, h = ohb.support(c, l, u)
    assert np.array_equal(np.signbit(obj), np.signbit(ref)) and np.array_equal(obj, ref)
    assert np.array_equal(x, h)


def test_empty(solver):
    c = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    l = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    assert solver.hyperbox(c, l, l).numel() == 0


def test_full_size_sampled(solver):
    """4,000,000 LPs of n = 5 (FP32) and 6,000,000 of n = 28 (FP64) at the benchmark's
    launch configuration; every 997th LP and the last ones against the oracle."""
    for count, n, dt in ((4_000_000, 5, np.float32), (6_000_000, 28, np.float64)):
        c, l, u = synth.hyperbox(count, n, seed=3, dtype=dt)
        obj, _ = _run(solver, c, l, u, want_x=False)
        idx = np.concatenate([np.arange(0, count, 997), np.arange(count - 40, count)])
        ref, _ = ohb.support(c[idx], l[idx], u[idx])
        assert np.array_equal(obj[idx], ref)
