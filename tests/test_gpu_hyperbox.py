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


def test_fp64_products_round_like_ieee(solver):
    """The FP64 kernel forms each product with a separately rounded multiply (no fused
    multiply-add into the sum); crafted pairs hit exact ties (round to even, both ways),
    carries into the exponent, the edges of the normal range, subnormals, zeros and signed
    zeros.  The oracle's float64 loop is IEEE."""
    eps = 2.0 ** -52
    pairs = [(1 + eps, 1.5), (1 + 3 * eps, 1.5), (1 + eps, 1 + eps), (2 - eps, 1 + eps), (2 - eps, 2 - eps),
             (1.5, 1 + 2 * eps), (3.0, 1 / 3), (2.0 ** 1000, 2.0 ** 23.5), (2.0 ** -1000, 2.0 ** -22),
             (2.0 ** -1022, 0.75), (2.0 ** -1074, 3.0), (2.0 ** 1023, 1.999), (1e300, 1e10), (-0.0, 5.0),
             (0.0, -7.0), (-(1 + eps), 1.5), (np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)),
             (1.0000000000000002, 0.9999999999999999), (2.0 ** -511, 2.0 ** -511), (2.0 ** -512, 2.0 ** -511)]
    rng = np.random.default_rng(3)
    n = 8
    c = np.zeros((len(pairs) * 4, n))
    l = np.full_like(c, -1.0)
    u = np.full_like(c, 1.0)
    for k, (a, b) in enumerate(pairs):
        for s in range(4):                     # each pair in its own LP, with both signs of c
            r = 4 * k + s
            sa = -1.0 if s & 1 else 1.0
            c[r, s] = sa * a
            if sa < 0:
                l[r, s] = -b
            else:
                u[r, s] = b
            c[r, 4:] = rng.normal(size=4)
    obj, x = _run(solver, c, l, u)
    ref, h = ohb.support(c, l, u)
    assert np.array_equal(obj.view(np.uint64), ref.view(np.uint64))
    assert np.array_equal(x, h)
