"""GPU backward (lpb_solve_backward through torch.autograd) against independent facts:

* with g_obj = 1 and g_x = 0 the gradients are the oracle's duals and vertex:
  d obj/db = y, d obj/dc = x*, d obj/dA = -y x*^T;
* for random upstream gradients, directional derivatives match central finite
  differences (h = 1e-6, FP64) of the oracle re-solved at perturbed data, on LPs the
  oracle certifies non-degenerate with a margin well above the perturbation;
* non-optimal LPs get zero gradients.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import certify

pytestmark = pytest.mark.gpu


def _dense(sb, k):
    A, b, c = sb.lp(k)
    return A, b, c


def _margin_ok(A, b, c, r, margin):
    m, n = A.shape
    basis = r["basis"]
    if r["status"] != 0 or np.any(basis < 0):
        return False
    z = np.concatenate([r["x"], b - A @ r["x"]])
    red = np.concatenate([A.T @ r["y"] - c, r["y"]])
    nb = np.setdiff1d(np.arange(n + m), basis)
    return bool(np.all(z[basis] > margin) and np.all(red[nb] > margin))


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_gradient_of_obj_is_duals_and_vertex(prec):
    from paper_1609_08114_gb300.autograd import solve
    sb = synth.type1(64, 20, 24, seed=31)
    A = torch.tensor(sb.A.reshape(64, 20, 24), device="cuda", requires_grad=True)
    b = torch.tensor(sb.b.reshape(64, 20), device="cuda", requires_grad=True)
    c = torch.tensor(sb.c.reshape(64, 24), device="cuda", requires_grad=True)
    obj, x, y, status = solve(A, b, c, prec=prec)
    obj.sum().backward()
    ref = oracle.solve_batch(sb)
    gA, gb, gc = A.grad.cpu().numpy(), b.grad.cpu().numpy(), c.grad.cpu().numpy()
    checked = 0
    for k in range(64):
        Ak, bk, ck = _dense(sb, k)
        rk = oracle.solve_one(Ak, bk, ck)
        if not certify.nondegenerate(Ak, bk, ck, rk["x"], rk["y"], rk["basis"]):
            continue
        checked += 1
        np.testing.assert_allclose(gb[k], rk["y"], atol=1e-9)
        np.testing.assert_allclose(gc[k], rk["x"], atol=1e-9)
        np.testing.assert_allclose(gA[k], -np.outer(rk["y"], rk["x"]), atol=1e-9)
    assert checked > 50


def _f(Ak, bk, ck, go, gx):
    r = oracle.solve_one(Ak, bk, ck)
    assert r["status"] == 0
    return go * r["obj"] + gx @ r["x"]


@pytest.mark.parametrize("sizes", [(30, 30), (12, 40), (60, 20)])
def test_finite_differences_obj_and_x(sizes):
    from paper_1609_08114_gb300.autograd import solve
    m, n = sizes
    cnt = 40
    sb = synth.type1(cnt, m, n, seed=m * 7 + n)
    rng = np.random.default_rng(5)
    g_obj = rng.standard_normal(cnt)
    g_x = rng.standard_normal((cnt, n))
    A = torch.tensor(sb.A.reshape(cnt, m, n), device="cuda", requires_grad=True)
    b = torch.tensor(sb.b.reshape(cnt, m), device="cuda", requires_grad=True)
    c = torch.tensor(sb.c.reshape(cnt, n), device="cuda", requires_grad=True)
    obj, x, _, status = solve(A, b, c, prec="fp32_refine")
    loss = (obj * torch.tensor(g_obj, device="cuda")).sum() + (x * torch.tensor(g_x, device="cuda")).sum()
    gA, gb, gc = torch.autograd.grad(loss, (A, b, c))
    gA, gb, gc = gA.cpu().numpy(), gb.cpu().numpy(), gc.cpu().numpy()
    h, checked = 1e-6, 0
    for k in range(cnt):
        Ak, bk, ck = _dense(sb, k)
        rk = oracle.solve_one(Ak, bk, ck)
        if not _margin_ok(Ak, bk, ck, rk, 1e-3):
            continue
        for _ in range(4):
            dA, db, dc = rng.standard_normal(Ak.shape), rng.standard_normal(m), rng.standard_normal(n)
            fp = _f(Ak + h * dA, bk + h * db, ck + h * dc, g_obj[k], g_x[k])
            fm = _f(Ak - h * dA, bk - h * db, ck - h * dc, g_obj[k], g_x[k])
            fd = (fp - fm) / (2 * h)
            an = np.sum(gA[k] * dA) + gb[k] @ db + gc[k] @ dc
            assert abs(fd - an) <= 1e-5 * (1 + abs(fd)), (k, fd, an)
        checked += 1
    assert checked >= 10


def test_packed_mixed_sizes_and_non_optimal_get_zero():
    from paper_1609_08114_gb300.autograd import solve
    t1 = synth.mixed_sizes(30, seed=9, lo=3, hi=40)
    t2 = synth.type2(20, 12, 10, seed=3, frac_infeasible=0.3, frac_unbounded=0.3)
    sb = synth.pack([t1.lp(k) for k in range(t1.count)] + [t2.lp(k) for k in range(t2.count)])
    A = torch.tensor(sb.A, device="cuda", requires_grad=True)
    b = torch.tensor(sb.b, device="cuda", requires_grad=True)
    c = torch.tensor(sb.c, device="cuda", requires_grad=True)
    obj, x, y, status = solve(A, b, c, sb.m, sb.n, prec="fp32_refine")
    st = status.cpu().numpy()
    ref = oracle.solve_batch(sb)
    assert np.array_equal(st, ref["status"])
    w = torch.where(status == 0, 1.0, 0.0).to(torch.float64)
    (obj.nan_to_num(0.0, 0.0, 0.0) * w).sum().backward()
    gb, gc, gA = b.grad.cpu().numpy(), c.grad.cpu().numpy(), A.grad.cpu().numpy()
    for k in range(sb.count):
        sl_b = slice(sb.b_off[k], sb.b_off[k] + sb.m[k])
        sl_c = slice(sb.c_off[k], sb.c_off[k] + sb.n[k])
        sl_a = slice(sb.a_off[k], sb.a_off[k] + sb.m[k] * sb.n[k])
        if st[k] != 0:
            assert not gb[sl_b].any() and not gc[sl_c].any() and not gA[sl_a].any()
        else:
            np.testing.assert_allclose(gc[sl_c], x.detach().cpu().numpy()[sl_c], atol=1e-12)
            np.testing.assert_allclose(gb[sl_b], y.detach().cpu().numpy()[sl_b], atol=1e-12)
