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


def _diag_dominant_lps(count, m, seed):
    """LPs whose optimum has most structurals basic (k > 64 basic structurals, so the
    backward kernel eliminates its k x k system in a workspace slot instead of shared
    memory): A = diag(U[1,2]) + 0.01 U[0,1], b ~ U[1,10], c ~ U[0.5,1]."""
    rng = np.random.default_rng(seed)
    lps = []
    for _ in range(count):
        A = np.diag(rng.uniform(1.0, 2.0, m)) + 0.01 * rng.uniform(0.0, 1.0, (m, m))
        lps.append((A, rng.uniform(1.0, 10.0, m), rng.uniform(0.5, 1.0, m)))
    return synth.pack(lps)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("cnt,m,kmin", [(24, 96, 65), (16, 48, 33)])
def test_backward_large_basic_systems(prec, cnt, m, kmin):
    """Systems beyond one warp's 32 rows (k in 33..64: block-wide elimination in shared
    memory; k > 64: in a workspace slot).  g_obj = 1: the gradients are the oracle's duals
    and vertex; random upstream grads: central finite differences of the oracle re-solved
    at perturbed data."""
    from paper_1609_08114_gb300.autograd import solve
    sb = _diag_dominant_lps(cnt, m, seed=77 if m == 96 else 78)
    ref = oracle.solve_batch(sb)
    ks = [int((ref["basis"][sb.b_off[k]:sb.b_off[k] + m] < m).sum()) for k in range(cnt)]
    assert min(ks) >= kmin and (kmin > 64 or max(ks) <= 64), ks
    A = torch.tensor(sb.A.reshape(cnt, m, m), device="cuda", requires_grad=True)
    b = torch.tensor(sb.b.reshape(cnt, m), device="cuda", requires_grad=True)
    c = torch.tensor(sb.c.reshape(cnt, m), device="cuda", requires_grad=True)
    obj, x, y, status = solve(A, b, c, prec=prec)
    assert torch.all(status == 0)
    rng = np.random.default_rng(3)
    g_obj = rng.standard_normal(cnt)
    g_x = rng.standard_normal((cnt, m))
    loss = (obj * torch.tensor(g_obj, device="cuda")).sum() + (x * torch.tensor(g_x, device="cuda")).sum()
    gA, gb, gc = (t.cpu().numpy() for t in torch.autograd.grad(loss, (A, b, c)))
    h = 1e-6
    for k in range(cnt):
        Ak, bk, ck = _dense(sb, k)
        rk = oracle.solve_one(Ak, bk, ck)
        assert _margin_ok(Ak, bk, ck, rk, 1e-4), k
        for _ in range(2):
            dA, db, dc = rng.standard_normal(Ak.shape), rng.standard_normal(m), rng.standard_normal(m)
            fd = (_f(Ak + h * dA, bk + h * db, ck + h * dc, g_obj[k], g_x[k]) -
                  _f(Ak - h * dA, bk - h * db, ck - h * dc, g_obj[k], g_x[k])) / (2 * h)
            an = np.sum(gA[k] * dA) + gb[k] @ db + gc[k] @ dc
            assert abs(fd - an) <= 1e-5 * (1 + abs(fd)), (k, fd, an)
    # g_obj = 1, g_x = 0: duals and vertex of the oracle
    A.grad = b.grad = c.grad = None
    obj, x, y, status = solve(A, b, c, prec=prec)
    obj.sum().backward()
    for k in range(cnt):
        np.testing.assert_allclose(b.grad[k].cpu().numpy(), ref["y"][sb.b_off[k]:sb.b_off[k] + m], atol=1e-9)
        np.testing.assert_allclose(c.grad[k].cpu().numpy(), ref["x"][sb.c_off[k]:sb.c_off[k] + m], atol=1e-9)


def test_mixed_size_batch_finite_differences_200_lps():
    """The mixed-size workload (m, n ~ U{8..256} independently, type-1 values, seed 4):
    forward and backward of the first 1,000 LPs in one batch (size classes, FP32 tableau +
    FP64 refinement); on 200 LPs that the oracle certifies non-degenerate with a margin of
    1e-3, 8 random directions each: <grad, v> against the central difference (h = 1e-6,
    FP64) of g_obj obj + g_x^T x* re-solved by the oracle at p +- h v."""
    from paper_1609_08114_gb300.autograd import solve
    sb = synth.mixed_sizes(20000, seed=4, first=0, stop=1000)
    ref = oracle.solve_batch(sb)
    rng = np.random.default_rng(11)
    g_obj = rng.standard_normal(sb.count)
    g_x = rng.standard_normal(sb.c.size)
    A = torch.tensor(sb.A, device="cuda", requires_grad=True)
    b = torch.tensor(sb.b, device="cuda", requires_grad=True)
    c = torch.tensor(sb.c, device="cuda", requires_grad=True)
    obj, x, y, status = solve(A, b, c, sb.m, sb.n, prec="fp32_refine")
    assert np.array_equal(status.cpu().numpy(), ref["status"])
    loss = (obj * torch.tensor(g_obj, device="cuda")).sum() + (x * torch.tensor(g_x, device="cuda")).sum()
    gA, gb, gc = (t.cpu().numpy() for t in torch.autograd.grad(loss, (A, b, c)))
    chosen = []
    for k in range(sb.count):
        Ak, bk, ck = _dense(sb, k)
        m, n = Ak.shape
        rk = dict(status=ref["status"][k], basis=ref["basis"][sb.b_off[k]:sb.b_off[k] + m],
                  x=ref["x"][sb.c_off[k]:sb.c_off[k] + n], y=ref["y"][sb.b_off[k]:sb.b_off[k] + m])
        if _margin_ok(Ak, bk, ck, rk, 1e-3):
            chosen.append(k)
        if len(chosen) == 200:
            break
    assert len(chosen) == 200
    h = 1e-6
    for c0 in range(0, 200, 25):
        lps, meta = [], []
        for k in chosen[c0:c0 + 25]:
            Ak, bk, ck = _dense(sb, k)
            for _ in range(8):
                dA, db, dc = rng.standard_normal(Ak.shape), rng.standard_normal(bk.shape), rng.standard_normal(ck.shape)
                lps += [(Ak + h * dA, bk + h * db, ck + h * dc), (Ak - h * dA, bk - h * db, ck - h * dc)]
                sa, sb_, sc = (slice(sb.a_off[k], sb.a_off[k] + Ak.size), slice(sb.b_off[k], sb.b_off[k] + bk.size),
                               slice(sb.c_off[k], sb.c_off[k] + ck.size))
                meta.append((k, float(np.sum(gA[sa] * dA.ravel()) + gb[sb_] @ db + gc[sc] @ dc)))
        pb = synth.pack(lps)
        rp = oracle.solve_batch(pb)
        assert np.all(rp["status"] == 0)
        for i, (k, an) in enumerate(meta):
            f = []
            for j in (2 * i, 2 * i + 1):
                xs = rp["x"][pb.c_off[j]:pb.c_off[j] + pb.n[j]]
                f.append(g_obj[k] * rp["obj"][j] + g_x[sb.c_off[k]:sb.c_off[k] + sb.n[k]] @ xs)
            fd = (f[0] - f[1]) / (2 * h)
            assert abs(fd - an) <= 1e-5 * (1 + abs(fd)), (k, fd, an)
