"""Differentiable batched LP solve (torch.autograd) on top of liblpb.

``solve(A, b, c, ...)`` returns ``(obj, x, y, status)`` for every LP
``max c^T x, A x <= b, x >= 0`` of a batch and differentiates ``obj`` and ``x``
with respect to ``(A, b, c)`` through the optimal basis: the backward pass is
liblpb's ``lpb_solve_backward`` kernel (d obj/dc = x*, d obj/db = y,
d obj/dA = -y x*^T, and for x*: v = B^{-T} g_B, d/db += v, d/dA += -v x*^T).
At a degenerate or tied optimum the map is not differentiable and the result
is the gradient for the basis the solver returned.  ``y`` and ``status`` carry
no gradient.
"""
from __future__ import annotations

import torch

from . import LPBatch, Solver

_default_solvers: dict = {}


def _solver_for(device) -> Solver:
    key = (device.type, device.index)
    s = _default_solvers.get(key)
    if s is None:
        s = Solver(device.index or 0)
        _default_solvers[key] = s
    return s


class _LPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, b, c, meta, solver, prec, kw):
        batch = LPBatch(meta["m"], meta["n"], meta["a_off"], meta["b_off"], meta["c_off"],
                        A.detach().reshape(-1), b.detach().reshape(-1), c.detach().reshape(-1),
                        meta["max_m"], meta["max_n"])
        res = solver.solve(batch, prec=prec, **kw)
        ctx.solver, ctx.batch, ctx.res = solver, batch, res
        ctx.shapes = (A.shape, b.shape, c.shape)
        ctx.mark_non_differentiable(res.y, res.status)
        return res.obj, res.x.view(c.shape), res.y.view(b.shape), res.status

    @staticmethod
    def backward(ctx, g_obj, g_x, g_y, g_status):
        g_c, g_b, g_A = ctx.solver.solve_backward(
            ctx.batch, ctx.res, g_obj, None if g_x is None else g_x.reshape(-1))
        sA, sb, sc = ctx.shapes
        dt = ctx.batch.A.dtype
        return g_A.view(sA).to(dt), g_b.view(sb).to(dt), g_c.view(sc).to(dt), None, None, None, None


def solve(A: torch.Tensor, b: torch.Tensor, c: torch.Tensor, m=None, n=None, *, prec: str = "fp32_refine",
          solver: Solver | None = None, **kw):
    """Solve a batch of LPs and make ``obj`` and ``x`` differentiable in ``A``, ``b``, ``c``.

    Dense form: ``A[count, m, n]``, ``b[count, m]``, ``c[count, n]``.  Packed form: flat
    ``A``, ``b``, ``c`` with int sizes ``m[count]``, ``n[count]`` (LP k's ``A`` row-major at
    the running offset).  Tensors live on one CUDA device, FP64 or FP32.
    Returns ``(obj[count], x like c, y like b, status[count])``.
    """
    dev = A.device
    if m is None:
        count, mm, nn = A.shape
        ar = torch.arange(count, device=dev, dtype=torch.int64)
        meta = dict(m=torch.full((count,), mm, dtype=torch.int32, device=dev),
                    n=torch.full((count,), nn, dtype=torch.int32, device=dev),
                    a_off=ar * (mm * nn), b_off=ar * mm, c_off=ar * nn, max_m=mm, max_n=nn)
    else:
        m = torch.as_tensor(m, dtype=torch.int32, device=dev)
        n = torch.as_tensor(n, dtype=torch.int32, device=dev)
        mn = m.to(torch.int64) * n.to(torch.int64)
        z = torch.zeros(1, dtype=torch.int64, device=dev)
        meta = dict(m=m, n=n, a_off=torch.cat([z, torch.cumsum(mn, 0)[:-1]]),
                    b_off=torch.cat([z, torch.cumsum(m.to(torch.int64), 0)[:-1]]),
                    c_off=torch.cat([z, torch.cumsum(n.to(torch.int64), 0)[:-1]]),
                    max_m=int(m.max().item()) if m.numel() else 1,
                    max_n=int(n.max().item()) if n.numel() else 1)
    solver = solver or _solver_for(dev)
    return _LPSolve.apply(A.contiguous(), b.contiguous(), c.contiguous(), meta, solver, prec, kw)
