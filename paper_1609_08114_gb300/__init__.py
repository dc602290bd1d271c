"""Batched linear programs on one GB300 GPU (liblpb, Python binding).

A thin layer over the C ABI of ``include/lpb.h``: it holds device tensors,
passes their pointers and the current torch stream to ``liblpb.so`` and
returns the output tensors.  Every step of the solver runs in liblpb's CUDA
kernels; the binding refuses to run without the library.

* :class:`Solver` -- ``solve`` (Section 3.1 Steps 1-3, two-phase when needed),
  ``hyperbox`` (Section 6, Eq. 8), stats and the device error word.
* :class:`LPBatch` -- a device-resident packed batch of LPs
  ``max c^T x, A x <= b, x >= 0`` of any sizes.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (BAD_SIZE, FP32, FP32_REFINE, FP64, INFEASIBLE, ITER_LIMIT, KERNEL_AUTO, KERNEL_GMEM,
                   KERNEL_PACK, KERNEL_REG, KERNEL_SMEM, KERNEL_WARP, NUMERIC, OPTIMAL, UNBOUNDED, LPBError)

__all__ = ["Solver", "LPBatch", "SolveResult", "LPBError", "OPTIMAL", "INFEASIBLE", "UNBOUNDED",
           "ITER_LIMIT", "NUMERIC", "BAD_SIZE", "FP64", "FP32_REFINE", "FP32", "KERNEL_AUTO",
           "KERNEL_SMEM", "KERNEL_GMEM", "KERNEL_REG", "KERNEL_PACK", "KERNEL_WARP", "PRECISIONS"]

PRECISIONS = {"fp64": FP64, "fp32_refine": FP32_REFINE, "fp32": FP32}
# Step 1 rules of Section 4.2: most negative reduced cost, or a random eligible column.
PIVOT_RULES = {"lpc": _lib.PIVOT_LPC, "rpc": _lib.PIVOT_RPC, "steepest": _lib.PIVOT_STEEPEST}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class LPBatch:
    """A packed batch on the device: LP k's ``A`` (m_k x n_k, row-major) at ``a_off[k]``,
    ``b`` at ``b_off[k]``, ``c`` at ``c_off[k]``."""

    def __init__(self, m, n, a_off, b_off, c_off, A, b, c, max_m: int, max_n: int, min_m: int = 0,
                 min_n: int = 0):
        self.m, self.n = m, n
        self.a_off, self.b_off, self.c_off = a_off, b_off, c_off
        self.A, self.b, self.c = A, b, c
        self.max_m, self.max_n = int(max_m), int(max_n)
        self.min_m, self.min_n = int(min_m), int(min_n)     # size hints, 0 = unknown

    @property
    def count(self) -> int:
        return int(self.m.numel())

    @property
    def device(self):
        return self.A.device

    @classmethod
    def from_packed(cls, m, n, A, b, c, device="cuda", dtype=torch.float64, max_m=None, max_n=None):
        """Build from host arrays (``A``, ``b``, ``c`` flat and packed in LP order)."""
        m = np.asarray(m, dtype=np.int32); n = np.asarray(n, dtype=np.int32)
        mn = m.astype(np.int64) * n.astype(np.int64)
        offs = [np.zeros(len(m), dtype=np.int64) for _ in range(3)]
        if len(m):
            offs[0][1:] = np.cumsum(mn)[:-1]
            offs[1][1:] = np.cumsum(m.astype(np.int64))[:-1]
            offs[2][1:] = np.cumsum(n.astype(np.int64))[:-1]
        dev = torch.device(device)
        to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dt)
        return cls(to(m, torch.int32), to(n, torch.int32), to(offs[0], torch.int64), to(offs[1], torch.int64),
                   to(offs[2], torch.int64), to(A, dtype), to(b, dtype), to(c, dtype),
                   max_m if max_m is not None else (int(m.max()) if len(m) else 1),
                   max_n if max_n is not None else (int(n.max()) if len(n) else 1),
                   int(m.min()) if len(m) else 0, int(n.min()) if len(n) else 0)

    def pin_memory(self) -> "LPBatch":
        """A copy of a host batch in page-locked memory (for ``Solver.solve_host``)."""
        t = [x.pin_memory() for x in (self.m, self.n, self.a_off, self.b_off, self.c_off, self.A, self.b, self.c)]
        return LPBatch(*t, self.max_m, self.max_n, self.min_m, self.min_n)

    @classmethod
    def from_dense(cls, A: torch.Tensor, b: torch.Tensor, c: torch.Tensor):
        """Fixed-size batch from device tensors ``A[count, m, n]``, ``b[count, m]``, ``c[count, n]``."""
        count, m, n = A.shape
        dev = A.device
        ar = torch.arange(count, device=dev, dtype=torch.int64)
        return cls(torch.full((count,), m, dtype=torch.int32, device=dev),
                   torch.full((count,), n, dtype=torch.int32, device=dev),
                   ar * (m * n), ar * m, ar * n, A.contiguous().view(-1), b.contiguous().view(-1),
                   c.contiguous().view(-1), m, n, m, n)

    def cstruct(self) -> _lib.Batch:
        dt = {torch.float32: _lib.DTYPE_F32, torch.float64: _lib.DTYPE_F64}[self.A.dtype]
        assert self.b.dtype == self.A.dtype and self.c.dtype == self.A.dtype
        return _lib.Batch(self.count, self.max_m, self.max_n, dt, _ptr(self.m), _ptr(self.n), _ptr(self.a_off),
                          _ptr(self.b_off), _ptr(self.c_off), _ptr(self.A), _ptr(self.b), _ptr(self.c),
                          self.min_m, self.min_n)


@dataclass
class SolveResult:
    status: torch.Tensor   # int32 [count]
    iters: torch.Tensor    # int32 [count]
    obj: torch.Tensor      # float64 [count]
    x: torch.Tensor        # float64, packed like c
    y: torch.Tensor        # float64, packed like b
    basis: torch.Tensor    # int32, packed like b

    def cstruct(self) -> _lib.Result:
        return _lib.Result(_ptr(self.status), _ptr(self.iters), _ptr(self.obj), _ptr(self.x), _ptr(self.y),
                           _ptr(self.basis))


class Solver:
    """A liblpb handle bound to one CUDA device, with a reusable workspace."""

    def __init__(self, device=0):
        self.lib = _lib.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        h = ctypes.c_void_p()
        _lib.check(self.lib.lpb_create(ctypes.byref(h), self.device.index or 0), "lpb_create")
        self.h = h
        self._ws = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- options / workspace ------------------------------------------------
    @staticmethod
    def options(prec="fp32_refine", max_iter=0, eps_p=0.0, eps_d=0.0, feas_tol=0.0, kernel=KERNEL_AUTO,
                threads=0, keep_basis_inverse=0, reg_warps=0, pivot_rule="lpc", seed=0) -> _lib.Options:
        p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        rule = PIVOT_RULES[pivot_rule] if isinstance(pivot_rule, str) else int(pivot_rule)
        return _lib.Options(p, int(max_iter), float(eps_p), float(eps_d), float(feas_tol),
                            int(keep_basis_inverse), int(kernel), int(threads), int(reg_warps), rule,
                            int(seed) & 0xFFFFFFFFFFFFFFFF)

    def workspace_size(self, batch: LPBatch, opt: _lib.Options) -> int:
        n = ctypes.c_size_t()
        cb = batch.cstruct()
        _lib.check(self.lib.lpb_workspace_size(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(n)),
                   "lpb_workspace_size")
        return int(n.value)

    def workspace(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def alloc_result(self, batch: LPBatch) -> SolveResult:
        dev = batch.device
        return SolveResult(torch.empty(batch.count, dtype=torch.int32, device=dev),
                           torch.empty(batch.count, dtype=torch.int32, device=dev),
                           torch.empty(batch.count, dtype=torch.float64, device=dev),
                           torch.empty(batch.c.numel(), dtype=torch.float64, device=dev),
                           torch.empty(batch.b.numel(), dtype=torch.float64, device=dev),
                           torch.empty(batch.b.numel(), dtype=torch.int32, device=dev))

    # -- calls --------------------------------------------------------------
    def solve(self, batch: LPBatch, prec="fp32_refine", out: SolveResult | None = None, **kw) -> SolveResult:
        """Solve every LP of ``batch`` on the current stream (asynchronous)."""
        opt = self.options(prec, **kw)
        res = out if out is not None else self.alloc_result(batch)
        ws = self.workspace(self.workspace_size(batch, opt))
        cb, cr = batch.cstruct(), res.cstruct()
        _lib.check(self.lib.lpb_solve(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(cr),
                                      _ptr(ws), ws.numel(), _stream_handle(self.device)), "lpb_solve")
        return res

    def alloc_host_result(self, batch: LPBatch) -> SolveResult:
        """Page-locked host result arrays for ``solve_host``."""
        pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory()
        return SolveResult(pin(batch.count, torch.int32), pin(batch.count, torch.int32),
                           pin(batch.count, torch.float64), pin(batch.c.numel(), torch.float64),
                           pin(batch.b.numel(), torch.float64), pin(batch.b.numel(), torch.int32))

    def solve_host(self, batch: LPBatch, prec="fp32_refine", chunk: int = 8192, out: SolveResult | None = None,
                   **kw) -> SolveResult:
        """Solve a batch held in (page-locked) host memory through the chunked copy / solve /
        copy-back pipeline of lpb_solve_host, on the current stream (asynchronous: synchronise
        the stream before reading the results)."""
        if batch.A.device.type != "cpu":
            raise ValueError("solve_host takes a batch in host memory (LPBatch.from_packed(..., device='cpu'))")
        opt = self.options(prec, **kw)
        res = out if out is not None else self.alloc_host_result(batch)
        cb, cr = batch.cstruct(), res.cstruct()
        n = ctypes.c_size_t()
        _lib.check(self.lib.lpb_workspace_size_host(self.h, ctypes.byref(cb), ctypes.byref(opt), int(chunk),
                                                    ctypes.byref(n)), "lpb_workspace_size_host")
        ws = self.workspace(int(n.value))
        _lib.check(self.lib.lpb_solve_host(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(cr), int(chunk),
                                           _ptr(ws), ws.numel(), _stream_handle(self.device)), "lpb_solve_host")
        return res

    def solve_shared(self, A: torch.Tensor, b: torch.Tensor, C: torch.Tensor, prec="fp32_refine",
                     out: SolveResult | None = None, **kw) -> SolveResult:
        """Support function of one polytope ``{A x <= b, x >= 0}`` in every direction of
        ``C[count, n]`` (lpb_solve_shared): x of direction k at ``k n``, y and basis at ``k m``."""
        m, n = A.shape
        count = C.shape[0]
        dt = {torch.float32: _lib.DTYPE_F32, torch.float64: _lib.DTYPE_F64}[A.dtype]
        if b.dtype != A.dtype or C.dtype != A.dtype or C.shape[1] != n or b.numel() != m:
            raise ValueError("A (m x n), b (m) and C (count x n) must share one dtype")
        A, b, C = A.contiguous(), b.contiguous(), C.contiguous()
        opt = self.options(prec, **kw)
        dev = A.device
        res = out if out is not None else SolveResult(
            torch.empty(count, dtype=torch.int32, device=dev), torch.empty(count, dtype=torch.int32, device=dev),
            torch.empty(count, dtype=torch.float64, device=dev), torch.empty(count * n, dtype=torch.float64, device=dev),
            torch.empty(count * m, dtype=torch.float64, device=dev), torch.empty(count * m, dtype=torch.int32, device=dev))
        nb = ctypes.c_size_t()
        _lib.check(self.lib.lpb_workspace_size_shared(self.h, m, n, dt, count, ctypes.byref(opt), ctypes.byref(nb)),
                   "lpb_workspace_size_shared")
        ws = self.workspace(int(nb.value))
        cr = res.cstruct()
        _lib.check(self.lib.lpb_solve_shared(self.h, m, n, dt, _ptr(A), _ptr(b), count, _ptr(C), ctypes.byref(opt),
                                             ctypes.byref(cr), _ptr(ws), ws.numel(), _stream_handle(self.device)),
                   "lpb_solve_shared")
        return res

    def solve_bounded(self, batch: LPBatch, l: torch.Tensor, u: torch.Tensor, prec="fp32_refine",
                      out: SolveResult | None = None, **kw) -> SolveResult:
        """Every LP ``max c^T x, A x <= b, l <= x <= u`` of an FP64 ``batch`` (lpb_solve_bounded);
        ``l`` (finite) and ``u`` (``+inf`` allowed) are packed like ``c``.  The result has no basis."""
        if l.dtype != torch.float64 or u.dtype != torch.float64 or batch.A.dtype != torch.float64:
            raise ValueError("solve_bounded takes an FP64 batch and FP64 bounds")
        opt = self.options(prec, **kw)
        dev = batch.device
        res = out if out is not None else SolveResult(
            torch.empty(batch.count, dtype=torch.int32, device=dev), torch.empty(batch.count, dtype=torch.int32, device=dev),
            torch.empty(batch.count, dtype=torch.float64, device=dev),
            torch.empty(batch.c.numel(), dtype=torch.float64, device=dev),
            torch.empty(batch.b.numel(), dtype=torch.float64, device=dev), None)
        cb, cr = batch.cstruct(), res.cstruct()
        nb = ctypes.c_size_t()
        _lib.check(self.lib.lpb_workspace_size_bounded(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(nb)),
                   "lpb_workspace_size_bounded")
        ws = self.workspace(int(nb.value))
        _lib.check(self.lib.lpb_solve_bounded(self.h, ctypes.byref(cb), _ptr(l.contiguous()), _ptr(u.contiguous()),
                                              ctypes.byref(opt), ctypes.byref(cr), _ptr(ws), ws.numel(),
                                              _stream_handle(self.device)), "lpb_solve_bounded")
        return res

    def autotune(self, batch: LPBatch, prec="fp32_refine", table_path: str | None = None,
                 out: SolveResult | None = None, **kw) -> float:
        """Pick the fastest schedule for batches shaped like ``batch`` (lpb_autotune); later solves
        with default options use it.  Returns the winner's ms per solve (0 if loaded from the table)."""
        opt = self.options(prec, **kw)
        res = out if out is not None else self.alloc_result(batch)
        ws = self.workspace(self.workspace_size(batch, opt))
        cb, cr = batch.cstruct(), res.cstruct()
        ms = ctypes.c_float()
        path = None if table_path is None else str(table_path).encode()
        _lib.check(self.lib.lpb_autotune(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(cr), _ptr(ws),
                                         ws.numel(), path, _stream_handle(self.device), ctypes.byref(ms)),
                   "lpb_autotune")
        return float(ms.value)

    def solve_backward(self, batch: LPBatch, res: SolveResult, g_obj: torch.Tensor | None,
                       g_x: torch.Tensor | None):
        """Vector-Jacobian product through the optimal basis of ``res`` (see lpb_solve_backward).
        Returns FP64 ``(g_c, g_b, g_A)`` packed like ``c``, ``b`` and ``A``."""
        dev = batch.device
        g_c = torch.empty(batch.c.numel(), dtype=torch.float64, device=dev)
        g_b = torch.empty(batch.b.numel(), dtype=torch.float64, device=dev)
        g_A = torch.empty(batch.A.numel(), dtype=torch.float64, device=dev)
        if g_obj is not None:
            g_obj = g_obj.to(torch.float64).contiguous()
        if g_x is not None:
            g_x = g_x.to(torch.float64).contiguous()
        opt = self.options()
        ws = self.workspace(self.workspace_size(batch, opt))
        cb, cr = batch.cstruct(), res.cstruct()
        _lib.check(self.lib.lpb_solve_backward(self.h, ctypes.byref(cb), ctypes.byref(opt), ctypes.byref(cr),
                                               _ptr(g_obj), _ptr(g_x), _ptr(g_c), _ptr(g_b), _ptr(g_A), _ptr(ws),
                                               ws.numel(), _stream_handle(self.device)), "lpb_solve_backward")
        return g_c, g_b, g_A

    def hyperbox(self, c: torch.Tensor, l: torch.Tensor, u: torch.Tensor, want_x: bool = False,
                 obj: torch.Tensor | None = None, x: torch.Tensor | None = None):
        """Support functions over boxes (Section 6, Eq. 8): ``c[count, n]`` with ``l, u`` of
        shape ``[count, n]`` (per-LP boxes) or ``[n]`` (one shared box)."""
        count, n = c.shape
        shared = l.dim() == 1
        dt = {torch.float32: _lib.DTYPE_F32, torch.float64: _lib.DTYPE_F64}[c.dtype]
        assert l.dtype == c.dtype and u.dtype == c.dtype and l.shape == u.shape
        assert c.is_contiguous() and l.is_contiguous() and u.is_contiguous()
        obj = obj if obj is not None else torch.empty(count, dtype=c.dtype, device=c.device)
        if want_x and x is None:
            x = torch.empty_like(c)
        _lib.check(self.lib.lpb_hyperbox(self.h, count, n, dt, _ptr(c), _ptr(l), _ptr(u), int(shared), _ptr(obj),
                                         _ptr(x) if want_x else None, _stream_handle(self.device)),
                   "lpb_hyperbox")
        return (obj, x) if want_x else obj

    def stats(self) -> dict:
        st = _lib.Stats()
        _lib.check(self.lib.lpb_get_stats(self.h, _stream_handle(self.device), ctypes.byref(st)), "lpb_get_stats")
        return {"resolved_fp64": int(st.resolved_fp64), "deferred": int(st.deferred), "kernels": int(st.kernels)}

    def profile_start(self, calls: int):
        """Record per-pass kernel times (CUDA events on the solve's stream) for the next calls."""
        _lib.check(self.lib.lpb_profile_start(self.h, int(calls)), "lpb_profile_start")

    def profile_read(self, max_calls: int = 256) -> np.ndarray:
        """[calls, 3] milliseconds of passes 0-2 of each recorded lpb_solve call."""
        buf = (ctypes.c_float * (3 * max_calls))()
        n = ctypes.c_int32()
        _lib.check(self.lib.lpb_profile_read(self.h, buf, int(max_calls), ctypes.byref(n)), "lpb_profile_read")
        return np.frombuffer(buf, dtype=np.float32, count=3 * n.value).reshape(n.value, 3).copy()

    def sync_error(self) -> int:
        w = ctypes.c_uint32()
        code = self.lib.lpb_sync_error(self.h, _stream_handle(self.device), ctypes.byref(w))
        if code not in (_lib.OK, _lib.EDEVICE):
            _lib.check(code, "lpb_sync_error")
        return int(w.value)


from .autograd import solve  # noqa: E402  (differentiable solve; needs Solver and LPBatch above)

__all__.append("solve")
