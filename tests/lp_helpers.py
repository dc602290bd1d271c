"""Helpers shared by the GPU parity tests: move synthetic batches to the device, run
the oracle on the same LPs, and compare results the way the solver is specified:
statuses exactly, objectives to a relative tolerance, x* and y only where the
oracle certifies the optimum unique, and the GPU's own (x, y) by KKT in FP64."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from oracle import certify


def to_device(sb, dtype=torch.float64, device="cuda", max_m=None, max_n=None):
    from paper_1609_08114_gb300 import LPBatch
    return LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=device, dtype=dtype, max_m=max_m, max_n=max_n)


def host(res):
    torch.cuda.synchronize()
    return {k: getattr(res, k).cpu().numpy() for k in ("status", "iters", "obj", "x", "y", "basis")}


def rel_vec_err(v, ref):
    """Norm-wise relative error of a vector: max|v - ref| / (1 + max|ref|)."""
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(v - ref)) / (1.0 + np.max(np.abs(ref))))


def compare(sb, got, ref=None, obj_rtol=1e-9, kkt_tol=1e-8, check_unique=True, data_dtype=np.float64,
            vec_rtol=None):
    """Assert parity of GPU results `got` with the oracle on batch `sb`.

    Statuses exactly; objectives to `obj_rtol` relative; on LPs whose optimum the oracle
    certifies unique, x* and y to `vec_rtol` (default: `obj_rtol`) in the norm-wise
    relative sense max|v - v_ref| / (1 + max|v_ref|); and KKT of the GPU's own (x, y)."""
    vec_rtol = obj_rtol if vec_rtol is None else vec_rtol
    if ref is None:
        ref = oracle.solve_batch(sb)
    st_g, st_r = got["status"], ref["status"]
    bad = np.nonzero(st_g != st_r)[0]
    assert bad.size == 0, f"status mismatch at LPs {bad[:10]}: gpu {st_g[bad[:10]]} oracle {st_r[bad[:10]]}"
    opt = np.nonzero(st_r == 0)[0]
    rel = np.abs(got["obj"][opt] - ref["obj"][opt]) / (1.0 + np.abs(ref["obj"][opt]))
    assert rel.size == 0 or rel.max() <= obj_rtol, f"obj rel err {rel.max():.3e} at LP {opt[rel.argmax()]}"
    n_unique = 0
    for k in opt:
        A, b, c = sb.lp(int(k))
        A = A.astype(data_dtype).astype(np.float64); b = b.astype(data_dtype).astype(np.float64)
        c = c.astype(data_dtype).astype(np.float64)
        m, n = A.shape
        x = got["x"][sb.c_off[k]:sb.c_off[k] + n]
        y = got["y"][sb.b_off[k]:sb.b_off[k] + m]
        assert certify.is_optimal_pair(A, b, c, x, y, tol=kkt_tol), f"KKT fails for LP {k}"
        if check_unique:
            xr = ref["x"][sb.c_off[k]:sb.c_off[k] + n]
            yr = ref["y"][sb.b_off[k]:sb.b_off[k] + m]
            br = ref["basis"][sb.b_off[k]:sb.b_off[k] + m]
            if certify.nondegenerate(A, b, c, xr, yr, br):
                n_unique += 1
                ex, ey = rel_vec_err(x, xr), rel_vec_err(y, yr)
                assert ex <= vec_rtol, f"x* rel err {ex:.3e} > {vec_rtol:.0e} at LP {k}"
                assert ey <= vec_rtol, f"y rel err {ey:.3e} > {vec_rtol:.0e} at LP {k}"
    return ref, n_unique
