"""ctypes declarations of the liblpb C ABI (include/lpb.h).

Marshalling only: every computation runs in the CUDA kernels of liblpb.so.
Loading fails loudly when the library has not been built -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpb.so")

# lpb_status
OPTIMAL, INFEASIBLE, UNBOUNDED, ITER_LIMIT, NUMERIC, BAD_SIZE = 0, 1, 2, 3, 4, 5
# lpb_err
OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, EDEVICE = 0, -1, -2, -3, -4, -5
# lpb_precision
FP64, FP32_REFINE, FP32 = 0, 1, 2
# lpb_dtype
DTYPE_F32, DTYPE_F64 = 0, 1
# lpb_kernel
KERNEL_AUTO, KERNEL_SMEM, KERNEL_GMEM, KERNEL_REG, KERNEL_PACK, KERNEL_WARP = 0, 1, 2, 3, 4, 5
# lpb_pivot_rule
PIVOT_LPC, PIVOT_RPC, PIVOT_STEEPEST = 0, 1, 2

P = ctypes.c_void_p


class Batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("max_m", ctypes.c_int32), ("max_n", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("m", P), ("n", P), ("a_off", P), ("b_off", P),
                ("c_off", P), ("A", P), ("b", P), ("c", P), ("min_m", ctypes.c_int32), ("min_n", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", P), ("iters", P), ("obj", P), ("x", P), ("y", P), ("basis", P)]


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("eps_p", ctypes.c_double),
                ("eps_d", ctypes.c_double), ("feas_tol", ctypes.c_double),
                ("keep_basis_inverse", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("reg_warps", ctypes.c_int32), ("pivot_rule", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("resolved_fp64", ctypes.c_int64), ("deferred", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 5)]


# name -> (restype, argtypes); every symbol declared in include/lpb.h
SIGNATURES = {
    "lpb_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int]),
    "lpb_destroy": (ctypes.c_int, [P]),
    "lpb_workspace_size": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "lpb_solve": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options), ctypes.POINTER(Result),
                                 P, ctypes.c_size_t, P]),
    "lpb_solve_backward": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                          ctypes.POINTER(Result), P, P, P, P, P, P, ctypes.c_size_t, P]),
    "lpb_workspace_size_host": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options), ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "lpb_solve_host": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options), ctypes.POINTER(Result),
                                      ctypes.c_int32, P, ctypes.c_size_t, P]),
    "lpb_workspace_size_shared": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                 ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_size_t)]),
    "lpb_solve_shared": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int64, P,
                                        ctypes.POINTER(Options), ctypes.POINTER(Result), P, ctypes.c_size_t, P]),
    "lpb_workspace_size_bounded": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "lpb_solve_bounded": (ctypes.c_int, [P, ctypes.POINTER(Batch), P, P, ctypes.POINTER(Options),
                                         ctypes.POINTER(Result), P, ctypes.c_size_t, P]),
    "lpb_hyperbox": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P, P,
                                    ctypes.c_int32, P, P, P]),
    "lpb_autotune": (ctypes.c_int, [P, ctypes.POINTER(Batch), ctypes.POINTER(Options), ctypes.POINTER(Result), P,
                                    ctypes.c_size_t, ctypes.c_char_p, P, ctypes.POINTER(ctypes.c_float)]),
    "lpb_sync_error": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_uint32)]),
    "lpb_get_stats": (ctypes.c_int, [P, P, ctypes.POINTER(Stats)]),
    "lpb_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(Batch), ctypes.POINTER(Options), ctypes.POINTER(Result),
                                         P]),
    "lpb_noalloc_sync_error": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint32)]),
    "lpb_profile_start": (ctypes.c_int, [P, ctypes.c_int32]),
    "lpb_profile_read": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "lpb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lpb_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblpb.so and declare its symbols (raises if it is missing)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_1609_08114_gb300.build` "
            "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


class LPBError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = load().lpb_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


def check(code: int, what: str = ""):
    if code != OK:
        raise LPBError(code, what)
