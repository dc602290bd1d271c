"""CPU oracle for the batched LP solver -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 implementations of what the solver computes, written from
the paper and independent of the CUDA path (no shared code, headers or
helpers).  Only the tests, the package's ``smoke()`` check and the
benchmark's CPU-baseline leg may import this package.

* :func:`solve_batch` / :func:`solve_one` -- the two-phase dense-tableau simplex
  of Section 3 (``simplex_oracle.c``, compiled with gcc, OpenMP over LPs).
* :func:`solve_bounded_batch` -- ``l <= x <= u`` in place of ``x >= 0``, by the change of
  variables ``x = l + z`` and one row ``z_j <= u_j - l_j`` per finite upper bound.
* :mod:`oracle.brute` -- vertex / extreme-ray enumeration for tiny LPs.
* :mod:`oracle.hyperbox` -- the closed form of Section 6, Eq. 8, in a fixed
  summation order.
* :mod:`oracle.certify` -- KKT, strong-duality, Farkas and ray checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

OPTIMAL, INFEASIBLE, UNBOUNDED, ITER_LIMIT, NUMERIC = 0, 1, 2, 3, 4
# Pivot rules of Section 4.2: most negative reduced cost (LPC, Dantzig) or a random eligible
# column (RPC; the random draw is a counter-based SplitMix64 key, see simplex_oracle.c); and
# steepest-edge pricing with exact tableau weights (SE; not in the paper, see simplex_oracle.c).
LPC, RPC, SE = 0, 1, 2
STATUS_NAMES = {0: "optimal", 1: "infeasible", 2: "unbounded", 3: "iter_limit", 4: "numeric"}

# Tolerances of the FP64 oracle (the paper states none): absolute, on data of order 1.
EPS_P = 1e-9       # pivot-column entries must exceed this to be eligible in Step 2
EPS_D = 1e-9       # reduced costs must be below -EPS_D to be eligible in Step 1
FEAS_TOL = 1e-9    # Phase I: infeasible when sum(artificials) > FEAS_TOL * (1 + max|b|)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``simplex_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _declare(lib):
    P = ctypes.c_void_p
    lib.oracle_solve_one.restype = ctypes.c_int
    lib.oracle_solve_one.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     P, P, P, P, P, P]
    lib.oracle_solve_batch.restype = None
    lib.oracle_solve_batch.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, P, P, P, P, P, P]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_solve_one_rule.restype = ctypes.c_int
    lib.oracle_solve_one_rule.argtypes = lib.oracle_solve_one.argtypes + [ctypes.c_int, ctypes.c_uint64,
                                                                          ctypes.c_int64]
    lib.oracle_solve_batch_rule.restype = None
    lib.oracle_solve_batch_rule.argtypes = lib.oracle_solve_batch.argtypes + [ctypes.c_int, ctypes.c_uint64,
                                                                              ctypes.c_int64]
    lib.oracle_splitmix64_next.restype = ctypes.c_uint64
    lib.oracle_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def load_variant(path: str):
    """Load another build of ``simplex_oracle.c`` (the tests compile mutated copies
    to check that the pins catch planted mistakes)."""
    return _declare(ctypes.CDLL(path))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def splitmix64(state: int, count: int):
    """The first ``count`` outputs of the oracle's SplitMix64 generator from ``state``."""
    st = ctypes.c_uint64(state)
    return [int(_load().oracle_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def solve_one(A, b, c, max_iter: int = 0, eps_p: float = EPS_P, eps_d: float = EPS_D,
              feas_tol: float = FEAS_TOL, lib=None, rule: int = LPC, seed: int = 0, lp: int = 0):
    """Solve ``max c^T x, A x <= b, x >= 0`` for one LP.

    Returns a dict with ``status, x, y, obj, basis, iters, cert`` (``cert`` is a
    ray over structurals+slacks when unbounded, a Farkas vector over the rows
    when infeasible).
    """
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(m)
    c = np.ascontiguousarray(c, dtype=np.float64).reshape(n)
    x = np.zeros(n); y = np.zeros(m); obj = np.zeros(1)
    basis = np.zeros(max(m, 1), dtype=np.int32); iters = np.zeros(1, dtype=np.int32)
    cert = np.zeros(n + m)
    L = lib or _load()
    if rule == LPC:
        st = L.oracle_solve_one(m, n, _p(A), _p(b), _p(c), int(max_iter), eps_p, eps_d, feas_tol,
                                _p(x), _p(y), _p(obj), _p(basis), _p(iters), _p(cert))
    else:
        st = L.oracle_solve_one_rule(m, n, _p(A), _p(b), _p(c), int(max_iter), eps_p, eps_d, feas_tol,
                                     _p(x), _p(y), _p(obj), _p(basis), _p(iters), _p(cert), int(rule),
                                     int(seed), int(lp))
    return dict(status=int(st), x=x, y=y, obj=float(obj[0]), basis=basis[:m].copy(),
                iters=int(iters[0]), cert=cert)


def solve_batch(batch, max_iter: int = 0, eps_p: float = EPS_P, eps_d: float = EPS_D,
                feas_tol: float = FEAS_TOL, nthreads: int = 0, rule: int = LPC, seed: int = 0,
                first_lp: int = 0):
    """Solve every LP of a packed batch (``m, n, a_off, b_off, c_off, A, b, c``).

    Outputs follow the batch's packing: ``x`` like ``c``, ``y`` and ``basis`` like
    ``b``, and one ``status``, ``obj`` and ``iters`` per LP.  Under ``rule=RPC`` LP k
    of the batch draws its random keys as LP ``first_lp + k`` with ``seed``.
    """
    cnt = len(batch.m)
    m = np.ascontiguousarray(batch.m, dtype=np.int32)
    n = np.ascontiguousarray(batch.n, dtype=np.int32)
    a_off = np.ascontiguousarray(batch.a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(batch.b_off, dtype=np.int64)
    c_off = np.ascontiguousarray(batch.c_off, dtype=np.int64)
    A = np.ascontiguousarray(batch.A, dtype=np.float64)
    b = np.ascontiguousarray(batch.b, dtype=np.float64)
    c = np.ascontiguousarray(batch.c, dtype=np.float64)
    status = np.zeros(cnt, dtype=np.int32); iters = np.zeros(cnt, dtype=np.int32)
    obj = np.zeros(cnt); x = np.zeros(c.size); y = np.zeros(b.size)
    basis = np.zeros(max(b.size, 1), dtype=np.int32)
    if cnt:
        _load().oracle_solve_batch_rule(cnt, _p(m), _p(n), _p(a_off), _p(b_off), _p(c_off), _p(A), _p(b),
                                        _p(c), int(max_iter), eps_p, eps_d, feas_tol, int(nthreads),
                                        _p(status), _p(x), _p(y), _p(obj), _p(basis), _p(iters), int(rule),
                                        int(seed), int(first_lp))
    return dict(status=status, x=x, y=y, obj=obj, basis=basis[:b.size], iters=iters)


def solve_bounded_batch(batch, l, u, nthreads: int = 0, **kw):
    """Every LP ``max c^T x, A x <= b, l <= x <= u`` of a packed batch, ``l`` and ``u``
    packed like ``c`` (``l`` finite, ``u`` may be ``+inf``).  With ``x = l + z`` the LP
    is ``max c^T z + c^T l`` subject to ``A z <= b - A l``, ``z_j <= u_j - l_j`` for every
    finite ``u_j`` and ``z >= 0``, which :func:`solve_batch` solves; the results map back
    to ``x = l + z``, ``obj + c^T l`` and the duals of the rows of ``A``."""
    import synth
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lps, fin = [], []
    for k in range(len(batch.m)):
        A, b, c = batch.lp(k)
        m, n = A.shape
        lk = l[batch.c_off[k]:batch.c_off[k] + n]
        uk = u[batch.c_off[k]:batch.c_off[k] + n]
        f = np.isfinite(uk)
        A2 = np.vstack([A, np.eye(n)[f]])
        b2 = np.concatenate([b - A @ lk, (uk - lk)[f]])
        lps.append((A2, b2, c))
        fin.append((m, n, lk, c))
    r = solve_batch(synth.pack(lps), nthreads=nthreads, **kw)
    cnt = len(batch.m)
    out = dict(status=r["status"].copy(), obj=r["obj"].copy(), iters=r["iters"].copy(),
               x=np.zeros(np.asarray(batch.c).size), y=np.zeros(np.asarray(batch.b).size))
    xo = yo = 0
    for k in range(cnt):
        m, n, lk, c = fin[k]
        m2 = lps[k][0].shape[0]
        if out["status"][k] == OPTIMAL:
            out["x"][batch.c_off[k]:batch.c_off[k] + n] = r["x"][xo:xo + n] + lk
            out["y"][batch.b_off[k]:batch.b_off[k] + m] = r["y"][yo:yo + m]
            out["obj"][k] += float(c @ lk)
        xo += n
        yo += m2
    return out
