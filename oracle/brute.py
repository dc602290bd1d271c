"""Brute-force LP solution by enumerating bases -- TEST INFRASTRUCTURE ONLY.

For ``max c^T x, A x <= b, x >= 0`` with slacks ``s = b - A x >= 0`` (Section 3,
Eq. 4) the feasible region is a pointed polyhedron, so if it is non-empty it has
a vertex, and a vertex is a basic feasible solution: ``m`` of the ``n + m``
variables ``(x, s)`` solve ``[A I] z = b`` with the others at zero, and all are
non-negative.  The LP is

* infeasible iff no basis gives a feasible solution;
* unbounded iff it is feasible and some extreme ray ``d`` of the recession cone
  ``{d >= 0, A d <= 0}`` has ``c^T d > 0``; the extreme rays are the vertices of
  ``{(d, t) >= 0 : A d + t = 0, sum(d) = 1}``, enumerated the same way;
* otherwise optimal with value ``max c^T x`` over the vertices.

This uses nothing of the simplex method and is exponential: it is meant for
``m + n <= 12`` or so.
"""
from __future__ import annotations

import itertools

import numpy as np

OPTIMAL, INFEASIBLE, UNBOUNDED = 0, 1, 2


def _basic_solutions(M: np.ndarray, rhs: np.ndarray, tol: float):
    rows, cols = M.shape
    for S in itertools.combinations(range(cols), rows):
        B = M[:, S]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        zB = np.linalg.solve(B, rhs)
        if np.all(zB >= -tol):
            z = np.zeros(cols)
            z[list(S)] = zB
            yield z


def vertices(A, b, tol: float = 1e-9):
    """All vertices ``x`` (structural part) of ``{A x <= b, x >= 0}``."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    M = np.hstack([A, np.eye(m)])
    return [z[:n] for z in _basic_solutions(M, np.asarray(b, dtype=np.float64), tol)]


def extreme_rays(A, tol: float = 1e-9):
    """Extreme rays ``d`` (normalised to ``sum(d) = 1``) of ``{d >= 0, A d <= 0}``."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    M = np.vstack([np.hstack([A, np.eye(m)]), np.hstack([np.ones((1, n)), np.zeros((1, m))])])
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    return [z[:n] for z in _basic_solutions(M, rhs, tol)]


def solve(A, b, c, tol: float = 1e-9):
    """Return ``(status, obj, x)`` by enumeration (``x`` is one maximising vertex)."""
    c = np.asarray(c, dtype=np.float64)
    V = vertices(A, b, tol)
    if not V:
        return INFEASIBLE, -np.inf, None
    for d in extreme_rays(A, tol):
        if float(c @ d) > tol:
            return UNBOUNDED, np.inf, None
    vals = [float(c @ v) for v in V]
    k = int(np.argmax(vals))
    return OPTIMAL, vals[k], V[k]


def solve_box(A, b, c, l, u, tol: float = 1e-9):
    """Return ``(status, obj, x)`` for ``max c^T x, A x <= b, l <= x <= u`` with finite
    bounds by enumeration: the region is a polytope, so it is empty (infeasible) or
    ``c^T x`` attains its maximum at a vertex, where ``n`` linearly independent
    constraints of ``G x <= h`` (the rows of A, x <= u and -x <= -l) are tight."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    G = np.vstack([A, np.eye(n), -np.eye(n)])
    h = np.concatenate([np.asarray(b, dtype=np.float64), np.asarray(u, dtype=np.float64),
                        -np.asarray(l, dtype=np.float64)])
    c = np.asarray(c, dtype=np.float64)
    best, bx = -np.inf, None
    for S in itertools.combinations(range(G.shape[0]), n):
        Gs = G[list(S)]
        if abs(np.linalg.det(Gs)) < 1e-12:
            continue
        x = np.linalg.solve(Gs, h[list(S)])
        if np.all(G @ x <= h + tol * (1 + np.abs(h))):
            v = float(c @ x)
            if v > best:
                best, bx = v, x
    if bx is None:
        return INFEASIBLE, -np.inf, None
    return OPTIMAL, best, bx
