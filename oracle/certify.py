"""Optimality and status certificates in FP64 -- TEST INFRASTRUCTURE ONLY.

These checks use only linear-programming duality for
``max c^T x, A x <= b, x >= 0`` (Section 3, Eq. 1-3) and its dual
``min b^T y, A^T y >= c, y >= 0``; they do not depend on how ``x`` and ``y``
were found.

* optimal:    ``x >= 0``, ``A x <= b``, ``y >= 0``, ``A^T y >= c`` and
  ``c^T x = b^T y`` (weak duality makes both optimal);
* unbounded:  a ray ``d >= 0``, ``A d <= 0``, ``c^T d > 0`` plus a feasible point;
* infeasible: a Farkas vector ``u >= 0``, ``A^T u >= 0``, ``b^T u < 0``.
"""
from __future__ import annotations

import numpy as np


def kkt_residuals(A, b, c, x, y):
    """Return the largest violations ``(primal, dual, gap)`` (scaled by 1 + data size)."""
    A = np.asarray(A, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64); x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sb = 1.0 + np.max(np.abs(b), initial=0.0)
    sc = 1.0 + np.max(np.abs(c), initial=0.0)
    primal = max(float(np.max(-x, initial=0.0)), float(np.max(A @ x - b, initial=0.0)) / sb)
    dual = max(float(np.max(-y, initial=0.0)), float(np.max(c - A.T @ y, initial=0.0)) / sc)
    gap = abs(float(c @ x) - float(b @ y)) / (1.0 + abs(float(c @ x)))
    return primal, dual, gap


def is_optimal_pair(A, b, c, x, y, tol: float = 1e-9) -> bool:
    return max(kkt_residuals(A, b, c, x, y)) <= tol


def is_ray(A, c, d, tol: float = 1e-9) -> bool:
    A = np.asarray(A, dtype=np.float64); d = np.asarray(d, dtype=np.float64)
    return (np.all(d >= -tol) and np.all(A @ d <= tol * (1 + np.abs(d).max()))
            and float(np.asarray(c) @ d) > tol)


def is_farkas(A, b, u, tol: float = 1e-9) -> bool:
    A = np.asarray(A, dtype=np.float64); u = np.asarray(u, dtype=np.float64)
    return (np.all(u >= -tol) and np.all(A.T @ u >= -tol * (1 + np.abs(u).max()))
            and float(np.asarray(b) @ u) < -tol)


def duals_from_basis(A, c, basis):
    """``y`` with ``B^T y = c_B`` for the basis (variable index per row; slacks are ``n + i``)."""
    A = np.asarray(A, dtype=np.float64); c = np.asarray(c, dtype=np.float64)
    m, n = A.shape
    M = np.hstack([A, np.eye(m)])
    cf = np.concatenate([c, np.zeros(m)])
    basis = np.asarray(basis)
    B = M[:, basis]
    return np.linalg.solve(B.T, cf[basis])


def primal_from_basis(A, b, basis):
    """Structural ``x`` with ``B x_B = b`` for the basis."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    M = np.hstack([A, np.eye(m)])
    basis = np.asarray(basis)
    zB = np.linalg.solve(M[:, basis], np.asarray(b, dtype=np.float64))
    x = np.zeros(n)
    for i, v in enumerate(basis):
        if v < n:
            x[v] = zB[i]
    return x


def nondegenerate(A, b, c, x, y, basis, margin: float = 1e-7) -> bool:
    """True when the optimum is unique in both ``x`` and ``y``: every basic variable is
    above ``margin`` and every non-basic reduced cost is above ``margin``."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    basis = np.asarray(basis)
    if np.any(basis < 0):
        return False
    z = np.concatenate([np.asarray(x, dtype=np.float64), np.asarray(b) - A @ np.asarray(x)])
    if np.any(z[basis] <= margin):
        return False
    red = np.concatenate([A.T @ np.asarray(y) - np.asarray(c), np.asarray(y)])
    nb = np.setdiff1d(np.arange(n + m), basis)
    return bool(np.all(red[nb] > margin))
