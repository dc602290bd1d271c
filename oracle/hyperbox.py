"""Hyperbox support functions -- TEST INFRASTRUCTURE ONLY.

Section 6, Eq. 8: over the box ``l <= x <= u`` the maximum of ``c . x`` is
``sum_i c_i h_i`` with ``h_i = l_i`` when ``c_i < 0`` and ``h_i = u_i`` otherwise
(the paper writes the box as ``[a_i, b_i]`` and the direction as ``l``).

The sum is taken in index order ``i = 0, 1, ..., n-1`` starting from ``+0.0``;
each product ``c_i * h_i`` is rounded to the working precision and then added
(round to nearest even, no fused multiply-add).  NumPy's elementwise float32 /
float64 operations round each operation separately, so the loop below over
``i`` (vectorised across LPs only) is that definition.
"""
from __future__ import annotations

import itertools

import numpy as np


def support(c, l, u, dtype=None):
    """Return ``(obj, x)`` for LPs ``c[k]`` over boxes ``l[k], u[k]`` (or one shared box).

    ``c`` is ``[count, n]``; ``l, u`` are ``[count, n]`` or ``[n]``.  ``dtype`` is the
    working precision (default: ``c``'s dtype).
    """
    c = np.asarray(c)
    dt = np.dtype(dtype or c.dtype)
    c = c.astype(dt, copy=False)
    l = np.asarray(l).astype(dt, copy=False)
    u = np.asarray(u).astype(dt, copy=False)
    count, n = c.shape
    l2 = np.broadcast_to(l, (count, n))
    u2 = np.broadcast_to(u, (count, n))
    h = np.where(c < 0, l2, u2)
    acc = np.zeros(count, dtype=dt)               # +0.0
    for i in range(n):
        prod = np.multiply(c[:, i], h[:, i], dtype=dt)
        acc = np.add(acc, prod, dtype=dt)
    return acc, h


def support_by_vertices(c, l, u):
    """Brute force: the largest ``c . v`` over the ``2^n`` box vertices (FP64; n <= ~12)."""
    c = np.asarray(c, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    n = c.shape[-1]
    best = -np.inf
    for pick in itertools.product((0, 1), repeat=n):
        v = np.where(np.array(pick, dtype=bool), u, l)
        best = max(best, float(c @ v))
    return best
