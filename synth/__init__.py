"""Seeded synthetic LP batches shaped like the paper's workloads.

This module only draws random numbers and lays them out; it holds none of
the solver's arithmetic.  Both the CPU oracle (through the tests) and the
CUDA path (through the tests and the benchmark) take their inputs from here.

The paper never states how its random LPs were drawn (Section 4.7 and
Section 6 give only sizes), so the distributions below are this project's
choice:

* type 1 (initial slack basis feasible, Section 4.7): ``A ~ U[0.1, 1]``,
  ``b ~ U[1, 10]``, ``c ~ U[0, 1]``.  With ``A > 0`` and ``b > 0`` every such LP
  is bounded, feasible and optimal.
* type 2 (initial slack basis infeasible, Section 4.7): ``x0 ~ U[0, 1]^n``,
  ``A ~ U[0.1, 1]``; the first half of the rows are ``<=`` rows with
  ``b_i = A_i x0 + U[0, 1]``, the second half ``>=`` rows with
  ``b_i = A_i x0 - U[0, 0.5]`` written as ``-A_i x <= -b_i``.  About 5% of the
  LPs are made infeasible (the last two rows become a contradicting pair) and
  about 5% unbounded (one column of ``A`` zeroed before ``b`` is formed, with
  ``c_j ~ U[0.5, 1]``).
* hyperbox (Section 6, Eq. 8): ``l ~ U[-10, 0]``, ``u ~ U[0, 10]``,
  ``c ~ N(0, 1)``; per-LP boxes or one shared box.
* mixed sizes: ``m, n ~ U{8..256}`` independently with type-1 values.

Every batch is drawn in blocks; block ``k`` of a batch with seed ``s`` uses
``numpy.random.PCG64(SeedSequence([s, k]))`` so that any LP can be regenerated
on its own (the oracle checks samples of full-size batches this way).
"""
from __future__ import annotations

import numpy as np

LP_BLOCK = 256          # LPs per RNG block for the simplex workloads
BOX_BLOCK = 1 << 16     # LPs per RNG block for the hyperbox workloads

__all__ = [
    "type1", "type2", "hyperbox", "mixed_sizes", "pack", "LPBatch",
]


def _rng(seed: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(block)])))


class LPBatch:
    """A packed batch of LPs ``max c^T x, A x <= b, x >= 0``.

    ``A`` holds each LP's ``m x n`` matrix row-major at ``a_off[k]``; ``b`` and ``c``
    hold ``m`` and ``n`` values at ``b_off[k]`` and ``c_off[k]``.  ``kind`` is an
    int8 tag per LP (0 = regular, 1 = built infeasible, 2 = built unbounded)
    recording how the generator built it.
    """

    def __init__(self, m, n, A, b, c, kind=None):
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        mn = self.m.astype(np.int64) * self.n.astype(np.int64)
        self.a_off = np.zeros(len(self.m), dtype=np.int64)
        self.b_off = np.zeros(len(self.m), dtype=np.int64)
        self.c_off = np.zeros(len(self.m), dtype=np.int64)
        if len(self.m):
            self.a_off[1:] = np.cumsum(mn)[:-1]
            self.b_off[1:] = np.cumsum(self.m.astype(np.int64))[:-1]
            self.c_off[1:] = np.cumsum(self.n.astype(np.int64))[:-1]
        self.A = np.ascontiguousarray(A, dtype=np.float64).reshape(-1)
        self.b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        self.c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
        self.kind = (np.zeros(len(self.m), dtype=np.int8) if kind is None
                     else np.ascontiguousarray(kind, dtype=np.int8))
        assert self.A.size == int(mn.sum())
        assert self.b.size == int(self.m.sum()) and self.c.size == int(self.n.sum())

    @property
    def count(self) -> int:
        return len(self.m)

    def lp(self, k: int):
        """Return ``(A, b, c)`` of LP ``k`` as fresh float64 arrays."""
        m, n = int(self.m[k]), int(self.n[k])
        A = self.A[self.a_off[k]:self.a_off[k] + m * n].reshape(m, n).copy()
        return A, self.b[self.b_off[k]:self.b_off[k] + m].copy(), self.c[self.c_off[k]:self.c_off[k] + n].copy()

    def subset(self, idx) -> "LPBatch":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.lp(int(k)) for k in idx]
        if not parts:
            return LPBatch(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
        return LPBatch(self.m[idx], self.n[idx],
                       np.concatenate([p[0].ravel() for p in parts]),
                       np.concatenate([p[1] for p in parts]),
                       np.concatenate([p[2] for p in parts]), self.kind[idx])


def pack(lps) -> LPBatch:
    """Pack a list of ``(A, b, c)`` triples (any sizes) into an :class:`LPBatch`."""
    lps = list(lps)
    m = [np.asarray(A).shape[0] for A, _, _ in lps]
    n = [np.asarray(A).shape[1] for A, _, _ in lps]
    if not lps:
        return LPBatch(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    return LPBatch(m, n,
                   np.concatenate([np.asarray(A, dtype=np.float64).ravel() for A, _, _ in lps]),
                   np.concatenate([np.asarray(b, dtype=np.float64).ravel() for _, b, _ in lps]),
                   np.concatenate([np.asarray(c, dtype=np.float64).ravel() for _, _, c in lps]))


def _blocks(count: int, first: int, stop: int, bsz: int):
    for blk in range(first // bsz, (stop + bsz - 1) // bsz):
        lo, hi = blk * bsz, min((blk + 1) * bsz, count)
        yield blk, lo, hi


def type1(count: int, m: int, n: int, seed: int = 0, first: int = 0, stop: int | None = None) -> LPBatch:
    """Type-1 LPs (origin feasible), all ``m x n``.  LPs ``first..stop-1`` of the batch."""
    stop = count if stop is None else min(stop, count)
    As, bs, cs = [], [], []
    for blk, lo, hi in _blocks(count, first, stop, LP_BLOCK):
        g = _rng(seed, blk)
        k = hi - lo
        A = g.uniform(0.1, 1.0, size=(k, m, n))
        b = g.uniform(1.0, 10.0, size=(k, m))
        c = g.uniform(0.0, 1.0, size=(k, n))
        s0, s1 = max(first, lo) - lo, min(stop, hi) - lo
        As.append(A[s0:s1]); bs.append(b[s0:s1]); cs.append(c[s0:s1])
    cnt = stop - first
    if cnt <= 0:
        return pack([])
    return LPBatch(np.full(cnt, m), np.full(cnt, n), np.concatenate(As), np.concatenate(bs), np.concatenate(cs))


def type2(count: int, m: int, n: int, seed: int = 2, first: int = 0, stop: int | None = None,
          frac_infeasible: float = 0.05, frac_unbounded: float = 0.05) -> LPBatch:
    """Type-2 LPs (slack basis infeasible), built as described in the module docstring."""
    assert m >= 4
    stop = count if stop is None else min(stop, count)
    As, bs, cs, ks = [], [], [], []
    half = m // 2
    for blk, lo, hi in _blocks(count, first, stop, LP_BLOCK):
        g = _rng(seed, blk)
        k = hi - lo
        x0 = g.uniform(0.0, 1.0, size=(k, n))
        A = g.uniform(0.1, 1.0, size=(k, m, n))
        c = g.uniform(0.0, 1.0, size=(k, n))
        u_le = g.uniform(0.0, 1.0, size=(k, half))
        u_ge = g.uniform(0.0, 0.5, size=(k, m - half))
        sel = g.uniform(0.0, 1.0, size=k)
        zcol = g.integers(0, n, size=k)
        cz = g.uniform(0.5, 1.0, size=k)
        a_pair = g.uniform(0.1, 1.0, size=(k, n))
        beta_u = g.uniform(0.0, 1.0, size=k)
        kind = np.zeros(k, dtype=np.int8)
        kind[sel < frac_infeasible] = 1
        kind[(sel >= frac_infeasible) & (sel < frac_infeasible + frac_unbounded)] = 2
        for t in np.nonzero(kind == 2)[0]:
            A[t, :, zcol[t]] = 0.0
            c[t, zcol[t]] = cz[t]
        Ax0 = np.einsum("kij,kj->ki", A, x0)
        b = np.empty((k, m))
        b[:, :half] = Ax0[:, :half] + u_le
        b[:, half:] = -(Ax0[:, half:] - u_ge)
        A[:, half:, :] *= -1.0
        for t in np.nonzero(kind == 1)[0]:
            a = a_pair[t]
            beta = float(a @ x0[t]) + beta_u[t]
            A[t, m - 2, :] = a
            b[t, m - 2] = beta
            A[t, m - 1, :] = -a
            b[t, m - 1] = -(beta + 1.0)
        s0, s1 = max(first, lo) - lo, min(stop, hi) - lo
        As.append(A[s0:s1]); bs.append(b[s0:s1]); cs.append(c[s0:s1]); ks.append(kind[s0:s1])
    cnt = stop - first
    if cnt <= 0:
        return pack([])
    return LPBatch(np.full(cnt, m), np.full(cnt, n), np.concatenate(As), np.concatenate(bs),
                   np.concatenate(cs), np.concatenate(ks))


def mixed_sizes(count: int, seed: int = 4, lo: int = 8, hi: int = 256, first: int = 0,
                stop: int | None = None) -> LPBatch:
    """Type-1 values with ``m, n ~ U{lo..hi}`` drawn independently per LP."""
    stop = count if stop is None else min(stop, count)
    ms, ns, As, bs, cs = [], [], [], [], []
    for blk, b_lo, b_hi in _blocks(count, first, stop, LP_BLOCK):
        g = _rng(seed, blk)
        k = b_hi - b_lo
        mm = g.integers(lo, hi + 1, size=k)
        nn = g.integers(lo, hi + 1, size=k)
        for t in range(k):
            if not (first <= b_lo + t < stop):
                continue
            gi = _rng(seed, (1 << 32) + b_lo + t)
            A = gi.uniform(0.1, 1.0, size=(mm[t], nn[t]))
            b = gi.uniform(1.0, 10.0, size=mm[t])
            c = gi.uniform(0.0, 1.0, size=nn[t])
            ms.append(mm[t]); ns.append(nn[t]); As.append(A.ravel()); bs.append(b); cs.append(c)
    if not ms:
        return pack([])
    return LPBatch(np.array(ms), np.array(ns), np.concatenate(As), np.concatenate(bs), np.concatenate(cs))


def hyperbox(count: int, n: int, seed: int = 3, shared_box: bool = False, dtype=np.float64,
             first: int = 0, stop: int | None = None):
    """Hyperbox support-function LPs ``max c^T x, l <= x <= u``.

    Returns ``(c, l, u)`` with ``c`` of shape ``[count, n]``; ``l`` and ``u`` are
    ``[count, n]`` (per-LP boxes) or ``[n]`` (one shared box, the paper's setting in
    Section 6 where many objectives sample one box).
    """
    stop = count if stop is None else min(stop, count)
    cnt = max(stop - first, 0)
    c = np.empty((cnt, n), dtype=dtype)
    l = np.empty((n,) if shared_box else (cnt, n), dtype=dtype)
    u = np.empty_like(l)
    if shared_box:
        g = _rng(seed, (1 << 40))
        l[:] = g.uniform(-10.0, 0.0, size=n)
        u[:] = g.uniform(0.0, 10.0, size=n)
    for blk, lo, hi in _blocks(count, first, stop, BOX_BLOCK):
        g = _rng(seed, blk)
        k = hi - lo
        cb = g.standard_normal(size=(k, n))
        s0, s1 = max(first, lo) - lo, min(stop, hi) - lo
        d0 = lo + s0 - first
        c[d0:d0 + s1 - s0] = cb[s0:s1]
        if not shared_box:
            lb = g.uniform(-10.0, 0.0, size=(k, n))
            ub = g.uniform(0.0, 10.0, size=(k, n))
            l[d0:d0 + s1 - s0] = lb[s0:s1]
            u[d0:d0 + s1 - s0] = ub[s0:s1]
    return c, l, u
