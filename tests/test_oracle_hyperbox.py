"""Pins of the hyperbox oracle (Section 6, Eq. 8)."""
import numpy as np

import synth
from oracle import hyperbox


def test_closed_form_equals_vertex_enumeration():
    rng = np.random.default_rng(0)
    for n in range(1, 9):
        c = rng.normal(size=(20, n)); l = rng.uniform(-10, 0, size=(20, n)); u = rng.uniform(0, 10, size=(20, n))
        obj, h = hyperbox.support(c, l, u)
        for k in range(20):
            assert abs(obj[k] - hyperbox.support_by_vertices(c[k], l[k], u[k])) <= 1e-12 * (1 + abs(obj[k]))
            # the maximiser is a vertex and attains the value
            assert abs(c[k] @ h[k] - obj[k]) <= 1e-12 * (1 + abs(obj[k]))


def test_shared_box_matches_per_lp_box():
    c, l, u = synth.hyperbox(500, 7, seed=1, shared_box=True)
    o1, _ = hyperbox.support(c, l, u)
    o2, _ = hyperbox.support(c, np.broadcast_to(l, c.shape), np.broadcast_to(u, c.shape))
    assert np.array_equal(o1, o2)


def test_tie_rule_and_signed_zero():
    """c_i = 0 takes the upper bound (Eq. 8's 'otherwise'); the sum starts at +0.0, so
    an all-zero direction gives +0.0 even with negative lower bounds."""
    c = np.zeros((1, 3)); l = -np.ones(3); u = np.full(3, 2.0)
    obj, h = hyperbox.support(c, l, u)
    assert np.all(h == 2.0)
    assert obj[0] == 0.0 and not np.signbit(obj[0])
    c = np.array([[-0.0, 0.0]])
    obj, h = hyperbox.support(c, np.array([-3.0, -3.0]), np.array([5.0, 5.0]))
    assert np.all(h == 5.0) and not np.signbit(obj[0])


def test_fp32_order_is_sequential_and_unfused():
    """The float32 result equals a scalar loop with per-operation float32 rounding and
    differs (for some inputs) from a fused or reordered sum, so order matters."""
    rng = np.random.default_rng(4)
    c = rng.normal(size=(2000, 28)).astype(np.float32)
    l = rng.uniform(-10, 0, size=(2000, 28)).astype(np.float32)
    u = rng.uniform(0, 10, size=(2000, 28)).astype(np.float32)
    obj, h = hyperbox.support(c, l, u)
    assert obj.dtype == np.float32
    for k in range(0, 2000, 97):
        acc = np.float32(0.0)
        for i in range(28):
            acc = np.float32(acc + np.float32(c[k, i] * h[k, i]))
        assert obj[k] == acc
    exact = (c.astype(np.float64) * h.astype(np.float64)).sum(axis=1)
    pairwise = (c * h).sum(axis=1, dtype=np.float32)
    assert np.any(pairwise != obj)          # a different order rounds differently
    assert np.max(np.abs(obj - exact) / (1 + np.abs(exact))) < 1e-5
