"""Pins for the FP64 collision-cost reductions (min / soft-min / hinge).

Checked against brute force, scipy's logsumexp, the soft-min's bounds and
limits, and finite differences of the per-waypoint cost through the MLP.
"""
import numpy as np
import pytest
from scipy.special import logsumexp

import synth
from oracle import mlp, reduce as red


def test_min_first_occurrence_on_ties():
    f = np.array([0.3, -0.1, 0.2, -0.1, 0.5])
    dq = np.arange(10, dtype=np.float64).reshape(5, 2)
    c, g, a = red.reduce_waypoint(red.MIN, 0.0, f, dq, np.array([9, 4, 7, 2, 1]))
    assert c == -0.1 and a == 4
    np.testing.assert_array_equal(g, dq[1])


def test_softmin_against_logsumexp_and_bounds():
    rng = synth.SplitMix64(3)
    for T in (0.02, 0.1, 1.0):
        f = rng.uniform(50, -1, 2)
        dq = rng.uniform(150).reshape(50, 3)
        c, g, _ = red.reduce_waypoint(red.SOFTMIN, T, f, dq, np.arange(50))
        assert c == pytest.approx(-T * logsumexp(-f / T), rel=1e-13, abs=1e-13)
        # min - T log m <= softmin <= min
        assert f.min() - T * np.log(f.size) - 1e-12 <= c <= f.min() + 1e-12
        w = np.exp(-f / T - logsumexp(-f / T))
        np.testing.assert_allclose(g, w @ dq, rtol=1e-12, atol=1e-14)


def test_softmin_tends_to_min():
    f = np.array([0.4, 0.1, 0.35, 0.9])
    dq = np.eye(4)
    c, g, _ = red.reduce_waypoint(red.SOFTMIN, 1e-4, f, dq, np.arange(4))
    assert c == pytest.approx(0.1, abs=1e-9)
    np.testing.assert_allclose(g, dq[1], atol=1e-12)


def test_hinge_brute_force():
    f = np.array([0.01, 0.2, -0.3, 0.049, 0.05])
    dq = np.arange(15, dtype=np.float64).reshape(5, 3)
    c, g, _ = red.reduce_waypoint(red.HINGE, 0.05, f, dq, np.arange(5))
    expect_c = sum(max(0.0, 0.05 - x) for x in f)
    expect_g = -(dq[0] + dq[2] + dq[3])
    assert c == pytest.approx(expect_c, rel=1e-15)
    np.testing.assert_array_equal(g, expect_g)


def test_empty_partition():
    z = np.zeros(0)
    dq = np.zeros((0, 4))
    for kind, want in ((red.MIN, np.inf), (red.SOFTMIN, np.inf), (red.HINGE, 0.0)):
        c, g, a = red.reduce_waypoint(kind, 0.05, z, dq, np.zeros(0, dtype=np.int64))
        assert c == want and a == -1
        np.testing.assert_array_equal(g, np.zeros(4))


@pytest.mark.parametrize("kind,param", [(red.SOFTMIN, 0.05), (red.HINGE, 0.4), (red.MIN, 0.0)])
def test_cost_gradient_matches_finite_differences(kind, param):
    """d c_i / d q_i by central differences through the whole MLP."""
    shape = synth.NetShape(9, 32, 3)
    w = synth.he_uniform_weights(shape, 21)
    rng = synth.SplitMix64(22)
    q = np.stack([synth.random_config(rng, 9, -1, 1) for _ in range(3)])
    p = synth.uniform_points(rng, 40, [-1, -1, 0], [1, 1, 1]).astype(np.float64)
    c, g, _ = red.collision_cost(9, 32, 3, w, q, p, kind, param)
    h = 1e-6
    for i in range(q.shape[0]):
        for k in range(9):
            qp = q.copy()
            qm = q.copy()
            qp[i, k] += h
            qm[i, k] -= h
            cp = red.collision_cost(9, 32, 3, w, qp, p, kind, param, waypoints=[i])[0][0]
            cm = red.collision_cost(9, 32, 3, w, qm, p, kind, param, waypoints=[i])[0][0]
            fd = (cp - cm) / (2 * h)
            assert abs(fd - g[i, k]) <= 1e-6 * max(1.0, abs(g[i]).max())


def test_csr_partition_equals_dense_subset():
    shape = synth.NetShape(9, 16, 3)
    w = synth.he_uniform_weights(shape, 1)
    rng = synth.SplitMix64(8)
    q = np.stack([synth.random_config(rng, 9, -1, 1) for _ in range(4)])
    p = synth.uniform_points(rng, 30, [-1, -1, 0], [1, 1, 1])
    off, idx = synth.random_partitions(rng, 4, 30, 12)
    c, g, a = red.collision_cost(9, 16, 3, w, q, p, red.SOFTMIN, 0.1, off, idx)
    for i in range(4):
        jj = idx[off[i]:off[i + 1]]
        f, dq = mlp.eval_pairs(9, 16, 3, w, q, p, np.full(jj.size, i), jj)
        ci, gi, ai = red.reduce_waypoint(red.SOFTMIN, 0.1, f, dq, jj)
        assert (c[i] == ci) or (np.isinf(c[i]) and np.isinf(ci))
        np.testing.assert_array_equal(g[i], gi)


def test_nan_propagates_to_the_waypoint_cost():
    """The header's contract: a NaN pair value makes that waypoint's cost NaN in
    every reduction (MIN ranks NaN first and reports its point), never a
    silently finite number."""
    from oracle import reduce as red
    f = np.array([0.3, np.nan, 0.1, np.nan])
    dq = np.arange(8, dtype=np.float64).reshape(4, 2)
    pidx = np.array([10, 11, 12, 13])
    c, g, a = red.reduce_waypoint(red.MIN, 0.0, f, dq, pidx)
    assert np.isnan(c) and a == 11 and np.array_equal(g, dq[1])
    c, g, a = red.reduce_waypoint(red.SOFTMIN, 0.02, f, dq, pidx)
    assert np.isnan(c)
    c, g, a = red.reduce_waypoint(red.HINGE, 0.05, f, dq, pidx)
    assert np.isnan(c)
