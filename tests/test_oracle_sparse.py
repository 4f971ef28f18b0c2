"""Pins of oracle/sparse.py: the partition against an independent distance
and its limit cases, Eq. (17) against a library sparse matrix, and the
projection of Theorem 1 against the exact (sampled) GCDF of a capsule robot."""
import math

import numpy as np
import pytest

import synth
from oracle import robot as R
from oracle import sparse as sp

from test_oracle_gcdf_exact import _arm_case


def _case(seed, N, M):
    r = synth.SplitMix64(seed)
    base = synth.uniform_points(r, N, [-4, -4, 0], [4, 4, 0])[:, :2]
    pts = synth.uniform_points(r, M, [-5, -5, 0], [5, 5, 2])
    return base.astype(np.float32), pts.astype(np.float32)


def test_partition_agrees_with_hypot_away_from_the_boundary():
    base, pts = _case(1, 13, 700)
    R_ = 2.5
    off, idx = sp.partition(base, pts, R_)
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == idx.size
    for i in range(base.shape[0]):
        sel = idx[off[i]: off[i + 1]]
        assert np.all(np.diff(sel) > 0)                         # increasing point order
        d = [math.hypot(float(p[0]) - float(base[i, 0]), float(p[1]) - float(base[i, 1])) for p in pts]
        want = [j for j, dj in enumerate(d) if dj < R_ - 1e-9]
        maybe = {j for j, dj in enumerate(d) if abs(dj - R_) <= 1e-9}
        got = set(sel.tolist())
        assert set(want) <= got and got - set(want) <= maybe


def test_partition_limits():
    base, pts = _case(2, 5, 300)
    off, idx = sp.partition(base, pts, np.inf)
    assert np.array_equal(off, np.arange(6) * 300) and np.array_equal(idx, np.tile(np.arange(300), 5))
    # R = 0 keeps exactly the points on the base position
    pts2 = pts.copy()
    pts2[[7, 123], 0] = base[3, 0]
    pts2[[7, 123], 1] = base[3, 1]
    off, idx = sp.partition(base, pts2, 0.0)
    assert np.array_equal(idx[off[3]: off[4]], [7, 123])
    off, idx = sp.partition(base[:0], pts, 1.0)
    assert np.array_equal(off, [0]) and idx.size == 0


def test_jacobian_matches_a_library_sparse_matrix():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(3)
    n, N = 4, 5
    offsets = np.array([0, 3, 3, 7, 8, 12])
    grad = rng.normal(size=(12, n))
    dense = sp.jacobian_dense(grad, offsets, n, N)
    assert dense.shape == (12, 2 * N * n)
    row_ptr, col, val = sp.jacobian_csr(grad, offsets, n)
    csr = scipy_sparse.csr_matrix((val, col, row_ptr), shape=(12, 2 * N * n)).toarray()
    assert np.array_equal(csr, dense)
    # the velocity columns of every state stay empty
    for i in range(N):
        assert not dense[:, 2 * n * i + n: 2 * n * (i + 1)].any()


def test_projection_reaches_the_nearest_zero_level_sample():
    """With the exact GCDF (Definition 1 over a sampled Z(p)) and its Theorem 1
    gradient, the projection lands exactly on the nearest sample."""
    arm, q0, p, Z = _arm_case()
    m = np.array([4.0, 4.0] + [1.0] * 7)
    rng = synth.SplitMix64(41)
    for _ in range(8):
        q = q0 + rng.uniform(9, -0.3, 0.3)
        f, g, k, two = R.gcdf_label(arm, p, q, Z, m)
        qz = sp.project(q[None], [f], g[None], m)[0]
        assert np.allclose(qz, Z[k], rtol=0, atol=1e-12)
        assert abs(R.sdf(arm, p, qz)) < 1e-10
