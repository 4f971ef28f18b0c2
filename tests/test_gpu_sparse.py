"""Spatial partition, dense->sparse Jacobian and single-step projection on the
GPU against oracle/sparse.py: the integer outputs bit for bit, the projection
within the field's tolerance."""
import numpy as np
import pytest

import synth
from oracle import metrics
from oracle import sparse as sp

from _helpers import lib, need_gpu, random_traj, small_net, to_dev

pytestmark = pytest.mark.gpu


def _case(seed, N, M):
    r = synth.SplitMix64(seed)
    base = synth.uniform_points(r, N, [-4, -4, 0], [4, 4, 0])[:, :2].astype(np.float32)
    pts = synth.uniform_points(r, M, [-5, -5, 0], [5, 5, 2]).astype(np.float32)
    return np.ascontiguousarray(base), pts


@pytest.mark.parametrize("N,M,R", [(13, 700, 2.5), (1, 5000, 1.0), (200, 3000, 0.7), (7, 2047, 3.0),
                                   (7, 2048, 3.0), (7, 2049, 3.0), (3, 40000, 9.0), (5, 300, np.inf),
                                   (4, 100, 0.0), (0, 100, 1.0), (6, 0, 1.0)])
def test_partition_bit_exact(N, M, R):
    torch = need_gpu()
    g = lib()
    base, pts = _case(N * 1000 + M, N, M)
    if N > 2 and M > 10:  # points exactly on a base and exactly at distance R along x
        pts[3, :2] = base[2]
        if np.isfinite(R):
            pts[5, 0] = np.float32(base[1, 0] + np.float32(R))
            pts[5, 1] = base[1, 1]
    off_ref, idx_ref = sp.partition(base, pts, R)
    off, idx = g.partition(to_dev(torch, base), to_dev(torch, pts.reshape(-1, 3)), R)
    assert np.array_equal(off.cpu().numpy(), off_ref)
    assert np.array_equal(idx.cpu().numpy(), idx_ref)


@pytest.mark.parametrize("csr", [False, True])
def test_jacobian_scatter_bit_exact(csr):
    torch = need_gpu()
    g = lib()
    rng = np.random.default_rng(5)
    n, N, M = 9, 11, 37
    if csr:
        lens = rng.integers(0, 60, N)
        lens[3] = 0
        offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    else:
        offsets = (np.arange(N + 1) * M).astype(np.int32)
    P = int(offsets[-1])
    grad = rng.normal(size=(P, n)).astype(np.float32)
    rp, col, val = g.jacobian_scatter(to_dev(torch, grad), N, to_dev(torch, offsets) if csr else None,
                                      0 if csr else M)
    rp_ref, col_ref, val_ref = sp.jacobian_csr(grad, offsets, n)
    assert np.array_equal(rp.cpu().numpy(), rp_ref)
    assert np.array_equal(col.cpu().numpy(), col_ref)
    assert np.array_equal(val.cpu().numpy(), val_ref.astype(np.float32))
    rp2, col2, none = g.jacobian_scatter(to_dev(torch, grad), N, to_dev(torch, offsets) if csr else None,
                                         0 if csr else M, with_values=False)
    assert none is None and torch.equal(col2, col) and torch.equal(rp2, rp)


# The step f M^-1 df/dq is a product of two outputs that are each within the
# field's tolerance t (1e-5 FP32, 2e-2 BF16), so its relative error is bounded
# by (1 + t)^2 - 1 = 2t + t^2.
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5 + 1e-10), ("bf16", 4e-2 + 4e-4)])
@pytest.mark.parametrize("with_m", [False, True])
def test_projection_matches_oracle(prec, tol, with_m):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, prec)
    q = random_traj(6, 9, 51, -2, 2).astype(np.float32)
    r = synth.SplitMix64(52)
    pts = synth.uniform_points(r, 300, [-2, -2, 0], [2, 2, 2]).astype(np.float32)
    m = np.array([4.0, 4.0] + [1.0] * 7, dtype=np.float32) if with_m else None
    # CSR lists from the partition around each waypoint's base
    base = np.ascontiguousarray(q[:, :2])
    off, idx = sp.partition(base, pts, 1.6)
    qz = g.project(net, to_dev(torch, q), to_dev(torch, pts), to_dev(torch, off.astype(np.int32)),
                   to_dev(torch, idx.astype(np.int32)), m_diag=None if m is None else to_dev(torch, m))
    ref = sp.project_pairs(9, shape.hidden, shape.n_layers, w, q.astype(np.float64), pts, off, idx,
                           m_diag=m)
    ii = np.repeat(np.arange(q.shape[0]), np.diff(off))
    # the kernel applies exactly q - f M^-1 g to the library's own query outputs
    f, gq = g.query(net, to_dev(torch, q), to_dev(torch, pts), to_dev(torch, off.astype(np.int32)),
                    to_dev(torch, idx.astype(np.int32)))
    own = q[ii] - f.cpu().numpy()[:, None] * (gq.cpu().numpy() / (1.0 if m is None else m))
    assert np.allclose(qz.cpu().numpy(), own, rtol=1e-6, atol=1e-6)
    step_gpu = q[ii].astype(np.float64) - qz.cpu().numpy()
    step_ref = q[ii].astype(np.float64) - ref
    err = metrics.rel_err_vector(step_gpu, step_ref)
    if prec == "fp32":
        assert err.max() <= tol
    else:
        assert np.quantile(err, 0.99) <= tol


def test_projection_dense_lists_and_rejects_bad_pointers():
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "fp32")
    q = random_traj(3, 9, 61, -2, 2).astype(np.float32)
    pts = synth.uniform_points(synth.SplitMix64(62), 50, [-2, -2, 0], [2, 2, 2]).astype(np.float32)
    qz = g.project(net, to_dev(torch, q), to_dev(torch, pts))
    ref = sp.project_pairs(9, shape.hidden, shape.n_layers, w, q.astype(np.float64), pts)
    ii = np.repeat(np.arange(3), 50)
    err = metrics.rel_err_vector(q[ii] - qz.cpu().numpy(), q[ii].astype(np.float64) - ref)
    assert err.max() <= 1e-5
    with pytest.raises(g.GcdfError):
        g.partition(to_dev(torch, np.zeros((2, 2), np.float32)), to_dev(torch, pts), -1.0)
