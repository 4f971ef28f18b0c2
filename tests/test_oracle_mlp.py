"""Pins for the FP64 MLP oracle (value, hand-derived input Jacobian, encoding).

Each check compares the oracle with something other than itself: textbook
values of the sigmoid, central finite differences, and PyTorch's float64
autograd on the same weights.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import mlp


def _small_case(n_dof=9, hidden=32, n_layers=4, n_wp=5, n_pt=7, seed=11):
    shape = synth.NetShape(n_dof, hidden, n_layers)
    w = synth.he_uniform_weights(shape, seed=seed)
    rng = synth.SplitMix64(seed + 1)
    q = np.stack([synth.random_config(rng, n_dof, -2, 2) for _ in range(n_wp)]).astype(np.float32)
    p = synth.uniform_points(rng, n_pt, [-2, -2, 0], [2, 2, 2])
    return shape, w, q, p


def test_silu_textbook_values():
    # sigmoid(1) = e / (1 + e); silu(-1) = -1 / (1 + e); silu'(0) = 1/2.
    e = math.e
    assert mlp.silu(np.float64(1.0)) == pytest.approx(e / (1 + e), rel=1e-15)
    assert mlp.silu(np.float64(-1.0)) == pytest.approx(-1 / (1 + e), rel=1e-15)
    assert mlp.silu_prime(np.float64(0.0)) == pytest.approx(0.5, rel=1e-15)
    # large positive z: silu -> z, silu' -> 1; large negative: both -> 0
    assert mlp.silu(np.float64(40.0)) == pytest.approx(40.0, rel=1e-15)
    assert mlp.silu_prime(np.float64(40.0)) == pytest.approx(1.0, rel=1e-15)
    assert abs(mlp.silu_prime(np.float64(-40.0))) < 1e-15


def test_silu_prime_matches_finite_difference():
    z = np.linspace(-6, 6, 97)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_prime(z), fd, rtol=0, atol=1e-9)


def test_single_unit_net_by_hand():
    """H = 1, L = 1 net reading only the x input: f = w_o * silu(a * x + c) + b_o."""
    n_dof, H, L = 3, 1, 1
    d_in = 3 + 2 + 2
    a, c, w_o, b_o = 0.7, -0.2, 1.5, 0.25
    W1 = np.zeros((H, d_in))
    W1[0, 3] = a  # column of x (after p_x, p_y, p_z)
    flat = np.concatenate([W1.ravel(), [c], [w_o], [b_o]])
    q = np.array([[0.9, -0.4, 0.3]])
    p = np.array([[0.1, 0.2, 0.3]])
    f, dq = mlp.eval_pairs(n_dof, H, L, flat, q, p, [0], [0])
    z = a * 0.9 + c
    sig = 1.0 / (1.0 + math.exp(-z))
    assert f[0] == pytest.approx(w_o * z * sig + b_o, rel=1e-14)
    d_silu = sig * (1 + z * (1 - sig))
    np.testing.assert_allclose(dq[0], [w_o * d_silu * a, 0.0, 0.0], rtol=1e-14, atol=1e-16)


def test_angle_chain_rule_single_angle():
    """Net reading only sin(theta) and cos(theta): f = silu(u sin th + v cos th)."""
    n_dof, H, L = 3, 1, 1
    d_in = 7
    u, v = 0.8, -1.3
    W1 = np.zeros((H, d_in))
    W1[0, 5] = u  # sin theta
    W1[0, 6] = v  # cos theta
    flat = np.concatenate([W1.ravel(), [0.0], [1.0], [0.0]])
    th = 0.6
    q = np.array([[0.0, 0.0, th]])
    p = np.zeros((1, 3))
    f, dq = mlp.eval_pairs(n_dof, H, L, flat, q, p, [0], [0])
    z = u * math.sin(th) + v * math.cos(th)
    dz = u * math.cos(th) - v * math.sin(th)
    assert f[0] == pytest.approx(float(mlp.silu(np.float64(z))), rel=1e-14)
    assert dq[0, 2] == pytest.approx(float(mlp.silu_prime(np.float64(z))) * dz, rel=1e-13)
    assert dq[0, 0] == 0.0 and dq[0, 1] == 0.0


@pytest.mark.parametrize("n_dof,hidden,n_layers", [(9, 32, 4), (10, 24, 5), (3, 8, 2)])
def test_jacobian_matches_central_differences(n_dof, hidden, n_layers):
    shape, w, q, p = _small_case(n_dof, hidden, n_layers)
    ii, jj = mlp.dense_pairs(q.shape[0], p.shape[0])
    f, dq = mlp.eval_pairs(n_dof, hidden, n_layers, w, q, p, ii, jj)
    h = 1e-6
    fd = np.zeros_like(dq)
    q64 = q.astype(np.float64)
    for k in range(n_dof):
        qp = q64.copy()
        qm = q64.copy()
        qp[:, k] += h
        qm[:, k] -= h
        fp, _ = mlp.eval_pairs(n_dof, hidden, n_layers, w, qp, p, ii, jj)
        fm, _ = mlp.eval_pairs(n_dof, hidden, n_layers, w, qm, p, ii, jj)
        fd[:, k] = (fp - fm) / (2 * h)
    scale = np.abs(dq).max()
    assert np.abs(fd - dq).max() <= 1e-7 * scale + 1e-9


def _torch_reference(shape, w, q, p, shift=None):
    """The same network written with torch.nn layers and differentiated by autograd."""
    layers = synth.unpack_weights(shape, w)
    mods = []
    for k, (W, b) in enumerate(layers):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W.astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(b.astype(np.float64)))
        mods.append(lin)
        if k < len(layers) - 1:
            mods.append(torch.nn.SiLU())
    net = torch.nn.Sequential(*mods)
    N, M = q.shape[0], p.shape[0]
    qt = torch.from_numpy(q.astype(np.float64)).repeat_interleave(M, 0).requires_grad_(True)
    pt = torch.from_numpy(p.astype(np.float64)).repeat(N, 1)
    xy = qt[:, :2]
    if shift is not None:
        st = torch.from_numpy(shift.astype(np.float64)).repeat_interleave(M, 0)
        xy = xy - st
        pt = torch.cat([pt[:, :2] - st, pt[:, 2:]], 1)
    ang = qt[:, 2:]
    sc = torch.stack([torch.sin(ang), torch.cos(ang)], dim=2).reshape(ang.shape[0], -1)
    v = torch.cat([pt, xy, sc], 1)
    f = net(v)[:, 0]
    (g,) = torch.autograd.grad(f.sum(), qt)
    return f.detach().numpy(), g.numpy()


@pytest.mark.parametrize("use_shift", [False, True])
def test_oracle_matches_torch_autograd(use_shift):
    shape, w, q, p = _small_case(9, 48, 4, n_wp=6, n_pt=9)
    shift = synth.random_shift(synth.SplitMix64(5), q) if use_shift else None
    ii, jj = mlp.dense_pairs(q.shape[0], p.shape[0])
    f, dq = mlp.eval_pairs(9, 48, 4, w, q, p, ii, jj, shift)
    ft, gt = _torch_reference(shape, w, q, p, shift)
    np.testing.assert_allclose(f, ft, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(dq, gt, rtol=1e-11, atol=1e-12)


def test_shift_is_a_translation_of_points_and_base():
    """A shift b gives the same result as moving p and (x, y) by -b by hand."""
    shape, w, q, p = _small_case(9, 16, 3, n_wp=3, n_pt=4)
    shift = np.array([[0.5, -0.25], [1.0, 2.0], [-3.0, 0.125]], dtype=np.float32)
    f1, g1 = mlp.eval_pairs(9, 16, 3, w, q, p, [0, 1, 2], [3, 0, 2], shift)
    qs = q.astype(np.float64)[[0, 1, 2]].copy()
    ps = p.astype(np.float64)[[3, 0, 2]].copy()
    qs[:, :2] -= shift
    ps[:, :2] -= shift
    f2, g2 = mlp.eval_pairs(9, 16, 3, w, qs, ps, [0, 1, 2], [0, 1, 2])
    np.testing.assert_allclose(f1, f2, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(g1, g2, rtol=1e-13, atol=1e-14)


def test_translation_equivariance_of_network_input():
    """Sec. III-C: moving the base and the point by the same planar offset with
    the shift set to the base position leaves the query unchanged."""
    shape, w, q, p = _small_case(9, 16, 3, n_wp=2, n_pt=3)
    d = np.array([3.5, -1.25], dtype=np.float64)
    q2 = q.astype(np.float64).copy()
    p2 = p.astype(np.float64).copy()
    q2[:, :2] += d
    p2[:, :2] += d
    s1 = q.astype(np.float64)[:, :2]
    s2 = q2[:, :2]
    ii, jj = mlp.dense_pairs(2, 3)
    f1, g1 = mlp.eval_pairs(9, 16, 3, w, q, p, ii, jj, s1)
    f2, g2 = mlp.eval_pairs(9, 16, 3, w, q2, p2, ii, jj, s2)
    np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g1, g2, rtol=1e-11, atol=1e-12)


def test_pair_orders_follow_stacked_vector():
    """Eq. (14): waypoint-major, then the points of that waypoint's partition."""
    ii, jj = mlp.dense_pairs(3, 4)
    assert list(ii) == [0] * 4 + [1] * 4 + [2] * 4
    assert list(jj) == [0, 1, 2, 3] * 3
    ii, jj = mlp.csr_pairs([0, 2, 2, 5], [7, 1, 4, 4, 0])
    assert list(ii) == [0, 0, 2, 2, 2]
    assert list(jj) == [7, 1, 4, 4, 0]


def test_weight_unpack_rejects_wrong_size():
    shape = synth.NetShape(9, 16, 3)
    w = synth.he_uniform_weights(shape, 0)
    with pytest.raises(ValueError):
        mlp.unpack(9, 16, 3, w[:-1])
