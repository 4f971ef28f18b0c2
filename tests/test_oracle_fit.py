"""Pins of oracle/fit.py: the forward equals the query oracle, and both
vector-Jacobian products match central finite differences in FP64 (h = 1e-4)."""
import numpy as np

import synth
from oracle import fit, mlp

from _helpers import small_net


def _batch(n_dof, B, seed):
    r = synth.SplitMix64(seed)
    q = np.stack([synth.random_config(r, n_dof, -2.0, 2.0) for _ in range(B)])
    p = synth.uniform_points(r, B, [-2, -2, 0], [2, 2, 2])
    return q, p


def test_forward_equals_the_query_oracle():
    shape, w = small_net(9, hidden=64, n_layers=3)
    q, p = _batch(9, 7, 1)
    f, _ = fit.forward(9, 64, 3, w, q, p)
    fq, _ = mlp.eval_pairs(9, 64, 3, w, q, p, np.arange(7), np.arange(7))
    assert np.allclose(f, fq, rtol=1e-12, atol=1e-12)


def test_weight_and_configuration_vjp_match_central_differences():
    n, H, L = 10, 32, 3
    shape, w = small_net(n, hidden=H, n_layers=L)
    w = np.asarray(w, dtype=np.float64)
    q, p = _batch(n, 5, 2)
    g = np.random.default_rng(3).normal(size=5)
    dw, dq = fit.vjp(n, H, L, w, q, p, g)
    h = 1e-4

    def loss(wv, qv):
        return float(g @ fit.forward(n, H, L, wv, qv, p)[0])
    rng = np.random.default_rng(4)
    # every block of the flat layout: first layer, hidden layers, biases, output
    picks = np.unique(np.concatenate([rng.integers(0, w.size, 60), [0, 3 * H, w.size - 1, w.size - 2]]))
    for k in picks:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (loss(wp, q) - loss(wm, q)) / (2 * h)
        assert abs(fd - dw[k]) <= 1e-6 * max(1.0, abs(dw[k]))
    for b in range(q.shape[0]):
        for d in range(n):
            qp, qm = q.copy(), q.copy()
            qp[b, d] += h
            qm[b, d] -= h
            fd = (loss(w, qp) - loss(w, qm)) / (2 * h)
            assert abs(fd - dq[b, d]) <= 1e-6 * max(1.0, abs(dq[b, d]))


def test_second_order_vjp_matches_central_differences_of_the_gradient_loss():
    """L = g . f + sum_b G_b . grad_q f_b with grad_q f from the query oracle
    (an independent reverse sweep): its weight gradient by central differences."""
    n, H, L = 9, 24, 3
    shape, w = small_net(n, hidden=H, n_layers=L)
    w = np.asarray(w, dtype=np.float64)
    q, p = _batch(n, 4, 5)
    rng = np.random.default_rng(6)
    g = rng.normal(size=4)
    G = rng.normal(size=(4, n))
    dw = fit.vjp2(n, H, L, w, q, p, g, G)

    def loss(wv):
        f, dq = mlp.eval_pairs(n, H, L, wv, q, p, np.arange(4), np.arange(4))
        return float(g @ f + np.sum(G * dq))
    h = 1e-4
    picks = np.unique(np.concatenate([rng.integers(0, w.size, 80), [0, 5, 3 * H, w.size - 1, w.size - 2]]))
    for k in picks:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (loss(wp) - loss(wm)) / (2 * h)
        assert abs(fd - dw[k]) <= 1e-6 * max(1.0, abs(dw[k])), (k, fd, dw[k])
    # with G = 0 it is the first-order weight gradient
    assert np.allclose(fit.vjp2(n, H, L, w, q, p, g, 0 * G), fit.vjp(n, H, L, w, q, p, g)[0], rtol=1e-12, atol=1e-12)
