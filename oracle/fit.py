"""FP64 oracle: the field's value per sample and its vector-Jacobian products
with respect to the weights and the configuration (test infrastructure only).

Used to fit the network on (q, p, f) samples with the distance loss of
Table I, L_dist = mean_b (f(q_b, p_b) - f_hat_b)^2 (Sec. III-C).  Per sample b
and upstream gradient g_b = dL/df_b, with v = [p, x, y, sin a_1, cos a_1, ...]
(the concatenated input of Sec. III-C), z_1 = W_1 v + b_1, h_l = s(z_l),
z_{l+1} = W_{l+1} h_l + b_{l+1}, f = w_o . h_L + b_o:

    delta_L = g w_o * s'(z_L)
    delta_{l-1} = (W_l^T delta_l) * s'(z_{l-1})
    dW_l = sum_b delta_l h_{l-1}^T,  db_l = sum_b delta_l   (h_0 = v)
    dw_o = sum_b g h_L,  db_o = sum_b g
    dv = W_1^T delta_1 -> dq by the sin/cos chain rule.

Weights and their gradient use the flat layout of gcdf_weight_count: for every
affine layer, W (fan_out x fan_in, row-major) then b.
"""
from __future__ import annotations

import numpy as np

from . import mlp


def _layers(n_dof, H, L, w):
    d_in = 3 + 2 + 2 * (n_dof - 2)
    dims = [(H, d_in)] + [(H, H)] * (L - 1) + [(1, H)]
    out, off = [], 0
    for (o, i) in dims:
        out.append((off, o, i))
        off += o * i + o
    return out, off


def _silu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return z * s, s * (1.0 + z * (1.0 - s))


def forward(n_dof, H, L, weights, q, p):
    """f (B,) and the activations (v, [z_l], [h_l])."""
    w = np.asarray(weights, dtype=np.float64)
    lay, _ = _layers(n_dof, H, L, w)
    v = mlp.network_input(np.asarray(q, np.float64), np.asarray(p, np.float64))
    hs, ds = [v], []
    h = v
    for (off, o, i) in lay[:-1]:
        W = w[off: off + o * i].reshape(o, i)
        b = w[off + o * i: off + o * i + o]
        h, d = _silu(h @ W.T + b)
        hs.append(h)
        ds.append(d)
    off, o, i = lay[-1]
    wo = w[off: off + i]
    bo = w[off + i]
    return h @ wo + bo, (hs, ds)


def vjp(n_dof, H, L, weights, q, p, g):
    """dL/dweights (flat) and dL/dq (B, n) for the upstream gradient g (B,)."""
    w = np.asarray(weights, dtype=np.float64)
    lay, total = _layers(n_dof, H, L, w)
    g = np.asarray(g, dtype=np.float64)
    _, (hs, ds) = forward(n_dof, H, L, w, q, p)
    dw = np.zeros(total)
    off, o, i = lay[-1]
    wo = w[off: off + i]
    dw[off: off + i] = g @ hs[-1]
    dw[off + i] = g.sum()
    delta = g[:, None] * wo[None, :] * ds[-1]
    for l in range(len(lay) - 2, -1, -1):
        off, o, i = lay[l]
        W = w[off: off + o * i].reshape(o, i)
        dw[off: off + o * i] = (delta.T @ hs[l]).reshape(-1)
        dw[off + o * i: off + o * i + o] = delta.sum(axis=0)
        back = delta @ W
        if l > 0:
            delta = back * ds[l - 1]
        else:
            dv = back
    q = np.asarray(q, dtype=np.float64)
    dq = np.empty((q.shape[0], n_dof))
    dq[:, 0] = dv[:, 3]
    dq[:, 1] = dv[:, 4]
    ang = q[:, 2:]
    dq[:, 2:] = np.cos(ang) * dv[:, 5::2] - np.sin(ang) * dv[:, 6::2]
    return dw, dq
