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


def _silu2(z):
    """s(z), s'(z), s''(z) of SiLU s(z) = z sigmoid(z)."""
    sg = 1.0 / (1.0 + np.exp(-z))
    return z * sg, sg * (1.0 + z * (1.0 - sg)), sg * (1.0 - sg) * (2.0 + z * (1.0 - 2.0 * sg))


def vjp2(n_dof, H, L, weights, q, p, g_f, G_q):
    """dL/dweights (flat) for L = sum_b g_b f_b + sum_b G_b . grad_q f_b: the
    weight gradient the regularisers of Table I (gradient direction, eikonal,
    tension — all functions of grad_q f) need.  With u = C^T G (C: dv -> dq, the
    sin/cos chain rule), r_1 = W_1 u, r_{l+1} = W_{l+1} (r_l * s'(z_l)), a_l the
    pre-activation factor of the reverse sweep (delta_l = a_l * s'(z_l)):
        dW_1 += delta_1 u^T;  dW_{l+1} += delta_{l+1} (r_l * s'(z_l))^T;  dw_o += r_L * s'(z_L)
    and the second-derivative terms e_l = r_l * a_l * s''(z_l), back-propagated
    with the value term through the forward network:
        eps_L = e_L + g w_o * s'(z_L);  eps_l = e_l + (W_{l+1}^T eps_{l+1}) * s'(z_l)
        dW_l += eps_l h_{l-1}^T;  db_l += eps_l;  dw_o += g h_L;  db_o += g."""
    w = np.asarray(weights, dtype=np.float64)
    lay, total = _layers(n_dof, H, L, w)
    q = np.asarray(q, dtype=np.float64)
    g = np.asarray(g_f, dtype=np.float64)
    G = np.asarray(G_q, dtype=np.float64)
    v = mlp.network_input(q, np.asarray(p, np.float64))
    Ws, bs = [], []
    for (off, o, i) in lay[:-1]:
        Ws.append(w[off: off + o * i].reshape(o, i))
        bs.append(w[off + o * i: off + o * i + o])
    off_o = lay[-1][0]
    wo = w[off_o: off_o + H]
    hs, s1, s2 = [v], [], []
    h = v
    for W, b in zip(Ws, bs):
        h, d1, d2 = _silu2(h @ W.T + b)
        hs.append(h)
        s1.append(d1)
        s2.append(d2)
    # reverse sweep: a_l and delta_l
    a = [None] * L
    dl = [None] * L
    a[L - 1] = np.broadcast_to(wo, (q.shape[0], H))
    dl[L - 1] = a[L - 1] * s1[L - 1]
    for l in range(L - 1, 0, -1):
        a[l - 1] = dl[l] @ Ws[l]
        dl[l - 1] = a[l - 1] * s1[l - 1]
    # u = C^T G (dv adjoint of the sin/cos chain rule)
    d_in = v.shape[1]
    u = np.zeros((q.shape[0], d_in))
    u[:, 3] = G[:, 0]
    u[:, 4] = G[:, 1]
    ang = q[:, 2:]
    u[:, 5::2] = np.cos(ang) * G[:, 2:]
    u[:, 6::2] = -np.sin(ang) * G[:, 2:]
    dw = np.zeros(total)
    # forward sweep of r and the first-derivative weight terms
    r = u @ Ws[0].T
    offs = [lay[l][0] for l in range(L)]
    dw[offs[0]: offs[0] + H * d_in] += (dl[0].T @ u).reshape(-1)
    e = [None] * L
    for l in range(L):
        e[l] = r * a[l] * s2[l]
        if l + 1 < L:
            rs = r * s1[l]
            dw[offs[l + 1]: offs[l + 1] + H * H] += (dl[l + 1].T @ rs).reshape(-1)
            r = rs @ Ws[l + 1].T
    dw[off_o: off_o + H] += (r * s1[L - 1]).sum(axis=0)
    # back-propagate the second-derivative terms with the value term
    eps = e[L - 1] + g[:, None] * wo[None, :] * s1[L - 1]
    dw[off_o: off_o + H] += g @ hs[L]
    dw[off_o + H] += g.sum()
    for l in range(L - 1, -1, -1):
        fan_in = d_in if l == 0 else H
        dw[offs[l]: offs[l] + H * fan_in] += (eps.T @ hs[l]).reshape(-1)
        dw[offs[l] + H * fan_in: offs[l] + H * fan_in + H] += eps.sum(axis=0)
        if l > 0:
            eps = e[l - 1] + (eps @ Ws[l]) * s1[l - 1]
    return dw
