"""FP64 oracle: neural GCDF value and input Jacobian (test infrastructure only).

Follows Sec. III-C ("Network Architecture"): the MLP takes the concatenation of
the point p and the configuration q and returns one GCDF value per pair.  The
synthetic net used here is

    v   = [p - (b, 0), x - b_x, y - b_y, sin a_1, cos a_1, ..., sin a_k, cos a_k]
    h_1 = s(W_1 v + b_1),   h_l = s(W_l h_{l-1} + b_l)   (l = 2..L)
    f   = w_o . h_L + b_o

with s(z) = z * sigmoid(z) (SiLU).  The optional per-waypoint shift b moves the
points and the base position into the waypoint's base frame before the query
(Sec. IV-A, Algorithm paragraph); it is a constant, so it carries no gradient.
Angles enter through (sin, cos); x and y enter raw.

The reverse sweep is derived by hand:
    g_L     = w_o * s'(z_L)
    g_{l-1} = (W_l^T g_l) * s'(z_{l-1})
    df/dv   = W_1^T g_1
    s'(z)   = sigma(z) * (1 + z * (1 - sigma(z)))
and the chain rule through the encoding gives df/dq:
    df/dx = df/dv_x,  df/dy = df/dv_y,
    df/da = cos(a) * df/dsin(a) - sin(a) * df/dcos(a).

Matrix products use numpy's float64 matmul (a library primitive); the loop over
pair chunks only bounds memory and changes no arithmetic.
"""
from __future__ import annotations

import numpy as np

CHUNK = 8192


def unpack(n_dof: int, hidden: int, n_layers: int, flat: np.ndarray):
    """Read the flat FP32 weight vector into FP64 (W, b) pairs, input to output.

    Layout: per affine layer, W (fan_out x fan_in, row-major) then b.  Layer 1
    has fan_in = 3 + 2 + 2 (n_dof - 2); layers 2..L are hidden x hidden; the
    output layer is 1 x hidden.
    """
    d_in = 3 + 2 + 2 * (n_dof - 2)
    dims = [(hidden, d_in)] + [(hidden, hidden)] * (n_layers - 1) + [(1, hidden)]
    flat = np.asarray(flat, dtype=np.float64)
    layers, off = [], 0
    for (o, i) in dims:
        W = flat[off: off + o * i].reshape(o, i)
        off += o * i
        b = flat[off: off + o]
        off += o
        layers.append((W, b))
    if off != flat.size:
        raise ValueError(f"weight vector has {flat.size} entries, shape needs {off}")
    return layers


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_prime(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def network_input(q_rows: np.ndarray, p_rows: np.ndarray, shift_rows=None) -> np.ndarray:
    """Concatenated input v = [p', enc(q')] for row-aligned q, p (and shift)."""
    q = np.asarray(q_rows, dtype=np.float64)
    p = np.asarray(p_rows, dtype=np.float64).copy()
    xy = q[:, 0:2].copy()
    if shift_rows is not None:
        b = np.asarray(shift_rows, dtype=np.float64)
        p[:, 0:2] -= b
        xy -= b
    ang = q[:, 2:]
    sc = np.empty((q.shape[0], 2 * ang.shape[1]))
    sc[:, 0::2] = np.sin(ang)
    sc[:, 1::2] = np.cos(ang)
    return np.concatenate([p, xy, sc], axis=1)


def value_and_input_grad(layers, v: np.ndarray):
    """f(v) and df/dv for a batch of input rows (one row per pair)."""
    zs, h = [], v
    for (W, b) in layers[:-1]:
        z = h @ W.T + b
        zs.append(z)
        h = silu(z)
    w_o, b_o = layers[-1]
    f = h @ w_o[0] + b_o[0]
    g = w_o[0][None, :] * silu_prime(zs[-1])
    for l in range(len(zs) - 1, 0, -1):
        W = layers[l][0]
        g = (g @ W) * silu_prime(zs[l - 1])
    dv = g @ layers[0][0]
    return f, dv


def chain_rule(q_rows: np.ndarray, dv: np.ndarray) -> np.ndarray:
    """df/dq from df/dv: the encoding's Jacobian applied row by row."""
    q = np.asarray(q_rows, dtype=np.float64)
    d_enc = dv[:, 3:]
    ang = q[:, 2:]
    dq = np.empty((q.shape[0], q.shape[1]))
    dq[:, 0:2] = d_enc[:, 0:2]
    dq[:, 2:] = np.cos(ang) * d_enc[:, 2::2] - np.sin(ang) * d_enc[:, 3::2]
    return dq


def eval_pairs(n_dof, hidden, n_layers, weights, q, p, ii, jj, shift=None):
    """GCDF value f and df/dq for the pairs (q[ii[k]], p[jj[k]]), k = 0..P-1.

    Returns f (P,) and dq (P, n) in FP64.
    """
    layers = unpack(n_dof, hidden, n_layers, weights)
    ii = np.asarray(ii, dtype=np.int64)
    jj = np.asarray(jj, dtype=np.int64)
    P = ii.size
    f = np.empty(P)
    dq = np.empty((P, n_dof))
    q = np.asarray(q, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    sh = None if shift is None else np.asarray(shift, dtype=np.float64)
    for s in range(0, P, CHUNK):
        e = min(P, s + CHUNK)
        qi = q[ii[s:e]]
        v = network_input(qi, p[jj[s:e]], None if sh is None else sh[ii[s:e]])
        fs, dv = value_and_input_grad(layers, v)
        f[s:e] = fs
        dq[s:e] = chain_rule(qi, dv)
    return f, dq


def dense_pairs(n_waypoints: int, n_points: int):
    """Pair order of Eq. (14) with every point in every partition: (i, j) -> i*M + j."""
    ii = np.repeat(np.arange(n_waypoints), n_points)
    jj = np.tile(np.arange(n_points), n_waypoints)
    return ii, jj


def csr_pairs(offsets, idx):
    """Pair order of Eq. (14) for per-waypoint point lists I_{M,i} in CSR form."""
    offsets = np.asarray(offsets, dtype=np.int64)
    lens = np.diff(offsets)
    ii = np.repeat(np.arange(lens.size), lens)
    jj = np.asarray(idx, dtype=np.int64)[: offsets[-1]]
    return ii, jj


def query(n_dof, hidden, n_layers, weights, q, p, offsets=None, idx=None, shift=None):
    """Stacked constraint vector c_gcdf (Eq. 14) and its dense gradient block
    (the (sum m_i) x n matrix of Eq. 15): f (P,), dq (P, n)."""
    if offsets is None:
        ii, jj = dense_pairs(q.shape[0], p.shape[0])
    else:
        ii, jj = csr_pairs(offsets, idx)
    return eval_pairs(n_dof, hidden, n_layers, weights, q, p, ii, jj, shift)
