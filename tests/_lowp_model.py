"""Model of where the tensor-core path rounds (test-side, NumPy float64).

It evaluates the same network as the kernels but rounds exactly where the
tcgen05 kernel stores 16-bit values: the hidden weight matrices W_2..W_L and
the input-Jacobian matrix W_1q (operands), the activations h_1..h_{L-1} and the
reverse gradients g_L..g_1 (operands), and the stash s'(z_2..z_{L-1}) (FP16).
The first layer, biases, output layer and every accumulation stay at high
precision, as in the kernel.  The sigmoid is exact here (the kernel uses the
hardware tanh approximation).

Its only use is to derive how much error the 16-bit format itself implies on
a given input: the BF16 parity bar is max(2e-2, 1.25 x this model's error
against the FP64 oracle).  It shares no code with the oracle or the library.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x):
    x32 = np.asarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def round_f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _layers(n_dof, H, L, w):
    d_in = 3 + 2 + 2 * (n_dof - 2)
    dims = [(H, d_in)] + [(H, H)] * (L - 1) + [(1, H)]
    w = np.asarray(w, dtype=np.float64)
    out, off = [], 0
    for (o, i) in dims:
        out.append((w[off: off + o * i].reshape(o, i), w[off + o * i: off + o * i + o]))
        off += o * i + o
    return out


def lowp_eval(n_dof, H, L, weights, q_rows, p_rows, shift_rows=None, fmt="bf16"):
    R = round_bf16 if fmt == "bf16" else round_f16
    lay = _layers(n_dof, H, L, weights)
    q = np.asarray(q_rows, dtype=np.float64)
    p = np.asarray(p_rows, dtype=np.float64).copy()
    xy = q[:, :2].copy()
    if shift_rows is not None:
        b = np.asarray(shift_rows, dtype=np.float64)
        p[:, :2] -= b
        xy -= b
    ang = q[:, 2:]
    enc = np.empty((q.shape[0], 2 * ang.shape[1]))
    enc[:, 0::2] = np.sin(ang)
    enc[:, 1::2] = np.cos(ang)
    v = np.concatenate([p, xy, enc], 1)
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    dsilu = lambda z: sig(z) * (1.0 + z * (1.0 - sig(z)))
    W1, b1 = lay[0]
    z = v @ W1.T + b1
    zs = [z]
    h = R(z * sig(z))
    for l in range(1, L):
        W, b = lay[l]
        z = h @ R(W).T + b
        zs.append(z)
        h = z * sig(z)
        if l < L - 1:
            h = R(h)
    wo, bo = lay[L]
    f = h @ wo[0] + bo[0]
    g = R(wo[0][None, :] * dsilu(zs[L - 1]))
    for l in range(L - 1, 0, -1):
        d = dsilu(zs[l - 1])
        if l - 1 >= 1:
            d = round_f16(d)
        g = R((g @ R(lay[l][0])) * d)
    denc = g @ R(W1[:, 3:])
    dq = np.empty((q.shape[0], n_dof))
    dq[:, :2] = denc[:, :2]
    dq[:, 2:] = np.cos(ang) * denc[:, 2::2] - np.sin(ang) * denc[:, 3::2]
    return f, dq
