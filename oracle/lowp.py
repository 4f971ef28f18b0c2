"""FP64 oracle of the network with 16-bit product operands (test infrastructure only).

What BF16 (or FP16) arithmetic costs the GCDF query by itself, independent of
any kernel: the same network, input and reverse sweep as ``mlp`` (Sec. III-C
network; gradients of Sec. IV-A), evaluated exactly in FP64 except that every
operand of a hidden-layer matrix product is first rounded to the 16-bit format
(round to nearest, ties to even):

  forward  z_l = R(W_l) R(h_{l-1}) + b_l          l = 2..L
  reverse  g_{l-1} = (R(W_l)^T R(g_l)) * s'(z_{l-1}) l = L..2,  g_L = w_o * s'(z_L)
  input    df/denc = R(W_1q)^T R(g_1)

The first layer's point columns W_1p, the biases, the output weights, the
activation function, the output dot product and every accumulation stay exact:
they are not matrix-product operands of a 16-bit tensor-core GEMM.  This model
is the reference of the 16-bit parity bar: it fixes how large the error of a
16-bit path must be from its format alone, so the bar does not move when a
kernel changes where or how often it rounds beyond these points.

Rounding is the IEEE definition written out: BF16 keeps the upper 16 bits of
the FP32 pattern after adding half an ulp of the kept part with ties to even
(inputs are FP64, first rounded to FP32 as every value handed to a kernel
is); FP16 uses numpy's float16 conversion (a library routine).
"""
from __future__ import annotations

import numpy as np

from . import mlp


def round_bf16(x):
    """x rounded to BF16 (via FP32), returned as FP64.  NaN stays NaN."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    keep_lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + keep_lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(x32), np.float64(np.nan), out)


def round_f16(x):
    """x rounded to FP16 (numpy's conversion), returned as FP64."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


_ROUND = {"bf16": round_bf16, "fp16": round_f16, "exact": lambda x: np.asarray(x, dtype=np.float64)}


def value_and_input_grad(layers, v, rnd, round_weights=True, round_operands=True):
    """f(v) and df/denc (the encoded-q columns of df/dv) with the product
    operands rounded by ``rnd``; either group can be left exact (weights:
    W_2..W_L and W_1q; operands: the activations h_1..h_{L-1} and the reverse
    vectors g_L..g_1)."""
    rw = rnd if round_weights else _ROUND["exact"]
    ro = rnd if round_operands else _ROUND["exact"]
    W1, b1 = layers[0]
    z = v @ W1.T + b1
    zs = [z]
    h = mlp.silu(z)
    for (W, b) in layers[1:-1]:
        z = ro(h) @ rw(W).T + b
        zs.append(z)
        h = mlp.silu(z)
    w_o, b_o = layers[-1]
    f = h @ w_o[0] + b_o[0]
    g = w_o[0][None, :] * mlp.silu_prime(zs[-1])
    for l in range(len(zs) - 1, 0, -1):
        g = (ro(g) @ rw(layers[l][0])) * mlp.silu_prime(zs[l - 1])
    d_enc = ro(g) @ rw(W1[:, 3:])
    return f, d_enc


def eval_pairs(n_dof, hidden, n_layers, weights, q, p, ii, jj, shift=None, fmt="bf16",
               round_weights=True, round_operands=True):
    """f (P,) and df/dq (P, n) of the pairs (q[ii[k]], p[jj[k]]) with the
    product operands in ``fmt`` ("bf16", "fp16" or "exact")."""
    rnd = _ROUND[fmt]
    layers = mlp.unpack(n_dof, hidden, n_layers, weights)
    ii = np.asarray(ii, dtype=np.int64)
    jj = np.asarray(jj, dtype=np.int64)
    P = ii.size
    f = np.empty(P)
    dq = np.empty((P, n_dof))
    q = np.asarray(q, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    sh = None if shift is None else np.asarray(shift, dtype=np.float64)
    for s in range(0, P, mlp.CHUNK):
        e = min(P, s + mlp.CHUNK)
        qi = q[ii[s:e]]
        v = mlp.network_input(qi, p[jj[s:e]], None if sh is None else sh[ii[s:e]])
        fs, d_enc = value_and_input_grad(layers, v, rnd, round_weights, round_operands)
        dv = np.concatenate([np.zeros((e - s, 3)), d_enc], axis=1)
        f[s:e] = fs
        dq[s:e] = mlp.chain_rule(qi, dv)
    return f, dq


def query(n_dof, hidden, n_layers, weights, q, p, offsets=None, idx=None, shift=None, fmt="bf16"):
    """As ``mlp.query`` (stacked order of Eq. 14) with 16-bit product operands."""
    if offsets is None:
        ii, jj = mlp.dense_pairs(q.shape[0], p.shape[0])
    else:
        ii, jj = mlp.csr_pairs(offsets, idx)
    return eval_pairs(n_dof, hidden, n_layers, weights, q, p, ii, jj, shift, fmt)
