"""Model of where the tensor-core path rounds (test-side, NumPy float64).

It evaluates the same network as the kernels but rounds exactly where the
tcgen05 kernel does:
  * operands: the hidden weight matrices W_2..W_L, the reverse copies W_l^T / 2
    and the input-Jacobian matrix W_1q; the activations h_1..h_{L-1} and the
    reverse gradients g_L..g_1 (BF16 or FP16);
  * epilogue arithmetic in packed FP16, one rounding per fused operation:
    the first layer u_1 = A_i / 2 + (W_1p / 2) p (the point and the halved
    weights in FP16, one fused multiply-add per coordinate), u = z / 2,
    t = tanh(u), s = u + u t, 2 s' = s (1 - t) + (1 + t), g_L = (w_o / 2) 2 s',
    and, for FP16 operands, the reverse product acc * 2 s' (BF16 operands form
    it in FP32 from the FP32 accumulator and round once, to BF16);
  * the stash 2 s'(z_2..z_{L-1}) (FP16);
  * the per-waypoint term A_i, the output sum f = w_o . s(z_L) + b_o and every
    matrix accumulation at high precision.
The sigmoid's tanh is exact here (the kernel uses the hardware approximation).

Its use: the kernel must stay close to this model on every pair, which shows
where the kernel's error comes from.  It does not set the parity bar: that
comes from oracle/lowp.py, which rounds only the operands of the hidden-layer
products and does not follow the kernel.  It shares no code with the oracle or
the library.
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


def _silu_f16(u):
    """Packed-FP16 SiLU of u = z / 2: returns s(z) and 2 s'(z)."""
    t = round_f16(np.tanh(u))
    h = round_f16(u * t + u)
    s2 = round_f16(h * round_f16(1.0 - t) + round_f16(1.0 + t))
    return h, s2


def _silu_bf16(u):
    """The BF16-operand epilogue of the hidden layers 1..L: t and 1 + t in FP16,
    s(z) = u (1 + t) exact (the product of two FP16 values, formed in FP32), and
    2 s'(z) = (1 + t) + (1 + t)(u - u t) by FP16 multiply-adds."""
    t = round_f16(np.tanh(u))
    tp1 = round_f16(1.0 + t)
    h = u * tp1
    s2 = round_f16(tp1 + tp1 * round_f16(u - u * t))
    return h, s2


def lowp_eval(n_dof, H, L, weights, q_rows, p_rows, shift_rows=None, fmt="bf16"):
    R = round_bf16 if fmt == "bf16" else round_f16
    silu = _silu_bf16 if fmt == "bf16" else _silu_f16
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
    W1, b1 = lay[0]
    # per-waypoint term: A = W_1q enc(q') + b_1 - W_1p[:, 0:2] shift (points enter raw)
    A = np.concatenate([xy, enc], 1) @ W1[:, 3:].T + b1
    if shift_rows is not None:
        A = A - np.asarray(shift_rows, dtype=np.float64) @ W1[:, 0:2].T
    praw = np.asarray(p_rows, dtype=np.float64)
    w1h = round_f16(0.5 * W1[:, 0:3])
    p16 = round_f16(praw)
    u1 = round_f16(0.5 * A)
    for d in range(3):
        u1 = round_f16(w1h[None, :, d] * p16[:, d:d + 1] + u1)
    h1, s2_1 = silu(u1)
    h = R(h1)
    stash = {}
    for l in range(1, L - 1):  # middle layers 2..L-1 (0-based index l)
        W, b = lay[l]
        zp = round_f16(h @ R(W).T)
        u = round_f16(zp * 0.5 + round_f16(0.5 * b))
        hl, stash[l] = silu(u)
        h = R(hl)
    W, b = lay[L - 1]
    zp = round_f16(h @ R(W).T)
    u = round_f16(zp * 0.5 + round_f16(0.5 * b))
    hL, s2L = silu(u)
    wo, bo = lay[L]
    f = hL @ wo[0] + bo[0]
    woh = round_f16(0.5 * wo[0])[None, :]
    # BF16: the product (w_o / 2) 2 s'(z_L) is exact in FP32 and rounded once
    g = R(woh * s2L) if fmt == "bf16" else R(round_f16(woh * s2L))
    for l in range(L - 1, 0, -1):  # reverse through W_{l+1} (0-based l)
        acc = g @ R(0.5 * lay[l][0])
        d2 = stash[l - 1] if l - 1 >= 1 else s2_1
        g = R(acc * d2) if fmt == "bf16" else R(round_f16(round_f16(acc) * d2))
    denc = g @ R(W1[:, 3:])
    dq = np.empty((q.shape[0], n_dof))
    dq[:, :2] = denc[:, :2]
    dq[:, 2:] = np.cos(ang) * denc[:, 2::2] - np.sin(ang) * denc[:, 3::2]
    return f, dq


def round_e4m3(x):
    """Round to FP8 E4M3 (3 mantissa bits, normals from 2^-6 with spacing
    2^(e-3), subnormal spacing 2^-9), nearest even, saturated to +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                       # a = m 2^e, m in [0.5, 1)
    sp = np.where(a >= 2.0 ** -6, np.ldexp(1.0, e - 4), 2.0 ** -9)
    r = np.minimum(np.round(a / sp) * sp, 448.0)
    return np.where(np.isnan(x), x, np.sign(x) * r)


def _fp8_weight(W):
    """Per-layer scale s = max |W| / 448 (FP32) and the dequantised E4M3 weights."""
    W32 = np.asarray(W, dtype=np.float32)
    s = np.float32(np.max(np.abs(W32))) / np.float32(448.0)
    return round_e4m3((W32 / s).astype(np.float64)) * np.float64(s)


def lowp_eval_fp8(n_dof, H, L, weights, q_rows, p_rows):
    """As lowp_eval for FP8 E4M3 operands: weights with one scale per layer
    (the reverse operand W^T / 2 uses the same bytes with half the scale),
    activations rounded FP16 -> E4M3, reverse operands 64 g rounded FP16 ->
    E4M3 (64 = the kernel's gradient-operand factor), W_1q with its own scale;
    epilogue arithmetic in FP16 as for the 16-bit formats."""
    lay = _layers(n_dof, H, L, weights)
    q = np.asarray(q_rows, dtype=np.float64)
    p = np.asarray(p_rows, dtype=np.float64)
    ang = q[:, 2:]
    enc = np.empty((q.shape[0], 2 * ang.shape[1]))
    enc[:, 0::2] = np.sin(ang)
    enc[:, 1::2] = np.cos(ang)
    W1, b1 = lay[0]
    A = np.concatenate([q[:, :2], enc], 1) @ W1[:, 3:].T + b1
    w1h = round_f16(0.5 * W1[:, 0:3])
    p16 = round_f16(p)
    u1 = round_f16(0.5 * A)
    for d in range(3):
        u1 = round_f16(w1h[None, :, d] * p16[:, d:d + 1] + u1)
    h1, s2_1 = _silu_f16(u1)
    h = round_e4m3(h1)
    stash, Wq = {}, {}
    for l in range(1, L):
        Wq[l] = _fp8_weight(lay[l][0])
    for l in range(1, L - 1):
        zp = round_f16(h @ Wq[l].T)
        u = round_f16(zp * 0.5 + round_f16(0.5 * lay[l][1]))
        hl, stash[l] = _silu_f16(u)
        h = round_e4m3(hl)
    zp = round_f16(h @ Wq[L - 1].T)
    u = round_f16(zp * 0.5 + round_f16(0.5 * lay[L - 1][1]))
    hL, s2L = _silu_f16(u)
    wo, bo = lay[L]
    f = hL @ wo[0] + bo[0]
    g = round_e4m3(round_f16(round_f16(32.0 * wo[0])[None, :] * s2L)) / 64.0
    for l in range(L - 1, 0, -1):
        acc64 = round_f16(64.0 * (g @ (0.5 * Wq[l])))
        d2 = stash[l - 1] if l - 1 >= 1 else s2_1
        g = round_e4m3(round_f16(acc64 * d2)) / 64.0
    W1q = np.asarray(W1[:, 3:], dtype=np.float32)
    sj = np.float32(np.max(np.abs(W1q))) / np.float32(448.0)
    W1q_q = round_e4m3((W1q / sj).astype(np.float64)) * np.float64(sj)
    denc = g @ W1q_q
    dq = np.empty((q.shape[0], n_dof))
    dq[:, :2] = denc[:, :2]
    dq[:, 2:] = np.cos(ang) * denc[:, 2::2] - np.sin(ang) * denc[:, 3::2]
    return f, dq


# ---------------------------------------------------------------------------
# Differentiable fit with BF16 GEMM operands (gcdf_fit_* with precision BF16):
# every matrix product rounds both operands to BF16 and accumulates exactly;
# the encoding, SiLU, s', s'', the element-wise products, the vector products
# (f, the bias and output-weight gradients) stay at high precision.  With
# rnd = identity this is the plain first- and second-order backpropagation.
# ---------------------------------------------------------------------------

def _fit_input(q, p):
    q = np.asarray(q, np.float64)
    p = np.asarray(p, np.float64)
    a = q[:, 2:]
    sc = np.empty((q.shape[0], 2 * a.shape[1]))
    sc[:, 0::2] = np.sin(a)
    sc[:, 1::2] = np.cos(a)
    return np.concatenate([p, q[:, :2], sc], axis=1).astype(np.float32).astype(np.float64)


def _fit_silu(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return z * sg, sg * (1.0 + z * (1.0 - sg)), sg * (1.0 - sg) * (2.0 + z * (1.0 - 2.0 * sg))


def _mm(a, b, rnd):
    return rnd(a) @ rnd(b)


def fit_model(n_dof, H, L, weights, q, p, g_f, G_q=None, rnd=round_bf16):
    """(f, dweights, dq) of the first-order products for g_f, or, with G_q,
    (f, grad_q f, dweights of sum g f + G . grad_q f)."""
    lay = _layers(n_dof, H, L, weights)
    Ws = [W for W, _ in lay[:-1]]
    bs = [b for _, b in lay[:-1]]
    wo, bo = lay[-1][0][0], lay[-1][1][0]
    q = np.asarray(q, np.float64)
    B = q.shape[0]
    g = np.asarray(g_f, np.float64)
    hs, s1, s2 = [_fit_input(q, p)], [], []
    for W, b in zip(Ws, bs):
        h, d1, d2 = _fit_silu(_mm(hs[-1], W.T, rnd) + b)
        hs.append(h)
        s1.append(d1)
        s2.append(d2)
    f = hs[-1] @ wo + bo
    grads = []  # flat blocks in the layout's order
    sizes = [(W.shape[0] * W.shape[1] + W.shape[0]) for W in Ws] + [H + 1]
    dw = np.zeros(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)

    def chain(dv):
        dq = np.empty((B, n_dof))
        dq[:, 0], dq[:, 1] = dv[:, 3], dv[:, 4]
        a = q[:, 2:].astype(np.float32).astype(np.float64)
        dq[:, 2:] = np.cos(a) * dv[:, 5::2] - np.sin(a) * dv[:, 6::2]
        return dq

    if G_q is None:
        dw[offs[L]: offs[L] + H] = g @ hs[L]
        dw[offs[L] + H] = g.sum()
        d = g[:, None] * wo[None, :] * s1[L - 1]
        for l in range(L - 1, -1, -1):
            o, i = Ws[l].shape
            dw[offs[l]: offs[l] + o * i] = _mm(d.T, hs[l], rnd).reshape(-1)
            dw[offs[l] + o * i: offs[l] + o * i + o] = d.sum(axis=0)
            back = _mm(d, Ws[l], rnd)
            if l > 0:
                d = back * s1[l - 1]
        return f, dw, chain(back)
    G = np.asarray(G_q, np.float64)
    # the field's own reverse sweep: a_l, delta_l
    A = [None] * L
    D = [None] * L
    D[L - 1] = wo[None, :] * s1[L - 1]
    for l in range(L - 1, 0, -1):
        A[l - 1] = _mm(D[l], Ws[l], rnd)
        D[l - 1] = A[l - 1] * s1[l - 1]
    dq = chain(_mm(D[0], Ws[0], rnd))
    u = np.zeros_like(hs[0])
    a = q[:, 2:].astype(np.float32).astype(np.float64)
    u[:, 3], u[:, 4] = G[:, 0], G[:, 1]
    u[:, 5::2] = np.cos(a) * G[:, 2:]
    u[:, 6::2] = -np.sin(a) * G[:, 2:]
    o0, i0 = Ws[0].shape
    dw[offs[0]: offs[0] + o0 * i0] = _mm(D[0].T, u, rnd).reshape(-1)
    r = _mm(u, Ws[0].T, rnd)
    E = [None] * L
    for l in range(L):
        E[l] = r * (A[l] if l < L - 1 else wo[None, :]) * s2[l]
        rs = r * s1[l]
        if l + 1 < L:
            dw[offs[l + 1]: offs[l + 1] + H * H] = _mm(D[l + 1].T, rs, rnd).reshape(-1)
            r = _mm(rs, Ws[l + 1].T, rnd)
        else:
            dw[offs[L]: offs[L] + H] = rs.sum(axis=0)
    dw[offs[L]: offs[L] + H] += g @ hs[L]
    dw[offs[L] + H] = g.sum()
    eps = E[L - 1] + g[:, None] * wo[None, :] * s1[L - 1]
    for l in range(L - 1, -1, -1):
        o, i = Ws[l].shape
        dw[offs[l]: offs[l] + o * i] += _mm(eps.T, hs[l], rnd).reshape(-1)
        dw[offs[l] + o * i: offs[l] + o * i + o] = eps.sum(axis=0)
        if l > 0:
            eps = E[l - 1] + _mm(eps, Ws[l], rnd) * s1[l - 1]
    return f, dq, dw
