"""Pins of oracle/lowp.py, the 16-bit-operand reference of the BF16 / FP16 parity
bars: it must reduce to the FP64 oracle without rounding, round like the
library's BF16 conversion, and round exactly the operands of the hidden-layer
products (weights W_2..W_L and W_1q, activations, reverse vectors)."""
import numpy as np
import pytest

import synth
from oracle import lowp, mlp


def _case(n_dof=9, H=32, L=3, seed=4, n_q=5, n_p=7):
    shape = synth.NetShape(n_dof, H, L)
    w = synth.he_uniform_weights(shape, seed)
    r = synth.SplitMix64(seed + 1)
    q = np.stack([synth.random_config(r, n_dof, -2, 2) for _ in range(n_q)])
    p = synth.uniform_points(r, n_p, [-2, -2, 0], [2, 2, 2])
    return shape, w, q, p


def test_exact_format_is_the_oracle():
    shape, w, q, p = _case()
    f0, g0 = mlp.query(shape.n_dof, shape.hidden, shape.n_layers, w, q, p)
    f1, g1 = lowp.query(shape.n_dof, shape.hidden, shape.n_layers, w, q, p, fmt="exact")
    assert np.allclose(f1, f0, rtol=1e-13, atol=1e-13)
    assert np.allclose(g1, g0, rtol=1e-13, atol=1e-13)


def test_bf16_rounding_matches_the_library_conversion():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0)
    x = np.concatenate([
        r.standard_normal(20000).astype(np.float32) * 10.0 ** r.integers(-30, 30, 20000),
        # exact ties between two BF16 neighbours, both parities of the kept bit
        (np.arange(1, 2000, dtype=np.uint32) << 16 | 0x8000).view(np.float32),
        np.array([0.0, -0.0, np.inf, -np.inf, 3.0e38, -3.3e38, 1e-40, -1e-45], dtype=np.float32)])
    ours = lowp.round_bf16(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, lib)
    assert np.isnan(lowp.round_bf16(np.array([np.nan]))[0])


def test_weight_rounding_equals_the_oracle_on_rounded_weights():
    """Weights only: the model equals the plain oracle run on a copy of the net
    whose W_2..W_L are rounded, when W_1q is already representable (the first
    layer's forward is not a 16-bit product, so its weights stay exact there)."""
    n_dof, H, L = 9, 32, 3
    shape, w, q, p = _case(n_dof, H, L)
    d_in = 3 + 2 + 2 * (n_dof - 2)
    w = np.array(w, dtype=np.float64)
    W1 = w[: H * d_in].reshape(H, d_in)
    W1[:, 3:] = lowp.round_bf16(W1[:, 3:])       # W_1q representable in BF16
    w[: H * d_in] = W1.ravel()
    w_r = w.copy()
    off = H * d_in + H
    for _ in range(L - 1):
        w_r[off: off + H * H] = lowp.round_bf16(w_r[off: off + H * H])
        off += H * H + H
    ii, jj = mlp.dense_pairs(q.shape[0], p.shape[0])
    f0, g0 = mlp.eval_pairs(n_dof, H, L, w_r, q, p, ii, jj)
    f1, g1 = lowp.eval_pairs(n_dof, H, L, w, q, p, ii, jj, fmt="bf16", round_operands=False)
    assert np.allclose(f1, f0, rtol=1e-12, atol=1e-12)
    assert np.allclose(g1, g0, rtol=1e-12, atol=1e-12)
    # and the rounding does change the result (the planted difference is visible)
    f2, _ = mlp.eval_pairs(n_dof, H, L, w, q, p, ii, jj)
    assert np.abs(f2 - f0).max() > 1e-6


def test_operand_rounding_on_an_identity_layer():
    """L = 2 with W_2 = I and b_2 = 0: the hidden product reduces to its rounded
    operand, so the model must give f = w_o . s(R(s(z_1))) + b_o and
    df/denc = R(R(w_o s'(z_2)) s'(z_1)) W_1q with z_2 = R(s(z_1)) — every R the
    library's BF16 conversion."""
    torch = pytest.importorskip("torch")

    def R(a):
        return torch.from_numpy(np.asarray(a, np.float64).astype(np.float32)).to(torch.bfloat16) \
            .to(torch.float64).numpy()

    n_dof, H, L = 5, 16, 2
    shape, w, q, p = _case(n_dof, H, L, seed=9)
    d_in = 3 + 2 + 2 * (n_dof - 2)
    w = np.array(w, dtype=np.float64)
    W1 = w[: H * d_in].reshape(H, d_in)
    W1[:, 3:] = R(W1[:, 3:])
    w[: H * d_in] = W1.ravel()
    off = H * d_in + H
    w[off: off + H * H] = np.eye(H).ravel()
    w[off + H * H: off + H * H + H] = 0.0
    layers = mlp.unpack(n_dof, H, L, w)
    ii, jj = mlp.dense_pairs(q.shape[0], p.shape[0])
    v = mlp.network_input(q[ii], p[jj])
    z1 = v @ layers[0][0].T + layers[0][1]
    z2 = R(mlp.silu(z1))
    wo, bo = layers[2][0][0], layers[2][1][0]
    f_exp = mlp.silu(z2) @ wo + bo
    g1 = R(wo[None, :] * mlp.silu_prime(z2)) * mlp.silu_prime(z1)
    denc = R(g1) @ W1[:, 3:]
    dq_exp = mlp.chain_rule(q[ii], np.concatenate([np.zeros((ii.size, 3)), denc], axis=1))
    f, dq = lowp.eval_pairs(n_dof, H, L, w, q, p, ii, jj, fmt="bf16")
    assert np.allclose(f, f_exp, rtol=1e-12, atol=1e-12)
    assert np.allclose(dq, dq_exp, rtol=1e-12, atol=1e-12)


def test_fp16_error_is_below_bf16_error():
    """Three more mantissa bits: the FP16 operands' error against the oracle is
    several times smaller than BF16's on the same pairs."""
    from oracle import metrics
    shape, w, q, p = _case(9, 64, 4, seed=2, n_q=6, n_p=40)
    f0, g0 = mlp.query(9, 64, 4, w, q, p)
    fb, gb = lowp.query(9, 64, 4, w, q, p, fmt="bf16")
    fh, gh = lowp.query(9, 64, 4, w, q, p, fmt="fp16")
    eb = metrics.rel_err_scalar(fb, f0).max()
    eh = metrics.rel_err_scalar(fh, f0).max()
    assert 0 < eh < eb / 3
