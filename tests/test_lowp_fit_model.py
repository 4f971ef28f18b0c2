"""The BF16 rounding model of the fit (tests/_lowp_model.py fit_model) is the
plain first- and second-order backpropagation when nothing is rounded: with
the identity in place of the BF16 rounding it reproduces the FP64 oracle
(up to the FP32 rounding of the encoded input, which it keeps)."""
import numpy as np
import pytest

import synth
from oracle import fit

from _helpers import small_net
from _lowp_model import fit_model, round_bf16


@pytest.mark.parametrize("n,H,L,B", [(9, 64, 3, 50), (3, 32, 1, 20), (10, 48, 2, 33)])
def test_unrounded_model_is_the_oracle(n, H, L, B):
    _, w = small_net(n, hidden=H, n_layers=L)
    r = synth.SplitMix64(5)
    q = np.stack([synth.random_config(r, n, -2.0, 2.0) for _ in range(B)]).astype(np.float32).astype(np.float64)
    p = synth.uniform_points(r, B, [-2, -2, 0], [2, 2, 2]).astype(np.float32).astype(np.float64)
    g = np.random.default_rng(1).normal(size=B)
    G = np.random.default_rng(2).normal(size=(B, n))

    def rel(a, b):
        return np.abs(a - b).max() / np.abs(b).max()

    ident = lambda x: x  # noqa: E731
    f, dw, dq = fit_model(n, H, L, w, q, p, g, rnd=ident)
    f_ref, _ = fit.forward(n, H, L, w, q, p)
    dw_ref, dq_ref = fit.vjp(n, H, L, w, q, p, g)
    assert rel(f, f_ref) < 1e-6 and rel(dw, dw_ref) < 1e-6 and rel(dq, dq_ref) < 1e-6
    f2, dq2, dw2 = fit_model(n, H, L, w, q, p, g, G, rnd=ident)
    _, dq1 = fit.vjp(n, H, L, w, q, p, np.ones(B))
    assert rel(dq2, dq1) < 1e-6 and rel(dw2, fit.vjp2(n, H, L, w, q, p, g, G)) < 1e-6
    # and the BF16 rounding moves it by about the format's resolution, not more
    fb, dwb, _ = fit_model(n, H, L, w, q, p, g)
    assert 1e-4 < rel(fb, f_ref) < 5e-2 and np.linalg.norm(dwb - dw_ref) < 5e-2 * np.linalg.norm(dw_ref)


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert round_bf16(np.array([1.0 + 2.0 ** -8 + 2.0 ** -12]))[0] == 1.0 + 2.0 ** -7
