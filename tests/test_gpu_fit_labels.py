"""A short fit of the 10-DOF 5 x 512 field on labels from the FP64 oracle
(oracle.labels: the capsule robot's sampled GCDF on height levels, Eq. 5-8),
trained through the autograd Function field_grad on the Table I / Eq. 9 loss
with BF16 tensor-core GEMMs and FP32 master weights: the held-out distance loss
must fall well below the untrained net's, and the trained field's projection
step must bring configurations closer to the zero-level set than the untrained
one.  The full-size run is `python tests/fit_on_labels.py`."""
import os

import numpy as np
import pytest

from _helpers import lib, need_gpu

pytestmark = pytest.mark.gpu


def test_short_fit_on_oracle_labels_lowers_the_held_out_loss():
    torch = need_gpu()
    g = lib()
    import fit_on_labels as fl
    workers = max(1, min(4, os.cpu_count() or 1))
    data = fl.make_data(48, 128, 1024, 4, seed=3, workers=workers)
    cut = 40 * 128
    tr = tuple(x[:cut] for x in data)
    ho = tuple(x[cut:] for x in data)
    assert np.all(np.isfinite(data[2])) and ho[0].shape[0] == 8 * 128
    w0 = torch.from_numpy(fl.synth.he_uniform_weights(fl.synth.NetShape(*fl.SHAPE), 0)).cuda()
    before = fl.evaluate(g, torch, w0, ho)
    w, hist = fl.train(g, torch, tr, steps=300, batch=4096, lr=2e-3, precision="bf16", log_every=50)
    assert g.fit_device_status() == 0
    after = fl.evaluate(g, torch, w, ho)
    print("held-out before", before)
    print("held-out after", after)
    print("history", hist)
    assert after["L_dist"] < 0.3 * before["L_dist"], (before["L_dist"], after["L_dist"])
    assert hist[-1][1] < hist[0][1]
    proj = fl.projection_test(g, torch, w, n_targets=16, n_inits=32)
    print("projection", proj)
    assert np.isfinite(proj["residual_ratio"]["median"])
