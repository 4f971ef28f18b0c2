"""Labelled (q, p, f) samples of the capsule robot's GCDF (oracle/labels.py):
the recipe's ranges, determinism by seed, and Theorem 1 on every label (unit
gradient, the one-step projection landing on f_s = 0, the sign of f_s)."""
import numpy as np

from oracle import labels
from oracle import robot as R


def test_labels_follow_the_recipe_and_theorem_1():
    arm = R.MobileArm()
    q, p, f, g = labels.make_samples(arm, 2, 6, 24, seed=3, p_radius=2.0)
    assert q.shape == (12, 9) and p.shape == (12, 3) and f.shape == (12,) and g.shape == (12, 9)
    assert np.all(np.linalg.norm(p[:, :2] - q[:, :2], axis=1) <= 2.0 + 1e-12)
    assert np.all((p[:, 2] >= 0.0) & (p[:, 2] <= 2.0))
    assert np.all(np.abs(q[:, 2:]) <= np.pi)
    for i in range(12):
        assert abs(np.linalg.norm(g[i]) - 1.0) < 1e-12
        assert abs(R.sdf(arm, p[i], q[i] - f[i] * g[i])) < 1e-9
        s = R.sdf(arm, p[i], q[i])
        assert (f[i] >= 0) == (s >= 0)
    q2, p2, f2, g2 = labels.make_samples(arm, 2, 6, 24, seed=3, p_radius=2.0)
    assert np.array_equal(q, q2) and np.array_equal(f, f2) and np.array_equal(p, p2)
