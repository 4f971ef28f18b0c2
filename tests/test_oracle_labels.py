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


def test_batched_sdf_and_zero_level_sampling_equal_the_line_by_line_definitions():
    import synth
    arm = R.mobile_arm_7()
    rng = np.random.default_rng(0)
    Q = np.concatenate([rng.uniform(-2, 2, (300, 2)), rng.uniform(-np.pi, np.pi, (300, 8))], 1)
    p = np.array([0.4, -0.2, 0.7])
    assert np.allclose(R.sdf_batch(arm, p, Q), [R.sdf(arm, p, q) for q in Q], rtol=0, atol=1e-14)
    r = synth.SplitMix64(5)
    starts = labels._configs(r, 10, 48, p[:2], 1.5)
    dirs = r.uniform(48 * 10, -1.0, 1.0).reshape(48, 10)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Z1 = R.sample_zero_level_set(arm, p, starts, dirs, t_max=6.0, n_steps=192)
    Z2 = R.sample_zero_level_set_batch(arm, p, starts, dirs, t_max=6.0, n_steps=192)
    assert Z1.shape == Z2.shape and Z1.shape[0] > 0
    assert np.allclose(Z1, Z2, rtol=0, atol=1e-12)
    f1 = [R.gcdf_label(arm, p, q, Z1)[0] for q in Q[:20]]
    f2, g2, _ = R.gcdf_label_batch(arm, p, Q[:20], Z1)
    assert np.allclose(f1, f2, rtol=0, atol=1e-13)


def test_height_level_labels_follow_theorem_1():
    """Points on height levels, each labelled against its level's subset moved
    by the point's planar position (Eq. 7): every moved sample is on f_s = 0 for
    its point, and every label satisfies Theorem 1."""
    arm = R.MobileArm()
    q, p, f, g, gap = labels.make_samples(arm, 5, 8, 300, seed=4, p_radius=2.0, n_heights=3, with_gap=True)
    assert set(np.round(p[:, 2], 12)) <= {0.0, 1.0, 2.0}
    assert np.all(np.linalg.norm(p[:, :2] - q[:, :2], axis=1) <= 2.0 + 1e-12)
    for i in range(q.shape[0]):
        assert abs(np.linalg.norm(g[i]) - 1.0) < 1e-12
        assert abs(R.sdf(arm, p[i], q[i] - f[i] * g[i])) < 1e-9
        assert (f[i] >= 0) == (R.sdf(arm, p[i], q[i]) >= 0)
    assert np.all(gap >= 0)
