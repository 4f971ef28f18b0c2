"""Pins for the brute-force GCDF of Definition 1 on synthetic capsule robots.

Closed forms: the 1-DoF planar link of Fig. 3 and the translation-only robot.
Theorem 1 (weighted eikonal and single-step projection) on the sampled field,
finite differences, f = 0 on contact configurations, and translation
equivariance (Sec. III-C).
"""
import math

import numpy as np
import pytest

import synth
from oracle import robot as R


def _golden_1dof():
    path = __file__.replace("test_oracle_gcdf_exact.py", "golden/one_dof_link.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def test_segment_distance_brute_force():
    rng = synth.SplitMix64(4)
    a = rng.uniform(3, -1, 1)
    b = rng.uniform(3, -1, 1)
    ts = np.linspace(0, 1, 200001)
    pts = a[None] + ts[:, None] * (b - a)[None]
    for _ in range(5):
        p = rng.uniform(3, -2, 2)
        brute = np.min(np.linalg.norm(pts - p[None], axis=1))
        assert R.segment_distance(p, a, b) == pytest.approx(brute, abs=1e-9)


def _one_dof_samples(link, p, n_starts=64, seed=7):
    rng = synth.SplitMix64(seed)
    starts = rng.uniform(n_starts, -math.pi, math.pi)[:, None]
    dirs = np.where(rng.uniform(n_starts) < 0.5, -1.0, 1.0)[:, None]
    return R.sample_zero_level_set(link, p, starts, dirs, t_max=2 * math.pi, n_steps=256)


def test_one_dof_link_closed_form():
    """Fig. 3: the point induces two contacts at phi +- asin(r / rho); the signed
    GCDF is +-min_k |theta - theta_k|, negative between the contacts."""
    for (length, radius, rho, phi, theta) in _golden_1dof():
        link = R.PlanarLink(length, radius)
        p = np.array([rho * math.cos(phi), rho * math.sin(phi), 0.0])
        Z = _one_dof_samples(link, p)
        half = math.asin(radius / rho)
        contacts = np.array([phi - half, phi + half])
        contacts = np.concatenate([contacts, contacts - 2 * math.pi, contacts + 2 * math.pi])
        # every sample lies on a closed-form contact
        for z in Z[:, 0]:
            assert np.min(np.abs(contacts - z)) < 1e-9
        d = np.min(np.abs(contacts - theta))
        inside = abs(math.remainder(theta - phi, 2 * math.pi)) < half
        want = -d if inside else d
        f, g, _, _ = R.gcdf_label(link, p, np.array([theta]), Z)
        assert f == pytest.approx(want, abs=1e-9)
        assert abs(g[0]) == pytest.approx(1.0, abs=1e-12)


def test_one_dof_signed_gradient_points_out_of_collision():
    """Sec. III-B: inside the obstacle the signed field's gradient points toward
    the nearer contact, so descent on -f escapes; the unsigned field has its
    spurious maximum at theta = phi instead."""
    link = R.PlanarLink(1.0, 0.1)
    rho, phi = 0.6, 0.3
    p = np.array([rho * math.cos(phi), rho * math.sin(phi), 0.0])
    Z = _one_dof_samples(link, p)
    for dth in (-0.1, -0.05, 0.05, 0.1):
        f, g, _, _ = R.gcdf_label(link, p, np.array([phi + dth]), Z)
        assert f < 0
        # increasing f means moving away from phi toward the nearer contact
        assert np.sign(g[0]) == np.sign(dth)
        # the unsigned distance |f| decreases toward the contact: its gradient
        # has the opposite sign, i.e. it peaks at theta = phi
        assert np.sign(-g[0]) == -np.sign(dth)


def test_translation_only_robot_closed_form_and_monotone():
    """n = 2 base-only robot: f = rho_xy - r on the capsule's straight part."""
    base = R.BaseOnly(0.35)
    p = np.array([0.7, -0.2, 0.25])
    rng = synth.SplitMix64(9)
    K = 3000
    ang = rng.uniform(K, 0, 2 * math.pi)
    rad = rng.uniform(K, 0.0, 1.2)
    starts = np.stack([p[0] + rad * np.cos(ang), p[1] + rad * np.sin(ang)], 1)
    dang = rng.uniform(K, 0, 2 * math.pi)
    dirs = np.stack([np.cos(dang), np.sin(dang)], 1)
    Z = R.sample_zero_level_set(base, p, starts, dirs, t_max=2.0, n_steps=64)
    # every sample lies on the circle of radius r around the point
    np.testing.assert_allclose(np.hypot(Z[:, 0] - p[0], Z[:, 1] - p[1]), 0.35, atol=1e-10)
    for q in (np.array([1.5, 0.4]), np.array([-0.6, -1.0]), np.array([0.8, -0.1])):
        rho = math.hypot(q[0] - p[0], q[1] - p[1])
        want = rho - 0.35
        prev = np.inf
        for k in (100, 400, 1600, Z.shape[0]):
            f, _, _, _ = R.gcdf_label(base, p, q, Z[:k])
            # nested samples: |f| never increases, and stays above the true distance
            assert abs(f) <= prev + 1e-15
            assert abs(f) >= abs(want) - 1e-12
            prev = abs(f)
        assert f == pytest.approx(want, abs=2e-3)


def _arm_case(seed=12):
    arm = R.MobileArm()
    rng = synth.SplitMix64(seed)
    q = np.concatenate([[0.0, 0.0], rng.uniform(7, -math.pi, math.pi)])
    A, B, Rr = arm.capsules(q)
    # a point a little outside the third link
    c = 0.5 * (A[3] + B[3])
    axis = (B[3] - A[3]) / np.linalg.norm(B[3] - A[3])
    perp = np.cross(axis, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp)
    p = c + (Rr[3] + 0.15) * perp
    K = 600
    starts = np.concatenate([
        q[None, :2] + rng.uniform(2 * K, -0.6, 0.6).reshape(K, 2),
        rng.uniform(7 * K, -math.pi, math.pi).reshape(K, 7)], 1)
    dirs = rng.uniform(9 * K, -1, 1).reshape(K, 9)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Z = R.sample_zero_level_set(arm, p, starts, dirs, t_max=3.0, n_steps=48)
    return arm, q, p, Z


def test_zero_level_samples_are_contacts():
    arm, q, p, Z = _arm_case()
    assert Z.shape[0] > 100
    for z in Z[:50]:
        assert abs(R.sdf(arm, p, z)) < 1e-10
        # a contact configuration is its own nearest sample: f = 0 exactly
        f, _, _, _ = R.gcdf_label(arm, p, z, Z)
        assert f == 0.0


def test_theorem1_on_sampled_field():
    """Weighted eikonal ||df/dq||_{M^-1} = 1 and the one-step projection
    q - f M^{-1} df/dq landing on f_s = 0, with M = diag(4, 4, 1, ..., 1)."""
    arm, q0, p, Z = _arm_case()
    m = np.array([4.0, 4.0] + [1.0] * 7)
    rng = synth.SplitMix64(31)
    for _ in range(10):
        q = q0 + rng.uniform(9, -0.3, 0.3)
        f, g, k, two = R.gcdf_label(arm, p, q, Z, m)
        assert math.sqrt(np.sum(g * g / m)) == pytest.approx(1.0, abs=1e-12)
        qz = q - f * g / m
        assert abs(R.sdf(arm, p, qz)) < 1e-10


def test_sampled_field_gradient_matches_finite_differences():
    arm, q0, p, Z = _arm_case()
    m = np.array([2.0, 2.0] + [1.0] * 7)
    fn = R.gcdf_label_field(arm, p, Z, m)
    rng = synth.SplitMix64(32)
    checked = 0
    for _ in range(20):
        q = q0 + rng.uniform(9, -0.4, 0.4)
        f, g, k, two = R.gcdf_label(arm, p, q, Z, m)
        if two[1] - two[0] < 1e-4:
            continue  # near a tie between two samples: f is not differentiable
        if abs(R.sdf(arm, p, q)) < 1e-3:
            continue  # the sign flips across the surface
        h = 1e-7
        fd = np.array([(fn(q + h * e) - fn(q - h * e)) / (2 * h) for e in np.eye(9)])
        np.testing.assert_allclose(fd, g, atol=1e-6)
        checked += 1
    assert checked >= 5


def test_sdf_translation_equivariance():
    """Sec. III-C: f_s(p + [dx, dy, 0], q + [dx, dy, 0...]) = f_s(p, q)."""
    arm = R.MobileArm()
    rng = synth.SplitMix64(40)
    for _ in range(10):
        q = np.concatenate([rng.uniform(2, -3, 3), rng.uniform(7, -math.pi, math.pi)])
        p = rng.uniform(3, -1, 1) + np.array([q[0], q[1], 0.8])
        d = rng.uniform(2, -5, 5)
        q2 = q.copy()
        q2[:2] += d
        p2 = p.copy()
        p2[:2] += d
        assert R.sdf(arm, p2, q2) == pytest.approx(R.sdf(arm, p, q), abs=1e-12)


def test_contact_configuration_has_zero_sdf():
    """Placing p on a capsule surface of a random q gives f_s(p, q) = 0."""
    arm = R.mobile_arm_7()
    rng = synth.SplitMix64(41)
    for _ in range(5):
        q = np.concatenate([rng.uniform(2, -1, 1), rng.uniform(8, -math.pi, math.pi)])
        A, B, Rr = arm.capsules(q)
        # the top of the base capsule's axis, moved up by its radius
        p = B[0] + np.array([0.0, 0.0, Rr[0]])
        # only meaningful if no arm link is closer
        if R.sdf(arm, p, q) < -1e-12:
            continue
        assert abs(R.sdf(arm, p, q)) < 1e-12
