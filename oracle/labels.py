"""FP64 oracle: labelled (q, p, f) samples of a capsule robot's GCDF, the
training data of the differentiable fit (test infrastructure only).

Data generation of Sec. III-C, with the brute-force field of ``robot``:
  * a point p is drawn relative to the robot base: planar offset uniform over
    the disc of radius ``p_radius`` around the base (area-uniform), height
    uniform in ``z_range``;
  * its zero-level set Z(p) is sampled (step ii of Sec. III-C): ``n_zero``
    configurations drawn as below, each moved along a random direction of
    configuration space until f_s(p, .) changes sign, then bisected onto
    f_s = 0 (``robot.sample_zero_level_set``);
  * ``per_point`` configurations q are drawn: yaw and arm joints uniform in
    [-pi, pi] (the joint limits of the synthetic arm), base position p_xy
    minus a disc offset as above, so that p lies within ``p_radius`` of the
    base; each is labelled f = sgn f_s(p, q) * min_k ||q - z_k||_M with the
    Theorem 1 gradient M (q - q_z) / f (``robot.gcdf_label``).

By translation equivariance (Sec. III-C) placing the base around p is the
same as placing p around the base.  ``make_samples`` returns FP64 arrays;
``python -m oracle.labels`` writes a data set with a pool of worker processes.
"""
from __future__ import annotations

import argparse
import math

import numpy as np

import synth

from . import robot as R


def _disc(u1, u2, radius):
    r = radius * np.sqrt(u1)
    a = 2.0 * math.pi * u2
    return np.stack([r * np.cos(a), r * np.sin(a)], axis=-1)


def _configs(rng, n_dof, k, centre_xy, p_radius):
    """k configurations whose base lies within p_radius of centre_xy."""
    off = _disc(rng.uniform(k), rng.uniform(k), p_radius)
    ang = rng.uniform(k * (n_dof - 2), -math.pi, math.pi).reshape(k, n_dof - 2)
    return np.concatenate([centre_xy[None, :] - off, ang], axis=1)


def point_samples(arm, p, n_zero, per_point, p_radius, rng, m_diag=None, t_max=6.0, n_steps=192):
    """Z(p) and the labelled configurations of one point: (q, f, grad, Z);
    f and grad are None when no line reached the robot (Z empty).  Lines run
    t_max in configuration-space units (long enough to carry the base to a
    point p_radius away), marched in n_steps."""
    n = arm.n_dof
    p = np.asarray(p, dtype=np.float64)
    starts = _configs(rng, n, n_zero, p[:2], p_radius)
    dirs = rng.uniform(n_zero * n, -1.0, 1.0).reshape(n_zero, n)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Z = R.sample_zero_level_set(arm, p, starts, dirs, t_max=t_max, n_steps=n_steps)
    q = _configs(rng, n, per_point, p[:2], p_radius)
    if Z.shape[0] == 0:
        return q, None, None, Z
    f = np.empty(per_point)
    g = np.empty((per_point, n))
    for i in range(per_point):
        f[i], g[i], _, _ = R.gcdf_label(arm, p, q[i], Z, m_diag)
    return q, f, g, Z


def make_samples(arm, n_points, per_point, n_zero, seed=0, p_radius=3.0, z_range=(0.0, 2.0), m_diag=None):
    """(q (S, n), p (S, 3), f (S,), grad (S, n)) with S = n_points * per_point.
    Points whose sampled Z(p) came out empty (no line reached the robot) are
    redrawn."""
    rng = synth.SplitMix64(seed)
    qs, ps, fs, gs = [], [], [], []
    while len(qs) < n_points:
        xy = _disc(rng.uniform(1), rng.uniform(1), p_radius)[0]
        p = np.array([xy[0], xy[1], rng.uniform(1, z_range[0], z_range[1])[0]])
        q, f, g, Z = point_samples(arm, p, n_zero, per_point, p_radius, rng, m_diag)
        if Z.shape[0] == 0:
            continue
        qs.append(q)
        ps.append(np.repeat(p[None, :], per_point, axis=0))
        fs.append(f)
        gs.append(g)
    return np.concatenate(qs), np.concatenate(ps), np.concatenate(fs), np.concatenate(gs)


def _job(args):
    n_dof, n_points, per_point, n_zero, seed, p_radius = args
    arm = R.mobile_arm_7() if n_dof == 10 else R.MobileArm()
    return make_samples(arm, n_points, per_point, n_zero, seed, p_radius)


def main(argv=None):
    ap = argparse.ArgumentParser(description="labelled (q, p, f) samples of the capsule robot's GCDF")
    ap.add_argument("--n-dof", type=int, default=10, choices=[9, 10])
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--per-point", type=int, default=256)
    ap.add_argument("--zero", type=int, default=256, help="zero-level samples per point")
    ap.add_argument("--p-radius", type=float, default=3.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--out", required=True, help=".npz file to write")
    a = ap.parse_args(argv)
    import multiprocessing as mp
    chunks = max(1, a.workers * 4)
    per = [a.points // chunks + (1 if k < a.points % chunks else 0) for k in range(chunks)]
    jobs = [(a.n_dof, c, a.per_point, a.zero, a.seed * 1000003 + k, a.p_radius) for k, c in enumerate(per) if c]
    with mp.get_context("spawn").Pool(a.workers) as pool:
        parts = pool.map(_job, jobs)
    q, p, f, g = (np.concatenate([x[i] for x in parts]) for i in range(4))
    np.savez(a.out, q=q, p=p, f=f, grad=g)
    print(f"{q.shape[0]} samples -> {a.out}")


if __name__ == "__main__":
    main()
