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
same as placing p around the base.

Height levels (``n_heights``; the point grid and the reconstruction of
Eq. 5-7): the points lie on a few height levels; for each level one dense
subset Z~ is sampled around p = (0, 0, z) and moved by (p_x, p_y) to every
point of that level, which makes the sample of Z(p) much denser for the same
work (the label min_k ||q - z_k|| then overestimates f much less).

``make_samples`` returns FP64 arrays (marching and bisection run for all lines
at once through ``robot.sample_zero_level_set_batch``, which gives the same
samples as the line-by-line ``robot.sample_zero_level_set``);
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
    Z = R.sample_zero_level_set_batch(arm, p, starts, dirs, t_max=t_max, n_steps=n_steps)
    q = _configs(rng, n, per_point, p[:2], p_radius)
    if Z.shape[0] == 0:
        return q, None, None, Z
    f, g, _ = R.gcdf_label_batch(arm, p, q, Z, m_diag)
    return q, f, g, Z


def zero_level_subset(arm, z, n_zero, reach, rng, t_max=6.0, n_steps=192):
    """Z~(p) of Eq. (5) for p = (0, 0, z): members of Z(p) found from n_zero
    start configurations whose base lies within `reach` of p (yaw and joints
    uniform), each moved along a random direction of configuration space onto
    f_s = 0 (step ii of Sec. III-C).  By translation equivariance (Eq. 7) the
    set Z~ + (p_x, p_y, 0, ..., 0) is a sample of Z(p) for every point p at
    height z."""
    n = arm.n_dof
    p0 = np.array([0.0, 0.0, z])
    starts = _configs(rng, n, n_zero, p0[:2], reach)
    dirs = rng.uniform(n_zero * n, -1.0, 1.0).reshape(n_zero, n)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    return R.sample_zero_level_set_batch(arm, p0, starts, dirs, t_max=t_max, n_steps=n_steps)


def samples_on_levels(arm, subsets, levels, n_points, per_point, seed=0, p_radius=3.0, m_diag=None):
    """Labelled samples of points on height levels: each point p is drawn with
    its planar offset uniform over the disc of radius p_radius and its height
    one of `levels`; its zero-level sample is that level's subset Z~ moved by
    (p_x, p_y) (Eq. 7).  Returns (q, p, f, grad, gap)."""
    rng = synth.SplitMix64(seed)
    qs, ps, fs, gs, gaps = [], [], [], [], []
    while len(qs) < n_points:
        xy = _disc(rng.uniform(1), rng.uniform(1), p_radius)[0]
        lv = min(int(rng.uniform(1)[0] * len(levels)), len(levels) - 1)
        if subsets[lv].shape[0] == 0:
            continue
        p = np.array([xy[0], xy[1], levels[lv]])
        Z = subsets[lv].copy()
        Z[:, 0] += p[0]
        Z[:, 1] += p[1]
        q = _configs(rng, arm.n_dof, per_point, p[:2], p_radius)
        f, g, two = R.gcdf_label_batch(arm, p, q, Z, m_diag)
        qs.append(q)
        ps.append(np.repeat(p[None, :], per_point, axis=0))
        fs.append(f)
        gs.append(g)
        gaps.append(two[:, 1] - two[:, 0])
    return tuple(np.concatenate(x) for x in (qs, ps, fs, gs, gaps))


def make_samples(arm, n_points, per_point, n_zero, seed=0, p_radius=3.0, z_range=(0.0, 2.0), m_diag=None,
                 n_heights=None, reach=1.5, with_gap=False):
    """(q (S, n), p (S, 3), f (S,), grad (S, n)) with S = n_points * per_point
    (and, with_gap, the difference of the two smallest sample distances (S,),
    small where two contacts nearly tie and f is not differentiable).

    n_heights None: every point gets its own sample of Z(p) (n_zero lines from
    configurations within p_radius of it); points whose sample came out empty
    (no line reached the robot) are redrawn.
    n_heights T: the points lie on T height levels spread over z_range (the
    grid of Sec. III-C); each level's subset Z~ (Eq. 5, n_zero lines from
    configurations within `reach`) is computed once and moved to every point of
    that level (Eq. 7)."""
    if n_heights is not None:
        levels = np.linspace(z_range[0], z_range[1], n_heights)
        rng = synth.SplitMix64(seed)
        subsets = [zero_level_subset(arm, z, n_zero, reach, rng) for z in levels]
        out = samples_on_levels(arm, subsets, levels, n_points, per_point, seed + 1, p_radius, m_diag)
        return out if with_gap else out[:4]
    rng = synth.SplitMix64(seed)
    qs, ps, fs, gs, gaps = [], [], [], [], []
    while len(qs) < n_points:
        xy = _disc(rng.uniform(1), rng.uniform(1), p_radius)[0]
        p = np.array([xy[0], xy[1], rng.uniform(1, z_range[0], z_range[1])[0]])
        q, f, g, Z = point_samples(arm, p, n_zero, per_point, p_radius, rng, m_diag)
        if Z.shape[0] == 0:
            continue
        _, _, two = R.gcdf_label_batch(arm, p, q, Z, m_diag)
        qs.append(q)
        ps.append(np.repeat(p[None, :], per_point, axis=0))
        fs.append(f)
        gs.append(g)
        gaps.append(two[:, 1] - two[:, 0])
    out = (np.concatenate(qs), np.concatenate(ps), np.concatenate(fs), np.concatenate(gs))
    return out + (np.concatenate(gaps),) if with_gap else out


def _arm(n_dof):
    return R.mobile_arm_7() if n_dof == 10 else R.MobileArm()


def _job(args):
    n_dof, n_points, per_point, n_zero, seed, p_radius = args
    return make_samples(_arm(n_dof), n_points, per_point, n_zero, seed, p_radius, with_gap=True)


def _level_job(args):
    n_dof, z, n_zero, reach, seed = args
    return zero_level_subset(_arm(n_dof), z, n_zero, reach, synth.SplitMix64(seed))


def _levels_label_job(args):
    n_dof, subsets, levels, n_points, per_point, seed, p_radius = args
    return samples_on_levels(_arm(n_dof), subsets, levels, n_points, per_point, seed, p_radius)


def generate(n_dof=10, points=4096, per_point=256, zero=256, p_radius=3.0, seed=0, workers=8, n_heights=None,
             z_range=(0.0, 2.0), reach=1.5):
    """A data set in `workers` spawned processes (the pool is started with
    'spawn', so it may be used after CUDA was initialised in the caller):
    (q, p, f, grad, gap) concatenated in job order, deterministic for a seed.
    With n_heights, one job per level computes its subset Z~ (zero lines each),
    then the points are labelled in chunks against the moved subsets."""
    import multiprocessing as mp
    chunks = max(1, workers * 4)
    per = [points // chunks + (1 if k < points % chunks else 0) for k in range(chunks)]
    with mp.get_context("spawn").Pool(workers) as pool:
        if n_heights is None:
            jobs = [(n_dof, c, per_point, zero, seed * 1000003 + k, p_radius) for k, c in enumerate(per) if c]
            parts = pool.map(_job, jobs)
        else:
            levels = np.linspace(z_range[0], z_range[1], n_heights)
            subsets = pool.map(_level_job, [(n_dof, float(z), zero, reach, seed * 7919 + k)
                                            for k, z in enumerate(levels)])
            jobs = [(n_dof, subsets, levels, c, per_point, seed * 1000003 + k, p_radius)
                    for k, c in enumerate(per) if c]
            parts = pool.map(_levels_label_job, jobs)
    return tuple(np.concatenate([x[i] for x in parts]) for i in range(5))


def main(argv=None):
    ap = argparse.ArgumentParser(description="labelled (q, p, f) samples of the capsule robot's GCDF")
    ap.add_argument("--n-dof", type=int, default=10, choices=[9, 10])
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--per-point", type=int, default=256)
    ap.add_argument("--zero", type=int, default=256, help="zero-level lines per point (or per height level)")
    ap.add_argument("--heights", type=int, default=None, help="height levels of the point grid (Eq. 5-7)")
    ap.add_argument("--p-radius", type=float, default=3.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--out", required=True, help=".npz file to write")
    a = ap.parse_args(argv)
    q, p, f, g, gap = generate(a.n_dof, a.points, a.per_point, a.zero, a.p_radius, a.seed, a.workers, a.heights)
    np.savez(a.out, q=q, p=p, f=f, grad=g, gap=gap)
    print(f"{q.shape[0]} samples -> {a.out}")


if __name__ == "__main__":
    main()
