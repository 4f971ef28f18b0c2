"""FP64 oracle: synthetic capsule robots and the brute-force GCDF (test infrastructure only).

The paper's robot geometry (a Kinova Gen3 on a mobile base, with a learned SDF)
is not available, so the field that the network approximates is defined here
on synthetic robots built from capsules (a segment with a radius).

  Robot SDF (Eq. 1): f_s(p, q) = min over capsules of (dist(p, segment) - r):
      positive outside the robot, negative inside, zero on its surface.
  Zero-level set (Eq. 2): Z(p) = {q : f_s(p, q) = 0}.  It is approximated by a
      finite sample (Sec. III-C, step ii): configurations are drawn at random
      and each is moved along a random straight line in configuration space
      until f_s changes sign; bisection on that sign places it on Z(p).
      (The paper descends f_s^2 with a quasi-Newton method; any procedure that
      lands on f_s = 0 produces valid members of Z(p).)
  GCDF label (Definition 1 / Eq. 8, second form):
      f(p, q) = sgn(f_s(p, q)) * min_{q_k in Z(p)} ||q - q_k||_M
  Gradient (Theorem 1, proof in Appendix A): with q_z the minimising sample,
      df/dq = M (q - q_z) / f, so ||df/dq||_{M^-1} = 1 and
      q - f * M^{-1} df/dq = q_z lies on Z(p) (single-step projection).

Configurations are q = [x, y, theta, a_1, ..., a_k]; the distance is the plain
weighted Euclidean norm with no angle wrapping, as in Definition 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# ---------------------------------------------------------------------------
# Geometry helpers
# ---------------------------------------------------------------------------

def segment_distance(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Euclidean distance from points p (..., 3) to segments [a, b] (..., 3)."""
    ab = b - a
    ap = p - a
    den = np.sum(ab * ab, axis=-1)
    t = np.where(den > 0, np.sum(ap * ab, axis=-1) / np.where(den > 0, den, 1.0), 0.0)
    t = np.clip(t, 0.0, 1.0)
    c = a + t[..., None] * ab
    return np.linalg.norm(p - c, axis=-1)


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


_ROT = {"z": rot_z, "y": rot_y}


# ---------------------------------------------------------------------------
# Robots
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class MobileArm:
    """Omnidirectional base (x, y, yaw) carrying a serial arm of capsule links.

    Base: vertical capsule from z = 0.1 to 0.4 m, radius 0.35 m, at (x, y).
    Arm: mounted at (0.2, 0, 0.45) in the yawed base frame; joint k rotates
    about axes[k] of the current frame, then the frame moves by offsets[k]
    along its own z axis; each link is the capsule between consecutive frame
    origins with radius radii[k].
    """

    axes: tuple = ("z", "y", "y", "z", "y", "z")
    offsets: tuple = (0.15, 0.40, 0.35, 0.10, 0.10, 0.12)
    radii: tuple = (0.06, 0.06, 0.05, 0.05, 0.05, 0.04)
    base_radius: float = 0.35
    base_z: tuple = (0.1, 0.4)
    mount: tuple = (0.2, 0.0, 0.45)

    @property
    def n_dof(self) -> int:
        return 3 + len(self.axes)

    def capsules(self, q: np.ndarray):
        q = np.asarray(q, dtype=np.float64)
        x, y, th = q[0], q[1], q[2]
        Rb = rot_z(th)
        tb = np.array([x, y, 0.0])
        A = [tb + np.array([0.0, 0.0, self.base_z[0]])]
        B = [tb + np.array([0.0, 0.0, self.base_z[1]])]
        R = [self.base_radius]
        pos = tb + Rb @ np.asarray(self.mount, dtype=np.float64)
        rot = Rb
        for k, ax in enumerate(self.axes):
            rot = rot @ _ROT[ax](q[3 + k])
            nxt = pos + rot @ np.array([0.0, 0.0, self.offsets[k]])
            A.append(pos)
            B.append(nxt)
            R.append(self.radii[k])
            pos = nxt
        return np.array(A), np.array(B), np.array(R)


    def capsules_batch(self, Q: np.ndarray):
        """capsules() for K configurations at once: A, B (K, C, 3) and R (C,).
        The same forward kinematics, with the rotations as (K, 3, 3) stacks."""
        Q = np.asarray(Q, dtype=np.float64).reshape(-1, self.n_dof)
        K = Q.shape[0]
        tb = np.stack([Q[:, 0], Q[:, 1], np.zeros(K)], axis=1)
        rot = _rot_batch("z", Q[:, 2])
        A = [tb + np.array([0.0, 0.0, self.base_z[0]])]
        B = [tb + np.array([0.0, 0.0, self.base_z[1]])]
        pos = tb + rot @ np.asarray(self.mount, dtype=np.float64)
        for k, ax in enumerate(self.axes):
            rot = rot @ _rot_batch(ax, Q[:, 3 + k])
            nxt = pos + self.offsets[k] * rot[:, :, 2]
            A.append(pos)
            B.append(nxt)
            pos = nxt
        R = np.array([self.base_radius] + list(self.radii))
        return np.stack(A, axis=1), np.stack(B, axis=1), R


def _rot_batch(axis: str, a: np.ndarray) -> np.ndarray:
    """rot_z / rot_y for an array of angles: (K, 3, 3)."""
    c, s = np.cos(a), np.sin(a)
    o, z = np.ones_like(a), np.zeros_like(a)
    if axis == "z":
        rows = [[c, -s, z], [s, c, z], [z, z, o]]
    else:
        rows = [[c, z, s], [z, o, z], [-s, z, c]]
    return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)


def mobile_arm_7() -> MobileArm:
    """10-DOF variant: a seventh (y) joint before the last link."""
    return MobileArm(axes=("z", "y", "y", "z", "y", "y", "z"),
                     offsets=(0.15, 0.40, 0.35, 0.10, 0.10, 0.08, 0.10),
                     radii=(0.06, 0.06, 0.05, 0.05, 0.05, 0.04, 0.04))


@dataclasses.dataclass
class PlanarLink:
    """1-DoF planar link (Fig. 3 of Sec. III-B): one capsule from the origin
    along (cos theta, sin theta, 0), length `length`, radius `radius`."""

    length: float = 1.0
    radius: float = 0.1

    n_dof: int = 1

    def capsules(self, q):
        th = float(np.asarray(q)[0])
        a = np.zeros(3)
        b = np.array([self.length * math.cos(th), self.length * math.sin(th), 0.0])
        return a[None], b[None], np.array([self.radius])


@dataclasses.dataclass
class BaseOnly:
    """Translation-only robot (n = 2): the vertical base capsule at (x, y)."""

    radius: float = 0.35
    z: tuple = (0.1, 0.4)
    n_dof: int = 2

    def capsules(self, q):
        q = np.asarray(q, dtype=np.float64)
        a = np.array([q[0], q[1], self.z[0]])
        b = np.array([q[0], q[1], self.z[1]])
        return a[None], b[None], np.array([self.radius])


def sdf(robot, p: np.ndarray, q: np.ndarray) -> float:
    """Robot SDF f_s(p, q) of Eq. (1) for capsule geometry."""
    A, B, R = robot.capsules(q)
    d = segment_distance(np.asarray(p, dtype=np.float64)[None, :], A, B) - R
    return float(np.min(d))


def sdf_batch(robot, p: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """sdf() of one point p for K configurations Q (K, n) at once (robots
    with capsules_batch); equal to sdf() up to the rounding of the stacked
    rotation products."""
    A, B, R = robot.capsules_batch(Q)
    d = segment_distance(np.asarray(p, dtype=np.float64)[None, None, :], A, B) - R[None, :]
    return np.min(d, axis=1)


# ---------------------------------------------------------------------------
# Sampled zero-level set and the GCDF label
# ---------------------------------------------------------------------------

def _bisect(robot, p, q0, u, t_lo, t_hi, s_lo, tol=1e-12, max_iter=200):
    """Bisection on the sign of f_s along q0 + t u between t_lo and t_hi."""
    for _ in range(max_iter):
        tm = 0.5 * (t_lo + t_hi)
        sm = sdf(robot, p, q0 + tm * u)
        if abs(sm) < tol or (t_hi - t_lo) < 1e-15:
            return tm
        if (sm > 0) == (s_lo > 0):
            t_lo, s_lo = tm, sm
        else:
            t_hi = tm
    return 0.5 * (t_lo + t_hi)


def line_to_boundary(robot, p, q0, u, t_max, n_steps):
    """March q0 + t u for t in (0, t_max]; return the first boundary crossing
    placed by bisection, or None when the sign never changes."""
    s0 = sdf(robot, p, q0)
    if s0 == 0.0:
        return np.array(q0, dtype=np.float64)
    t_prev, s_prev = 0.0, s0
    for k in range(1, n_steps + 1):
        t = t_max * k / n_steps
        s = sdf(robot, p, q0 + t * u)
        if s == 0.0:
            return q0 + t * u
        if (s > 0) != (s_prev > 0):
            tb = _bisect(robot, p, q0, u, t_prev, t, s_prev)
            return q0 + tb * u
        t_prev, s_prev = t, s
    return None


def sample_zero_level_set(robot, p, starts: np.ndarray, dirs: np.ndarray,
                          t_max: float = 2.0, n_steps: int = 64) -> np.ndarray:
    """Members of Z(p): each start configuration moved along its direction (and,
    failing that, the opposite one) until f_s(p, .) = 0.  Returns (K', n)."""
    out = []
    for q0, u in zip(starts, dirs):
        z = line_to_boundary(robot, p, q0, u, t_max, n_steps)
        if z is None:
            z = line_to_boundary(robot, p, q0, -u, t_max, n_steps)
        if z is not None:
            out.append(z)
    return np.array(out).reshape(-1, robot.n_dof)


def sample_zero_level_set_batch(robot, p, starts: np.ndarray, dirs: np.ndarray,
                                t_max: float = 2.0, n_steps: int = 64, tol: float = 1e-12,
                                max_iter: int = 200) -> np.ndarray:
    """sample_zero_level_set with every line marched and bisected at once
    (robots with capsules_batch): the same march of n_steps points per line,
    the first sign change (or an exact zero) of f_s, bisection on the sign
    until |f_s| < tol, and the opposite direction for lines that never
    change sign.  Returns (K', n) in the order of the starts."""
    starts = np.asarray(starts, dtype=np.float64)
    dirs = np.asarray(dirs, dtype=np.float64)
    K, n = starts.shape
    found = np.zeros((K, n))
    ok = np.zeros(K, dtype=bool)
    for sgn in (1.0, -1.0):
        todo = np.nonzero(~ok)[0]
        if todo.size == 0:
            break
        q0, u = starts[todo], sgn * dirs[todo]
        ts = t_max * np.arange(n_steps + 1) / n_steps          # t = 0 (start), then the march
        pts = q0[:, None, :] + ts[None, :, None] * u[:, None, :]
        S = sdf_batch(robot, p, pts.reshape(-1, n)).reshape(todo.size, n_steps + 1)
        pos = S > 0
        change = np.zeros_like(S, dtype=bool)
        change[:, 1:] = (pos[:, 1:] != pos[:, :-1]) | (S[:, 1:] == 0.0)
        change[:, 0] = S[:, 0] == 0.0
        hit = change.any(axis=1)
        k = np.argmax(change, axis=1)
        exact = hit & (S[np.arange(todo.size), k] == 0.0)
        t_hit = np.where(exact, ts[k], 0.0)
        # bisection on [t_{k-1}, t_k] for the lines whose sign changed
        bis = hit & ~exact
        t_lo = np.where(bis, ts[np.maximum(k - 1, 0)], 0.0)
        t_hi = np.where(bis, ts[k], 0.0)
        s_lo = np.where(bis, S[np.arange(todo.size), np.maximum(k - 1, 0)], 1.0)
        tm = 0.5 * (t_lo + t_hi)
        active = bis.copy()
        for _ in range(max_iter):
            if not active.any():
                break
            ia = np.nonzero(active)[0]
            tm[ia] = 0.5 * (t_lo[ia] + t_hi[ia])
            sm = sdf_batch(robot, p, q0[ia] + tm[ia, None] * u[ia])
            done = (np.abs(sm) < tol) | ((t_hi[ia] - t_lo[ia]) < 1e-15)
            same = (sm > 0) == (s_lo[ia] > 0)
            upd_lo = ~done & same
            upd_hi = ~done & ~same
            t_lo[ia[upd_lo]] = tm[ia[upd_lo]]
            s_lo[ia[upd_lo]] = sm[upd_lo]
            t_hi[ia[upd_hi]] = tm[ia[upd_hi]]
            active[ia[done]] = False
        tm[active] = 0.5 * (t_lo[active] + t_hi[active])
        t_fin = np.where(exact, t_hit, tm)
        found[todo[hit]] = q0[hit] + t_fin[hit, None] * u[hit]
        ok[todo[hit]] = True
    return found[ok].reshape(-1, n)


def gcdf_label_batch(robot, p, Qs: np.ndarray, Z: np.ndarray, m_diag=None):
    """gcdf_label for configurations Qs (S, n) at once: f (S,), grad (S, n) and
    the two smallest distances (S, 2)."""
    Qs = np.asarray(Qs, dtype=np.float64)
    m = np.ones(Qs.shape[1]) if m_diag is None else np.asarray(m_diag, dtype=np.float64)
    diff = Qs[:, None, :] - Z[None, :, :]
    d = np.sqrt(np.sum(diff * diff * m[None, None, :], axis=2))
    k = np.argmin(d, axis=1)
    sgn = np.where(sdf_batch(robot, p, Qs) >= 0, 1.0, -1.0)
    f = sgn * d[np.arange(Qs.shape[0]), k]
    dk = diff[np.arange(Qs.shape[0]), k]
    safe = np.where(f != 0, f, 1.0)
    grad = np.where((f != 0)[:, None], m[None, :] * dk / safe[:, None], 0.0)
    two = np.sort(d, axis=1)[:, :2] if d.shape[1] >= 2 else np.repeat(d, 2, axis=1)
    return f, grad, two


def gcdf_label(robot, p, q, Z: np.ndarray, m_diag=None):
    """Definition 1 / Eq. (8): f = sgn(f_s(p, q)) * min_k ||q - Z_k||_M and the
    Theorem 1 gradient M (q - q_z) / f at the minimising sample q_z.

    Returns (f, grad, k_star, d_sorted) where d_sorted holds the two smallest
    distances (used to skip near-ties, where f is not differentiable)."""
    q = np.asarray(q, dtype=np.float64)
    m = np.ones(q.size) if m_diag is None else np.asarray(m_diag, dtype=np.float64)
    diff = q[None, :] - Z
    d = np.sqrt(np.sum(diff * diff * m[None, :], axis=1))
    k = int(np.argmin(d))
    sgn = 1.0 if sdf(robot, p, q) >= 0 else -1.0
    f = sgn * d[k]
    grad = m * diff[k] / f if f != 0 else np.zeros(q.size)
    two = np.sort(d)[:2]
    return f, grad, k, two


def gcdf_label_field(robot, p, Z, m_diag=None):
    """q -> f(p, q) over a fixed sample Z (for finite differences)."""
    def fn(q):
        return gcdf_label(robot, p, q, Z, m_diag)[0]
    return fn
