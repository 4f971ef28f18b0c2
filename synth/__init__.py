"""Seeded synthetic inputs for the neural GCDF hot path.

This module only *draws numbers*: network weights, trajectories and obstacle
point clouds.  It holds none of the method's arithmetic (no encoding, no MLP,
no reduction), so both the FP64 oracle and the CUDA path may consume its
output without sharing any computation.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), stated here from its published
definition so the draw never depends on a library's generator:

    state <- state + 0x9E3779B97F4A7C15            (mod 2^64)
    z     <- state
    z     <- (z xor (z >> 30)) * 0xBF58476D1CE4E5B9 (mod 2^64)
    z     <- (z xor (z >> 27)) * 0x94D049BB133111EB (mod 2^64)
    out   <- z xor (z >> 31)

and a uniform double in [0, 1) is (out >> 11) * 2^-53.

Workload shapes follow the paper's problem statement (Sec. IV-A, Eq. 11: N
waypoints q_i in R^n, M obstacle points p_j in R^3, constraints for every
(i, j)) and its benchmark scenes (Sec. V-B: rectangular obstacles at varying
heights, allowed to overlap).  The network shape (4 hidden layers of width 256,
SiLU, sin/cos angle inputs; He-uniform weights) is the synthetic stand-in for
the paper's trained "7-layer MLP" (Sec. III-C), whose width is not printed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-style SplitMix64 stream; ``uniform(k)`` returns the next k doubles."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, k: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = np.arange(1, k + 1, dtype=np.uint64)
            z = self.state + steps * _GOLDEN
            self.state = self.state + np.uint64(k) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _MIX1
            z = (z ^ (z >> np.uint64(27))) * _MIX2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u


# ---------------------------------------------------------------------------
# Network description and weights
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class NetShape:
    """Shape of the coordinate MLP f(q, p).

    n_dof      n = 2 translational (x, y) + (n - 2) angles (base yaw + arm joints)
    hidden     H, width of every hidden layer
    n_layers   L, number of hidden (SiLU) layers; L - 1 of them are H x H
    """

    n_dof: int = 9
    hidden: int = 256
    n_layers: int = 4

    @property
    def n_angles(self) -> int:
        return self.n_dof - 2

    @property
    def d_q(self) -> int:
        # encoded configuration: x, y, then (sin, cos) of every angle
        return 2 + 2 * self.n_angles

    @property
    def d_in(self) -> int:
        # network input: point (3) followed by the encoded configuration
        return 3 + self.d_q

    def layer_dims(self):
        """(fan_out, fan_in) of every affine layer, input to output."""
        dims = [(self.hidden, self.d_in)]
        dims += [(self.hidden, self.hidden)] * (self.n_layers - 1)
        dims += [(1, self.hidden)]
        return dims

    def n_params(self) -> int:
        return sum(o * i + o for (o, i) in self.layer_dims())


def he_uniform_weights(shape: NetShape, seed: int = 0) -> np.ndarray:
    """Flat FP32 weight vector in the library's file order.

    Order: for every affine layer from input to output, the weight matrix
    (fan_out x fan_in, row-major; input columns of the first layer are
    [p_x, p_y, p_z, x, y, sin a_1, cos a_1, ..., sin a_k, cos a_k]) followed by
    its bias.  W ~ U(+-sqrt(6 / fan_in)) (He-uniform), b ~ U(+-1 / sqrt(fan_in)),
    each drawn from one SplitMix64 stream in that order and rounded to FP32.
    """
    rng = SplitMix64(seed)
    parts = []
    for (fan_out, fan_in) in shape.layer_dims():
        wb = math.sqrt(6.0 / fan_in)
        bb = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(fan_out * fan_in, -wb, wb))
        parts.append(rng.uniform(fan_out, -bb, bb))
    return np.concatenate(parts).astype(np.float32)


def unpack_weights(shape: NetShape, flat: np.ndarray):
    """Split a flat weight vector into [(W, b), ...] views (no arithmetic)."""
    out = []
    off = 0
    for (fan_out, fan_in) in shape.layer_dims():
        W = flat[off: off + fan_out * fan_in].reshape(fan_out, fan_in)
        off += fan_out * fan_in
        b = flat[off: off + fan_out]
        off += fan_out
        out.append((W, b))
    assert off == flat.size, (off, flat.size)
    return out


# ---------------------------------------------------------------------------
# Trajectories and point clouds
# ---------------------------------------------------------------------------

def random_config(rng: SplitMix64, n_dof: int, xy_lo: float, xy_hi: float) -> np.ndarray:
    """x, y ~ U[xy_lo, xy_hi]; base yaw and joints ~ U[-pi, pi]."""
    xy = rng.uniform(2, xy_lo, xy_hi)
    ang = rng.uniform(n_dof - 2, -math.pi, math.pi)
    return np.concatenate([xy, ang])


def linear_trajectory(q_start: np.ndarray, q_goal: np.ndarray, n_waypoints: int) -> np.ndarray:
    """Element-wise linear interpolation (angles are not wrapped), FP32 (N, n)."""
    t = np.linspace(0.0, 1.0, n_waypoints)[:, None]
    return ((1.0 - t) * q_start[None, :] + t * q_goal[None, :]).astype(np.float32)


def uniform_points(rng: SplitMix64, m: int, lo, hi) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = rng.uniform(3 * m).reshape(m, 3)
    return (lo + (hi - lo) * u).astype(np.float32)


def random_boxes(rng: SplitMix64, n_boxes: int, room_lo, room_hi, edge_lo=0.1, edge_hi=1.0):
    """Axis-aligned boxes (centre, half-extent) lying inside the room; may overlap."""
    room_lo = np.asarray(room_lo, dtype=np.float64)
    room_hi = np.asarray(room_hi, dtype=np.float64)
    edges = rng.uniform(3 * n_boxes, edge_lo, edge_hi).reshape(n_boxes, 3)
    u = rng.uniform(3 * n_boxes).reshape(n_boxes, 3)
    lo = room_lo + edges / 2
    hi = room_hi - edges / 2
    centres = lo + (hi - lo) * u
    return centres, edges / 2


def box_surface_points(rng: SplitMix64, centres, halves, m: int) -> np.ndarray:
    """m points uniform over the union of box surfaces, weighted by face area."""
    faces = []  # (box, axis, sign, area)
    for b in range(centres.shape[0]):
        h = halves[b]
        for ax in range(3):
            o1, o2 = [a for a in range(3) if a != ax]
            area = 4.0 * h[o1] * h[o2]
            faces.append((b, ax, -1.0, area))
            faces.append((b, ax, +1.0, area))
    areas = np.array([f[3] for f in faces])
    cdf = np.cumsum(areas) / areas.sum()
    u_face = rng.uniform(m)
    u_a = rng.uniform(m)
    u_b = rng.uniform(m)
    idx = np.minimum(np.searchsorted(cdf, u_face, side="right"), len(faces) - 1)
    pts = np.empty((m, 3), dtype=np.float64)
    for k in range(m):
        b, ax, sgn, _ = faces[idx[k]]
        o1, o2 = [a for a in range(3) if a != ax]
        c, h = centres[b], halves[b]
        p = np.empty(3)
        p[ax] = c[ax] + sgn * h[ax]
        p[o1] = c[o1] + (2 * u_a[k] - 1) * h[o1]
        p[o2] = c[o2] + (2 * u_b[k] - 1) * h[o2]
        pts[k] = p
    return pts.astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    shape: NetShape
    weights: np.ndarray          # flat FP32
    q: np.ndarray                # (N, n) FP32
    p: np.ndarray                # (M, 3) FP32
    reduction: str = "softmin"   # min | softmin | hinge
    param: float = 0.02          # temperature T (softmin) or margin delta (hinge)

    @property
    def n_pairs(self) -> int:
        return self.q.shape[0] * self.p.shape[0]


def tiny_query(n_waypoints: int = 64, n_points: int = 256) -> Workload:
    """9-DOF net (4 x 256 SiLU, seed 0); one trajectory of 64 waypoints linearly
    interpolated between two configurations drawn with seed 1 (x, y in [-2, 2]);
    256 points uniform in [-2, 2]^2 x [0, 2] (seed 2)."""
    shape = NetShape(9, 256, 4)
    w = he_uniform_weights(shape, seed=0)
    r1 = SplitMix64(1)
    qs = random_config(r1, 9, -2.0, 2.0)
    qg = random_config(r1, 9, -2.0, 2.0)
    q = linear_trajectory(qs, qg, n_waypoints)
    p = uniform_points(SplitMix64(2), n_points, [-2, -2, 0], [2, 2, 2])
    return Workload("tiny_query_64x256", shape, w, q, p, "min", 0.0)


def box_scene(n_waypoints: int = 128, n_points: int = 16384, n_boxes: int = 20,
              seed_scene: int = 3, seed_traj: int = 4, n_dof: int = 9,
              temperature: float = 0.02) -> Workload:
    """Single-trajectory scene: 9-DOF net (seed 0); room [-5, 5]^2 x [0, 2] with
    20 axis-aligned boxes (edges U[0.1, 1.0] m, seed 3); points area-weighted
    uniform on the box surfaces; waypoints linearly interpolated between two
    configurations in the room (seed 4); soft-min temperature 0.02."""
    shape = NetShape(n_dof, 256, 4)
    w = he_uniform_weights(shape, seed=0)
    rs = SplitMix64(seed_scene)
    centres, halves = random_boxes(rs, n_boxes, [-5, -5, 0], [5, 5, 2])
    p = box_surface_points(rs, centres, halves, n_points)
    rt = SplitMix64(seed_traj)
    qs = random_config(rt, n_dof, -5.0, 5.0)
    qg = random_config(rt, n_dof, -5.0, 5.0)
    q = linear_trajectory(qs, qg, n_waypoints)
    return Workload(f"box_scene_{n_waypoints}x{n_points}", shape, w, q, p, "softmin", temperature)


def random_partitions(rng: SplitMix64, n_waypoints: int, n_points: int, max_len: int,
                      p_empty: float = 0.1):
    """CSR point lists (offsets (N+1,), indices) of uneven length, some empty,
    standing in for the per-waypoint spatial partitions of Sec. IV-A."""
    lens = np.floor(rng.uniform(n_waypoints, 0, max_len + 1)).astype(np.int64)
    empty = rng.uniform(n_waypoints) < p_empty
    lens[empty] = 0
    offsets = np.zeros(n_waypoints + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(lens)
    idx = np.floor(rng.uniform(int(offsets[-1]), 0, n_points)).astype(np.int32)
    idx = np.minimum(idx, n_points - 1)
    return offsets, idx


def random_shift(rng: SplitMix64, q: np.ndarray, jitter: float = 0.3) -> np.ndarray:
    """Per-waypoint reference base position (N, 2): the waypoint's own x, y plus
    a uniform jitter, as a stand-in for the reference base of Sec. IV-A."""
    n = q.shape[0]
    j = rng.uniform(2 * n, -jitter, jitter).reshape(n, 2)
    return (q[:, :2].astype(np.float64) + j).astype(np.float32)
