"""FP64 oracle: trajectory optimisation with the GCDF collision cost
(test infrastructure only).

Problem (Sec. IV-A, Eq. 10).  Waypoints q_1 .. q_N of an n-DOF mobile
manipulator, q_1 = q_start fixed (the initial condition), velocity controls
eliminated through the integrator of Eq. (10): the rotational velocity of step
i is (q^r_{i+1} - q^r_i) / dt, and the base velocity is the planar difference
rotated into the base frame, whose norm equals || q^t_{i+1} - q^t_i || / dt
because a rotation keeps lengths.  The quadratic control cost J_c and a
goal-tracking cost J_t (both "standard quadratic costs") plus the l1 penalty
of the GCDF rows of Eq. (12) give

    J(Q) = (1/dt^2) sum_{i=1}^{N-1} sum_d W_d (q_{i+1,d} - q_{i,d})^2
           + w_goal ||q_N - q_goal||^2
           + mu sum_{i=1}^{N} sum_j max(0, delta - f(p_j, q_i))

with W_d = w_trans for x, y and w_rot for the yaw and the arm joints.

Iteration (the reading used here, since the paper's SCP solver is an external
package): a Levenberg-Marquardt step preconditioned by the exact Hessian of
the smooth part, which is block-diagonal over the DOFs and tridiagonal over
the waypoints,

    (A_d + lambda diag(A_d)) s_d = g_d   for every DOF d,   Q_trial = Q - s,

(with a partition radius R > 0 waypoint i only considers the points within
planar range R of its reference base, the (x, y) of the initial guess),

solved by a tridiagonal Cholesky factorisation in FP64.  A trial that lowers
J is accepted and lambda is halved (floor lambda_min); otherwise lambda is
multiplied by 4 (cap lambda_max).  A fixed number of steps, each one
collision-cost evaluation (the first evaluation is the initial guess, the
straight line from q_start to q_goal).  Configurations enter the field in
FP32 (the library's input type): the collision term is evaluated at the FP32
rounding of the trial, the smooth terms at its FP64 value.

Pins: tests/test_oracle_planner.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import reduce as red
from . import sparse


@dataclasses.dataclass
class Params:
    dt: float = 0.1
    w_trans: float = 1.0
    w_rot: float = 0.5
    w_goal: float = 100.0
    mu: float = 1.0
    delta: float = 0.05
    lam0: float = 1.0
    lam_min: float = 1e-6
    lam_max: float = 1e8
    iters: int = 50
    partition_radius: float = 0.0   # > 0: per-waypoint point lists (Sec. IV-A partitions)


def smooth_weights(n_dof, prm: Params) -> np.ndarray:
    W = np.full(n_dof, prm.w_rot)
    W[:2] = prm.w_trans
    return W


def smooth_cost_grad(Q, q_goal, prm: Params):
    """J_c + J_t and its gradient with respect to every waypoint (row 0, the
    fixed start, gets the formula's value too; callers ignore it)."""
    Q = np.asarray(Q, dtype=np.float64)
    W = smooth_weights(Q.shape[1], prm)
    s = 1.0 / (prm.dt * prm.dt)
    D = Q[1:] - Q[:-1]                       # (N-1, n) differences
    e = Q[-1] - np.asarray(q_goal, np.float64)
    J = s * float(np.sum(W * D * D)) + prm.w_goal * float(np.sum(e * e))
    G = np.zeros_like(Q)
    G[1:] += 2.0 * s * W * D                 # d/dq_{i+1} of (q_{i+1} - q_i)^2
    G[:-1] -= 2.0 * s * W * D                # d/dq_i
    G[-1] += 2.0 * prm.w_goal * e
    return J, G


def smooth_hessian_tridiag(N, n_dof, prm: Params):
    """Hessian of J_c + J_t over the free waypoints q_2 .. q_N, per DOF:
    diagonal (n, N-1) and sub-diagonal (n, N-2)."""
    W = smooth_weights(n_dof, prm)
    s = 2.0 / (prm.dt * prm.dt)
    m = N - 1
    diag = np.empty((n_dof, m))
    off = np.empty((n_dof, max(m - 1, 0)))
    for d in range(n_dof):
        diag[d, :] = 2.0 * s * W[d]
        diag[d, -1] = s * W[d] + 2.0 * prm.w_goal
        off[d, :] = -s * W[d]
    return diag, off


def tridiag_cholesky_solve(diag, off, rhs):
    """Solve T x = rhs for a symmetric positive definite tridiagonal T (diagonal
    `diag`, sub-diagonal `off`) by its Cholesky factor T = L L^T, L lower
    bidiagonal: l_0 = sqrt(t_0); e_i = off_{i-1} / l_{i-1};
    l_i = sqrt(t_i - e_i^2); then forward and back substitution."""
    m = len(diag)
    l = np.empty(m)
    e = np.zeros(m)
    y = np.empty(m)
    l[0] = np.sqrt(diag[0])
    y[0] = rhs[0] / l[0]
    for i in range(1, m):
        e[i] = off[i - 1] / l[i - 1]
        l[i] = np.sqrt(diag[i] - e[i] * e[i])
        y[i] = (rhs[i] - e[i] * y[i - 1]) / l[i]
    x = np.empty(m)
    x[m - 1] = y[m - 1] / l[m - 1]
    for i in range(m - 2, -1, -1):
        x[i] = (y[i] - e[i + 1] * x[i + 1]) / l[i]
    return x


def lm_step(G, diag, off, lam):
    """Step s (N, n) with s[0] = 0 (fixed start) from the gradient G (N, n)."""
    N, n = G.shape
    S = np.zeros_like(G)
    if N < 2:
        return S
    for d in range(n):
        S[1:, d] = tridiag_cholesky_solve(diag[d] * (1.0 + lam), off[d], G[1:, d])
    return S


def straight_line(q_start, q_goal, N):
    qs = np.asarray(q_start, np.float64)
    qg = np.asarray(q_goal, np.float64)
    t = np.arange(N, dtype=np.float64)[:, None] / max(N - 1, 1)
    return qs[None, :] + t * (qg - qs)[None, :]


class Field:
    """The collision term through the FP64 MLP oracle (Eq. 11 rows, HINGE)."""

    def __init__(self, n_dof, hidden, n_layers, weights, points, offsets=None, idx=None):
        self.shape = (n_dof, hidden, n_layers)
        self.weights = np.asarray(weights)
        self.points = np.asarray(points, dtype=np.float64).reshape(-1, 3)
        self.offsets, self.idx = offsets, idx

    def hinge(self, Q, delta):
        n_dof, H, L = self.shape
        N = Q.shape[0]
        if self.points.shape[0] == 0:
            return np.zeros(N), np.zeros((N, n_dof))
        q32 = np.asarray(Q, dtype=np.float32).astype(np.float64)
        c, g, _ = red.collision_cost(n_dof, H, L, self.weights, q32, self.points, red.HINGE, delta,
                                     self.offsets, self.idx)
        return c, g


def total_cost_grad(Q, q_goal, field: Field, prm: Params):
    Js, Gs = smooth_cost_grad(Q, q_goal, prm)
    c, gc = field.hinge(Q, prm.delta)
    J = Js + prm.mu * float(np.sum(c))
    G = Gs + prm.mu * gc
    return J, G


def plan(q_start, q_goal, N, field: Field, prm: Params, q_init=None):
    """Run prm.iters steps.  Returns the final trajectory (N, n) and a record
    per evaluation: merit after it, trial merit, accepted flag, lambda used."""
    Q = straight_line(q_start, q_goal, N) if q_init is None else np.array(q_init, dtype=np.float64)
    Q[0] = np.asarray(q_start, np.float64)
    n = Q.shape[1]
    if prm.partition_radius > 0:
        # lists around the reference bases: the (x, y) of the initial guess as the
        # field sees it (FP32)
        off, idx = sparse.partition(Q.astype(np.float32)[:, :2], field.points, prm.partition_radius)
        field = Field(*field.shape, field.weights, field.points, off, idx)
    diag, off = smooth_hessian_tridiag(N, n, prm)
    J, G = total_cost_grad(Q, q_goal, field, prm)
    lam = prm.lam0
    hist = {"merit": [J], "trial": [J], "accepted": [True], "lam": [lam]}
    for _ in range(prm.iters):
        S = lm_step(G, diag, off, lam)
        Qt = Q - S
        Jt, Gt = total_cost_grad(Qt, q_goal, field, prm)
        hist["lam"].append(lam)
        hist["trial"].append(Jt)
        if Jt < J:
            Q, J, G = Qt, Jt, Gt
            lam = max(lam * 0.5, prm.lam_min)
            hist["accepted"].append(True)
        else:
            lam = min(lam * 4.0, prm.lam_max)
            hist["accepted"].append(False)
        hist["merit"].append(J)
    return Q, hist
