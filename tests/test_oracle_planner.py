"""Pins of the trajectory-optimisation oracle (oracle/planner.py) against
what the mathematics fixes, independent of the oracle's own formulas."""
import dataclasses

import numpy as np

import synth
from oracle import planner as pl

from _helpers import small_net


def _residual_system(N, n, q_start, q_goal, prm):
    """J_c + J_t written as || R x - r ||^2 over x = [q_2 .. q_N] (row-major),
    from the definition: one residual per difference and per goal coordinate."""
    W = pl.smooth_weights(n, prm)
    m = N - 1
    rows, rhs = [], []
    for i in range(N - 1):          # residual sqrt(W_d) / dt (q_{i+1,d} - q_{i,d})
        for d in range(n):
            row = np.zeros(m * n)
            c = np.sqrt(W[d]) / prm.dt
            row[i * n + d] += c     # q_{i+1} is unknown i (0-based)
            if i == 0:
                rhs.append(c * q_start[d])
            else:
                row[(i - 1) * n + d] -= c
                rhs.append(0.0)
            rows.append(row)
    for d in range(n):              # residual sqrt(w_goal) (q_N - g)
        row = np.zeros(m * n)
        row[(m - 1) * n + d] = np.sqrt(prm.w_goal)
        rows.append(row)
        rhs.append(np.sqrt(prm.w_goal) * q_goal[d])
    return np.array(rows), np.array(rhs)


def test_tridiagonal_cholesky_matches_dense_solve():
    rng = np.random.default_rng(0)
    for m in (1, 2, 7, 64):
        off = rng.uniform(-1, 1, max(m - 1, 0))
        diag = np.abs(np.concatenate([[0.0], off])) + np.abs(np.concatenate([off, [0.0]])) + rng.uniform(0.1, 2, m)
        T = np.diag(diag) + np.diag(off, -1) + np.diag(off, 1)
        b = rng.normal(size=m)
        x = pl.tridiag_cholesky_solve(diag, off, b)
        assert np.allclose(x, np.linalg.solve(T, b), rtol=1e-12, atol=1e-12)


def test_smooth_hessian_matches_finite_differences_of_the_gradient():
    prm = pl.Params(dt=0.2, w_trans=1.5, w_rot=0.3, w_goal=7.0)
    rng = np.random.default_rng(1)
    N, n = 6, 4
    Q = rng.normal(size=(N, n))
    g = rng.normal(size=n)
    diag, off = pl.smooth_hessian_tridiag(N, n, prm)
    h = 1e-5
    for d in range(n):
        T = np.diag(diag[d]) + np.diag(off[d], -1) + np.diag(off[d], 1)
        for i in range(1, N):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[i, d] += h
            Qm[i, d] -= h
            col = (pl.smooth_cost_grad(Qp, g, prm)[1] - pl.smooth_cost_grad(Qm, g, prm)[1])[1:, d] / (2 * h)
            assert np.allclose(col, T[:, i - 1], rtol=1e-6, atol=1e-6)
            # no coupling between DOFs
            other = (pl.smooth_cost_grad(Qp, g, prm)[1] - pl.smooth_cost_grad(Qm, g, prm)[1])[1:, [k for k in range(n) if k != d]]
            assert np.abs(other).max() < 1e-6


def test_obstacle_free_plan_reaches_the_least_squares_optimum():
    """No points: J is quadratic; its minimiser is the least-squares solution
    of the residual system built above (a library solve)."""
    prm = pl.Params(dt=0.1, w_trans=1.0, w_rot=0.5, w_goal=50.0, iters=50)
    n = 9
    r = synth.SplitMix64(5)
    qs = synth.random_config(r, n, -2.0, 2.0)
    qg = synth.random_config(r, n, -2.0, 2.0)
    N = 17
    shape, w = small_net(n)
    field = pl.Field(n, shape.hidden, shape.n_layers, w, np.zeros((0, 3)))
    R, b = _residual_system(N, n, qs, qg, prm)
    x = np.linalg.lstsq(R, b, rcond=None)[0].reshape(N - 1, n)
    Q, hist = pl.plan(qs, qg, N, field, prm)
    # a step is accepted only when it lowers J (about 141 here) in FP64, so
    # near the minimum the position resolves to about sqrt(eps J / h_min) ~ 2e-8
    assert np.allclose(Q[1:], x, rtol=1e-7, atol=1e-7)
    assert np.array_equal(Q[0], qs.astype(np.float64))
    # one undamped step from the straight line is the Newton step of a quadratic
    prm0 = dataclasses.replace(prm, lam0=0.0, lam_min=0.0, iters=1)
    Q1, _ = pl.plan(qs, qg, N, field, prm0)
    assert np.allclose(Q1[1:], x, rtol=1e-9, atol=1e-9)


def test_total_gradient_matches_central_differences():
    """Smooth terms plus the hinge through the FP64 MLP, away from the kinks
    of the hinge (no pair within 1e-3 of delta)."""
    n = 9
    shape, w = small_net(n)
    r = synth.SplitMix64(8)
    pts = synth.uniform_points(r, 24, [-1.5, -1.5, 0.0], [1.5, 1.5, 1.5])
    qs = synth.random_config(r, n, -1.0, 1.0)
    qg = synth.random_config(r, n, -1.0, 1.0)
    N = 4
    Q = pl.straight_line(qs, qg, N)
    from oracle import mlp
    ii = np.repeat(np.arange(N), pts.shape[0])
    jj = np.tile(np.arange(pts.shape[0]), N)
    f, _ = mlp.eval_pairs(n, shape.hidden, shape.n_layers, w, Q, pts, ii, jj, None)
    delta = float(np.quantile(f, 0.4))  # about 40 % of the pairs active
    if np.min(np.abs(f - delta)) < 1e-3:
        delta += 2e-3
    prm = pl.Params(delta=delta, mu=0.7)

    class F64(pl.Field):  # no FP32 rounding of the field input, for the derivative check
        def hinge(self, Q, d):
            from oracle import reduce as red
            c, g, _ = red.collision_cost(n, shape.hidden, shape.n_layers, w, Q, pts, red.HINGE, d)
            return c, g

    field = F64(n, shape.hidden, shape.n_layers, w, pts)
    J, G = pl.total_cost_grad(Q, qg, field, prm)
    h = 1e-6
    for i in range(1, N):
        for d in range(n):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[i, d] += h
            Qm[i, d] -= h
            fd = (pl.total_cost_grad(Qp, qg, field, prm)[0] - pl.total_cost_grad(Qm, qg, field, prm)[0]) / (2 * h)
            assert abs(fd - G[i, d]) <= 1e-5 * max(1.0, abs(G[i, d]))


def test_plan_merit_never_increases_and_collisions_drop():
    n = 9
    shape, w = small_net(n)
    wl = synth.box_scene(n_waypoints=12, n_points=96)
    prm = pl.Params(iters=8, mu=0.5)
    field = pl.Field(n, shape.hidden, shape.n_layers, w, wl.p)
    Q, hist = pl.plan(wl.q[0], wl.q[-1], 12, field, prm)
    m = np.array(hist["merit"])
    assert np.all(np.diff(m) <= 0.0)
    acc = np.array(hist["accepted"][1:])
    tri = np.array(hist["trial"][1:])
    assert np.all(tri[acc] == m[1:][acc]) and np.all(tri[~acc] >= m[:-1][~acc])
    assert m[-1] < m[0]


def test_plan_at_rest_stays_at_rest():
    n = 9
    shape, w = small_net(n)
    q = synth.random_config(synth.SplitMix64(3), n, -1.0, 1.0)
    field = pl.Field(n, shape.hidden, shape.n_layers, w, np.zeros((0, 3)))
    Q, hist = pl.plan(q, q, 9, field, pl.Params(iters=3))
    assert np.array_equal(Q, np.tile(q.astype(np.float64), (9, 1)))
    assert hist["merit"][-1] == 0.0


def test_partition_with_an_unbounded_radius_changes_nothing_and_keeps_the_merit_monotone():
    n = 9
    shape, w = small_net(n)
    wl = synth.box_scene(n_waypoints=10, n_points=80)
    field = pl.Field(n, shape.hidden, shape.n_layers, w, wl.p)
    Q0, h0 = pl.plan(wl.q[0], wl.q[-1], 10, field, pl.Params(iters=5, mu=0.5))
    Q1, h1 = pl.plan(wl.q[0], wl.q[-1], 10, field, pl.Params(iters=5, mu=0.5, partition_radius=1e9))
    assert np.array_equal(Q0, Q1) and h0["merit"] == h1["merit"]
    Q2, h2 = pl.plan(wl.q[0], wl.q[-1], 10, field, pl.Params(iters=5, mu=0.5, partition_radius=1.5))
    assert np.all(np.diff(h2["merit"]) <= 0.0)
