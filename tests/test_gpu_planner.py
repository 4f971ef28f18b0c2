"""Trajectory optimiser (gcdf_plan_solve) and planning server
(gcdf_plan_submit / gcdf_plan_poll) on the GPU, against the FP64 oracle of
oracle/planner.py and against themselves (batched == alone, bit for bit)."""
import time

import numpy as np
import pytest

import synth
from oracle import planner as pl

from _helpers import lib, need_gpu, small_net, to_dev

pytestmark = pytest.mark.gpu


def _params(g, iters, **kw):
    base = dict(dt=0.1, w_trans=1.0, w_rot=0.5, w_goal=100.0, mu=1.0, delta=0.05,
                lambda0=1.0, lambda_min=1e-6, lambda_max=1e8, iterations=iters, partition_radius=0.0)
    base.update(kw)
    return g.PlanParams(**base), pl.Params(lam0=base["lambda0"], lam_min=base["lambda_min"],
                                           lam_max=base["lambda_max"], iters=iters,
                                           **{k: base[k] for k in ("dt", "w_trans", "w_rot", "w_goal", "mu", "delta",
                                                                   "partition_radius")})


def _scene_problem(seed, N, M, n_dof=9):
    wl = synth.box_scene(n_waypoints=2, n_points=M, seed_scene=seed, seed_traj=seed + 100, n_dof=n_dof)
    return wl.q[0].astype(np.float32), wl.q[-1].astype(np.float32), wl.p.astype(np.float32), N


def _dev_problem(torch, qs, qg, pts, N):
    return {"n_waypoints": N, "q_start": to_dev(torch, qs), "q_goal": to_dev(torch, qg),
            "points": to_dev(torch, pts.reshape(-1, 3))}


@pytest.mark.parametrize("radius", [0.0, 2.0])
def test_plan_matches_oracle_step_by_step_fp32(radius):
    """FP32 field: the merit after every evaluation and every accept/reject
    decision follow the FP64 oracle (up to the first near-tie, if any), with
    every point or with the partition lists of radius 2 m."""
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "fp32")
    gp, op = _params(g, 8, mu=0.5, partition_radius=radius)
    probs = [_scene_problem(3, 12, 96), _scene_problem(5, 9, 64)]
    q, merit, acc = g.plan_solve(net, [_dev_problem(torch, *p) for p in probs], gp)
    q, merit, acc = q.cpu().numpy(), merit.cpu().numpy(), acc.cpu().numpy()
    row = 0
    for r, (qs, qg, pts, N) in enumerate(probs):
        field = pl.Field(9, shape.hidden, shape.n_layers, w, pts)
        Q, hist = pl.plan(qs, qg, N, field, op)
        m_ref, a_ref, t_ref = np.array(hist["merit"]), np.array(hist["accepted"]), np.array(hist["trial"])
        for k in range(op.iters + 1):
            if acc[r, k] != a_ref[k]:
                # only a near-tie may flip a decision
                assert abs(t_ref[k] - m_ref[k - 1]) <= 1e-5 * abs(m_ref[k - 1])
                break
            assert abs(merit[r, k] - m_ref[k]) <= 1e-5 * abs(m_ref[k])
        else:
            assert np.allclose(q[row: row + N], Q, rtol=1e-5, atol=1e-5)
        row += N


def test_obstacle_free_plan_reaches_the_least_squares_optimum():
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "bf16")
    gp, op = _params(g, 50, w_goal=50.0)
    r = synth.SplitMix64(5)
    qs = synth.random_config(r, 9, -2.0, 2.0).astype(np.float32)
    qg = synth.random_config(r, 9, -2.0, 2.0).astype(np.float32)
    N = 17
    field = pl.Field(9, shape.hidden, shape.n_layers, w, np.zeros((0, 3)))
    Q, _ = pl.plan(qs, qg, N, field, op)   # the oracle's value, pinned to least squares on the CPU
    q, merit, acc = g.plan_solve(net, [_dev_problem(torch, qs, qg, np.zeros((0, 3), np.float32), N)], gp)
    assert np.allclose(q.cpu().numpy(), Q, rtol=2e-6, atol=2e-6)
    assert np.all(np.diff(merit.cpu().numpy()[0]) <= 0)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_batched_problems_are_bit_identical_to_alone(prec):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, prec)
    gp, _ = _params(g, 6)
    probs = [_scene_problem(7, 40, 700), _scene_problem(8, 17, 129), _scene_problem(9, 64, 1000)]
    dev = [_dev_problem(torch, *p) for p in probs]
    qb, mb, ab = g.plan_solve(net, dev, gp)
    row = 0
    for r, p in enumerate(dev):
        qa, ma, aa = g.plan_solve(net, [p], gp)
        N = p["n_waypoints"]
        assert torch.equal(qa, qb[row: row + N])
        assert torch.equal(ma[0], mb[r]) and torch.equal(aa[0], ab[r])
        row += N


def test_bf16_plan_lowers_the_merit_and_agrees_with_fp64_evaluation():
    """BF16 field: the merit never increases; the merit the GPU reports for its
    final trajectory agrees with the FP64 oracle's cost of that trajectory."""
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "bf16")
    gp, op = _params(g, 20)
    qs, qg, pts, N = _scene_problem(11, 48, 2048)
    q, merit, acc = g.plan_solve(net, [_dev_problem(torch, qs, qg, pts, N)], gp)
    m = merit.cpu().numpy()[0]
    assert np.all(np.diff(m) <= 0) and m[-1] < m[0]
    field = pl.Field(9, shape.hidden, shape.n_layers, w, pts)
    J, _ = pl.total_cost_grad(q.cpu().numpy().astype(np.float64), qg, field, op)
    assert abs(J - m[-1]) <= 2e-2 * abs(J)


def test_rejects_bad_requests():
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "bf16")
    gp, _ = _params(g, 2)
    qs, qg, pts, _ = _scene_problem(3, 2, 16)
    with pytest.raises(g.GcdfError):
        g.plan_solve(net, [_dev_problem(torch, qs, qg, pts, 1)], gp)   # N < 2
    bad, _ = _params(g, 2, dt=0.0)
    with pytest.raises(g.GcdfError):
        g.plan_solve(net, [_dev_problem(torch, qs, qg, pts, 4)], bad)


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("radius", [0.0, 2.5])
def test_server_results_equal_solving_alone_in_a_mix(radius):
    """Requests of uneven size and two robots (9 and 10 DOF) submitted while
    others run: each result is bit-identical to gcdf_plan_solve of that
    request alone (continuous batching does not change any result), with and
    without partition lists."""
    torch = need_gpu()
    g = lib()
    nets = {}
    for n in (9, 10):
        shape, w = small_net(n)
        nets[n] = g.create_net(n, shape.hidden, shape.n_layers, w, "bf16")
    gp, _ = _params(g, 10, partition_radius=radius)
    reqs = [(9, _scene_problem(20, 32, 900)), (10, _scene_problem(21, 48, 400, n_dof=10)),
            (9, _scene_problem(22, 17, 1500)), (10, _scene_problem(23, 64, 256, n_dof=10)),
            (9, _scene_problem(24, 40, 3000))]
    srv = g.Server(budget_bytes=1 << 30, max_active=3, max_queued=16, params=gp)
    try:
        tickets = []
        for i, (n, (qs, qg, pts, N)) in enumerate(reqs):
            tickets.append(srv.submit(nets[n], N, qs, qg, pts))
            if i == 1:
                time.sleep(0.01)  # later requests arrive while the first ones run
        res = _wait(srv, tickets)
    finally:
        srv.close()
    for t, (n, (qs, qg, pts, N)) in zip(tickets, reqs):
        qa, ma, aa = g.plan_solve(nets[n], [_dev_problem(torch, qs, qg, pts, N)], gp)
        assert np.array_equal(res[t]["q"], qa.cpu().numpy())
        assert res[t]["merit"] == float(ma[0, -1].cpu())
        assert res[t]["accepted_steps"] == int(aa[0, 1:].sum().cpu())
        assert res[t]["submit_s"] <= res[t]["admit_s"] <= res[t]["done_s"]


def test_server_budget_admits_one_at_a_time():
    """A budget that holds one request but not two: admissions are serialised
    (each admitted after the previous one finished) and every result is the
    same; a request larger than the whole budget is refused."""
    torch = need_gpu()
    g = lib()
    from paper_2601_18548_gb300 import _lib
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "bf16")
    gp, _ = _params(g, 4)
    qs, qg, pts, N = _scene_problem(30, 24, 2000)
    need = g.plan_request_bytes(net, N, pts.shape[0])
    assert need > pts.shape[0] * 12
    srv = g.Server(budget_bytes=int(need * 1.5), max_active=8, max_queued=8, params=gp)
    try:
        ts = [srv.submit(net, N, qs, qg, pts) for _ in range(3)]
        r = _wait(srv, ts)
        with pytest.raises(g.GcdfError) as e:
            srv.submit(net, 2 * N, qs, qg, pts)  # needs more than the whole budget
        assert e.value.code == _lib.GCDF_EINVAL
    finally:
        srv.close()
    for x in ts[1:]:
        assert np.array_equal(r[x]["q"], r[ts[0]]["q"])
    times = sorted((r[x]["admit_s"], r[x]["done_s"]) for x in ts)
    for (a0, d0), (a1, d1) in zip(times, times[1:]):
        assert a1 >= d0


def test_server_queue_full_and_unknown_ticket():
    torch = need_gpu()
    g = lib()
    from paper_2601_18548_gb300 import _lib
    shape, w = small_net(9)
    net = g.create_net(9, shape.hidden, shape.n_layers, w, "bf16")
    gp, _ = _params(g, 30)
    qs, qg, pts, N = _scene_problem(31, 64, 4000)
    srv = g.Server(budget_bytes=1 << 40, max_active=1, max_queued=1, params=gp)
    try:
        codes = []
        ts = []
        for _ in range(6):
            try:
                ts.append(srv.submit(net, N, qs, qg, pts))
            except g.GcdfError as e:
                codes.append(e.code)
        assert _lib.GCDF_EAGAIN in codes
        with pytest.raises(g.GcdfError):
            srv._shapes[987654] = (N, 9)
            srv.poll(987654)
        _wait(srv, ts)
    finally:
        srv.close()
