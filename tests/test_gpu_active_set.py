"""HINGE and MIN with active sets (the default): a value-only pass over every
pair, then value and gradient over the pairs the reduction needs (f < delta,
or the first minimising entry).  Checked against the one-pass evaluation
(gcdf_set_active_set(net, 0)) and the FP64 oracle:

* a value-only query (grad NULL) gives the same f, bit for bit, as the query
  with gradients (the forward arithmetic is the same);
* MIN is bit-identical to one pass (the same pair is selected and its value
  and gradient are computed by the same arithmetic);
* HINGE gives the same active set, argmin and cost / gradient up to the order
  of its sums; all-inactive, all-active, empty and NaN-holding lists included.
"""
import numpy as np
import pytest

import synth
from oracle import metrics

from _helpers import lib, need_gpu, oracle_cost, random_traj, small_net, to_dev

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "fp16"]


def _both(g, torch, net, q, p, kind, param, off=None, idx=None, shift=None):
    args = dict(part_offsets=None if off is None else to_dev(torch, off),
                part_idx=None if idx is None else to_dev(torch, idx),
                shift=None if shift is None else to_dev(torch, shift))
    qd, pd = to_dev(torch, q), to_dev(torch, p)
    g.set_active_set(net, True)
    a = [x.cpu().numpy() for x in g.collision_cost(net, qd, pd, kind, param, **args)]
    g.set_active_set(net, False)
    b = [x.cpu().numpy() for x in g.collision_cost(net, qd, pd, kind, param, **args)]
    g.set_active_set(net, True)
    torch.cuda.synchronize()
    assert g.device_status(net) == 0
    return a, b


@pytest.mark.parametrize("prec", PRECS + ["fp8"])
def test_value_only_query_equals_the_value_of_the_full_query(prec):
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=9, n_points=1000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, prec)
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    f_full, _ = g.query(net, q, p)
    f_val, gr = g.query(net, q, p, with_grad=False)
    torch.cuda.synchronize()
    assert gr is None and g.device_status(net) == 0
    assert np.array_equal(f_val.cpu().numpy(), f_full.cpu().numpy())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_layers", [2, 3, 4])
def test_value_only_query_shapes(prec, n_layers):
    """Every depth (the forward-only tile tail differs from the full sweep's),
    with tile counts of 1, an odd count and many tiles per CTA pair."""
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9, 256, n_layers, seed=n_layers)
    net = g.create_net(9, 256, n_layers, w, prec)
    for n_wp, n_pts in ((1, 50), (3, 300), (40, 4100)):
        q = to_dev(torch, random_traj(n_wp, 9, 7 + n_wp))
        p = to_dev(torch, synth.uniform_points(synth.SplitMix64(n_pts), n_pts, [-2, -2, 0], [2, 2, 2]))
        f_full, _ = g.query(net, q, p)
        f_val, _ = g.query(net, q, p, with_grad=False)
        torch.cuda.synchronize()
        assert np.array_equal(f_val.cpu().numpy(), f_full.cpu().numpy()), (prec, n_layers, n_wp)


@pytest.mark.parametrize("prec", PRECS)
def test_min_is_bit_identical_to_one_pass(prec):
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=21, n_points=3000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, prec)
    a, b = _both(g, torch, net, wl.q, wl.p, "min", 0.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("delta", [-10.0, 0.3, 1.0, 100.0])
def test_hinge_matches_one_pass(prec, delta):
    """delta -10: nothing active (cost 0, zero gradient, argmin kept); 100: every
    pair active; 0.3 / 1.0: partly active lists."""
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=19, n_points=2500)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, prec)
    a, b = _both(g, torch, net, wl.q, wl.p, "hinge", delta)
    assert np.array_equal(a[2], b[2])  # argmin
    tol = 1e-5 if prec == "fp32" else 1e-4
    assert np.all(np.abs(a[0] - b[0]) <= tol * np.maximum(1.0, np.abs(b[0])))
    assert metrics.rel_err_vector(a[1], b[1]).max() <= tol
    if delta < 0:
        assert np.all(a[0] == 0) and np.all(a[1] == 0)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_hinge_and_min_csr_lists_with_empty_lists_shift_and_nan(prec):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9, 256, 4, seed=11)
    q = random_traj(15, 9, 12, -3, 3)
    rng = synth.SplitMix64(14)
    p = synth.uniform_points(rng, 900, [-3, -3, 0], [3, 3, 2])
    off, idx = synth.random_partitions(rng, 15, 900, 400, p_empty=0.3)
    shift = synth.random_shift(rng, q)
    p_nan = p.copy()
    p_nan[int(idx[off[2]]) if off[3] > off[2] else 0, 0] = np.nan
    net = g.create_net(9, 256, 4, w, prec)
    for pts in (p, p_nan):
        for kind, param in (("hinge", 0.4), ("min", 0.0)):
            a, b = _both(g, torch, net, q, pts, kind, param, off, idx, shift)
            assert np.array_equal(np.isnan(a[0]), np.isnan(b[0]))
            assert np.array_equal(np.isinf(a[0]), np.isinf(b[0]))  # MIN over an empty list: +inf
            assert np.array_equal(a[2], b[2])
            fin = np.isfinite(a[0])
            assert np.all(np.abs(a[0][fin] - b[0][fin]) <= 1e-4 * np.maximum(1.0, np.abs(b[0][fin])))
            empty = np.diff(off) == 0
            assert np.all(a[2][empty] == -1) and np.all(a[1][empty] == 0)
            if pts is p:
                c_ref, g_ref, _ = oracle_cost(shape, w, q, pts, kind, param, off, idx, shift)
                tol = 1e-5 if prec == "fp32" else 3e-2
                ne = ~empty
                assert metrics.rel_err_scalar(a[0][ne], c_ref[ne]).max() <= tol


def test_planner_collision_pass_uses_active_sets():
    """gcdf_plan_solve with the active set on and off: FP32 field, merits equal
    within 1e-5 relative (the HINGE sums are added in another order) and the
    same accept / reject decisions."""
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9, 256, 4, seed=0)
    net = g.create_net(9, 256, 4, w, "fp32")
    wl = synth.box_scene(n_waypoints=2, n_points=3000, seed_scene=41)
    r = synth.SplitMix64(42)
    probs = []
    for k in range(3):
        qs = synth.random_config(r, 9, -4, 4).astype(np.float32)
        qg = synth.random_config(r, 9, -4, 4).astype(np.float32)
        probs.append({"n_waypoints": 40 + 7 * k, "q_start": torch.from_numpy(qs).cuda(),
                      "q_goal": torch.from_numpy(qg).cuda(),
                      "points": torch.from_numpy(np.ascontiguousarray(wl.p[: 1000 + 900 * k])).cuda()})
    params = g.PlanParams(iterations=6, delta=0.3)
    g.set_active_set(net, True)
    qa, ma, aa = g.plan_solve(net, probs, params)
    g.set_active_set(net, False)
    qb, mb, ab = g.plan_solve(net, probs, params)
    g.set_active_set(net, True)
    ma, mb = ma.cpu().numpy(), mb.cpu().numpy()
    assert np.array_equal(aa.cpu().numpy(), ab.cpu().numpy())
    assert np.all(np.abs(ma - mb) <= 1e-5 * np.maximum(1.0, np.abs(mb)))
