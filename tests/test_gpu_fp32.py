"""FP32 CUDA-core path against the FP64 oracle, element by element.

Tolerance 1e-5 relative (err_f, err_g of oracle.metrics) for per-pair values
and gradients and for the MIN / HINGE costs.  The SOFTMIN gradient amplifies a
value error e_f by |f| / T in the weights exp(-f / T); its bound is
1e-5 + 4 max|f| 1e-6 / T (FP32 values carry about 1e-6 relative error).
"""
import numpy as np
import pytest

import synth
from oracle import metrics

from _helpers import errs, lib, need_gpu, oracle_cost, oracle_query, random_traj, small_net, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _run_query(g, torch, prec, shape, w, q, p, offsets=None, idx=None, shift=None):
    net = g.create_net(shape.n_dof, shape.hidden, shape.n_layers, w, prec)
    args = dict(part_offsets=None if offsets is None else to_dev(torch, offsets),
                part_idx=None if idx is None else to_dev(torch, idx),
                shift=None if shift is None else to_dev(torch, shift))
    f, gr = g.query(net, to_dev(torch, q), to_dev(torch, p), **args)
    torch.cuda.synchronize()
    return f.cpu().numpy(), gr.cpu().numpy()


def test_query_tiny_workload():
    """64 waypoints x 256 points, every pair (the tiny FP32 query workload)."""
    torch = need_gpu()
    g = lib()
    wl = synth.tiny_query()
    f, gr = _run_query(g, torch, "fp32", wl.shape, wl.weights, wl.q, wl.p)
    f_ref, g_ref = oracle_query(wl.shape, wl.weights, wl.q, wl.p)
    ef, eg = errs(f, gr, f_ref, g_ref)
    assert ef["max"] <= TOL and eg["max"] <= TOL, (ef, eg)


@pytest.mark.parametrize("hidden,n_layers,n_dof", [(64, 2, 3), (128, 3, 9), (256, 5, 10), (512, 5, 10)])
def test_query_other_shapes_ragged(hidden, n_layers, n_dof):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(n_dof, hidden, n_layers, seed=5)
    q = random_traj(5, n_dof, 6)
    p = synth.uniform_points(synth.SplitMix64(7), 301, [-2, -2, 0], [2, 2, 2])
    f, gr = _run_query(g, torch, "fp32", shape, w, q, p)
    f_ref, g_ref = oracle_query(shape, w, q, p)
    ef, eg = errs(f, gr, f_ref, g_ref)
    assert ef["max"] <= TOL and eg["max"] <= TOL, (ef, eg)


def test_query_csr_partitions_with_shift():
    """Per-waypoint point lists (some empty, with repeats) and a base shift."""
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    q = random_traj(9, 9, 8, -4, 4)
    rng = synth.SplitMix64(9)
    p = synth.uniform_points(rng, 500, [-4, -4, 0], [4, 4, 2])
    off, idx = synth.random_partitions(rng, 9, 500, 150, p_empty=0.25)
    shift = synth.random_shift(rng, q)
    f, gr = _run_query(g, torch, "fp32", shape, w, q, p, off, idx, shift)
    f_ref, g_ref = oracle_query(shape, w, q, p, off, idx, shift)
    assert f.shape[0] == off[-1]
    ef, eg = errs(f, gr, f_ref, g_ref)
    assert ef["max"] <= TOL and eg["max"] <= TOL, (ef, eg)


@pytest.mark.parametrize("kind,param", [("min", 0.0), ("hinge", 0.05), ("softmin", 0.1), ("softmin", 0.02)])
def test_collision_cost_scene(kind, param):
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=12, n_points=1500)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp32")
    c, gc, am = g.collision_cost(net, to_dev(torch, wl.q), to_dev(torch, wl.p), kind, param)
    torch.cuda.synchronize()
    c, gc, am = c.cpu().numpy(), gc.cpu().numpy(), am.cpu().numpy()
    c_ref, g_ref, a_ref = oracle_cost(s, wl.weights, wl.q, wl.p, kind, param)
    f_all, _ = oracle_query(s, wl.weights, wl.q, wl.p)
    ec = metrics.rel_err_scalar(c, c_ref).max()
    eg = metrics.rel_err_vector(gc, g_ref).max()
    tol_g = TOL if kind != "softmin" else TOL + 4 * np.abs(f_all).max() * 1e-6 / param
    assert ec <= TOL, ec
    assert eg <= tol_g, (eg, tol_g)
    # argmin: the reported point attains the minimum within the value tolerance
    f_all = f_all.reshape(wl.q.shape[0], -1)
    for i in range(wl.q.shape[0]):
        assert f_all[i, am[i]] <= f_all[i].min() + TOL * max(1.0, abs(f_all[i].min()))


def test_collision_cost_csr_and_empty_lists():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    q = random_traj(11, 9, 12, -3, 3)
    rng = synth.SplitMix64(13)
    p = synth.uniform_points(rng, 700, [-3, -3, 0], [3, 3, 2])
    off, idx = synth.random_partitions(rng, 11, 700, 400, p_empty=0.3)
    shift = synth.random_shift(rng, q)
    net = g.create_net(9, 256, 4, w, "fp32")
    for kind, param in (("min", 0.0), ("hinge", 0.3), ("softmin", 0.1)):
        c, gc, am = g.collision_cost(net, to_dev(torch, q), to_dev(torch, p), kind, param,
                                     part_offsets=to_dev(torch, off), part_idx=to_dev(torch, idx),
                                     shift=to_dev(torch, shift))
        torch.cuda.synchronize()
        c, gc, am = c.cpu().numpy(), gc.cpu().numpy(), am.cpu().numpy()
        c_ref, g_ref, a_ref = oracle_cost(shape, w, q, p, kind, param, off, idx, shift)
        empty = np.diff(off) == 0
        assert np.array_equal(am[empty], a_ref[empty])
        assert np.array_equal(c[empty], c_ref[empty])
        assert np.all(gc[empty] == 0)
        ne = ~empty
        assert metrics.rel_err_scalar(c[ne], c_ref[ne]).max() <= TOL
        assert metrics.rel_err_vector(gc[ne], g_ref[ne]).max() <= TOL


def test_empty_inputs():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    net = g.create_net(9, 256, 4, w, "fp32")
    q = to_dev(torch, random_traj(3, 9, 1))
    p0 = torch.zeros(0, 3, device="cuda")
    f, gr = g.query(net, q, p0)
    assert f.numel() == 0
    c, gc, am = g.collision_cost(net, q, p0, "softmin", 0.1)
    c2, gc2, am2 = g.collision_cost(net, q, p0, "hinge", 0.1)
    torch.cuda.synchronize()
    assert np.all(np.isinf(c.cpu().numpy())) and np.all(c2.cpu().numpy() == 0)
    assert np.all(am.cpu().numpy() == -1) and np.all(gc.cpu().numpy() == 0)
    q0 = torch.zeros(0, 9, device="cuda")
    f, gr = g.query(net, q0, to_dev(torch, synth.uniform_points(synth.SplitMix64(1), 10, [0, 0, 0], [1, 1, 1])))
    assert f.numel() == 0


def test_argument_errors():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    net = g.create_net(9, 256, 4, w, "fp32")
    q = to_dev(torch, random_traj(3, 9, 1))
    p = to_dev(torch, synth.uniform_points(synth.SplitMix64(1), 10, [0, 0, 0], [1, 1, 1]))
    with pytest.raises(g.GcdfError) as e:
        g.collision_cost(net, q, p, "softmin", 0.0)
    assert e.value.code == 1
    with pytest.raises(g.GcdfError):
        g.create_net(9, 256, 4, w[:-1], "fp32")
    # misaligned pointer (offset by one float)
    qq = torch.zeros(3 * 9 + 1, device="cuda")[1:].view(3, 9)
    with pytest.raises(g.GcdfError):
        g.query(net, qq, p)


def test_deterministic_repeat():
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=6, n_points=2000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp32")
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    a = [x.cpu().numpy() for x in g.collision_cost(net, q, p, "softmin", 0.02)]
    b = [x.cpu().numpy() for x in g.collision_cost(net, q, p, "softmin", 0.02)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_full_size_scene_sampled_waypoints():
    """The benchmark workload (128 waypoints x 16,384 points, soft-min T = 0.02)
    on the FP32 path in the bench's launch configuration; the oracle checks 4
    whole waypoints: per-pair f and df/dq within 1e-5, the soft-min cost within
    1e-5 and its gradient within the soft-min bound above."""
    from oracle import mlp
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene()
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp32")
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    c, gc, am = g.collision_cost(net, q, p, "softmin", 0.02)
    f, gr = g.query(net, q, p)
    torch.cuda.synchronize()
    wps = [0, 41, 90, 127]
    M = wl.p.shape[0]
    fs = f.cpu().numpy().reshape(-1, M)[wps].ravel()
    gs = gr.cpu().numpy().reshape(-1, M, 9)[wps].reshape(-1, 9)
    ii = np.repeat(wps, M)
    jj = np.tile(np.arange(M), len(wps))
    f_ref, gq_ref = mlp.eval_pairs(9, 256, 4, wl.weights, wl.q, wl.p, ii, jj)
    ef, eg = errs(fs, gs, f_ref, gq_ref)
    print("fp32 full-size sampled: err_f", ef, "err_g", eg)
    assert ef["max"] <= TOL and eg["max"] <= TOL, (ef, eg)
    c_ref, g_ref, _ = oracle_cost(s, wl.weights, wl.q, wl.p, "softmin", 0.02, waypoints=wps)
    ec = metrics.rel_err_scalar(c.cpu().numpy()[wps], c_ref).max()
    egc = metrics.rel_err_vector(gc.cpu().numpy()[wps], g_ref).max()
    print(f"fp32 full-size soft-min cost err {ec:.3e} grad err {egc:.3e}")
    assert ec <= TOL
    assert egc <= TOL + 4 * np.abs(f_ref).max() * 1e-6 / 0.02
