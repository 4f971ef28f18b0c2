"""gcdf_collision_cost_noalloc: the collision cost for callers that must not
allocate device memory once running (for example an optimizer inside a
real-time control loop, where an allocation can block or fail at an
unpredictable moment).  Its temporaries live in one fixed array inside the
library, so it must give the results of gcdf_collision_cost, call after call.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import metrics

from _helpers import lib, need_gpu, random_traj, small_net, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _noalloc(g, torch, net, q, p, kind, param, off=None, idx=None, shift=None):
    """Call the C entry point directly through ctypes."""
    raw = g._lib.load()
    N = q.shape[0]
    cost = torch.full((N,), float("nan"), device="cuda")
    grad = torch.full((N, net.n_dof), float("nan"), device="cuda")
    amin = torch.full((N,), -7, device="cuda", dtype=torch.int32)
    P = N * p.shape[0] if off is None else int(idx.numel())
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    rc = raw.gcdf_collision_cost_noalloc(net.handle, ptr(q), N, ptr(p), p.shape[0], ptr(off), ptr(idx), P,
                                         ptr(shift), g._RED[kind], float(param), ptr(cost), ptr(grad), ptr(amin),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, g.last_error()
    return cost, grad, amin


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind,param", [("softmin", 0.02), ("min", 0.0), ("hinge", 0.05)])
def test_noalloc_matches_collision_cost_twice(prec, kind, param):
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=40, n_points=3000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, prec)
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    ref = [x.cpu().numpy() for x in g.collision_cost(net, q, p, kind, param)]
    for _ in range(2):  # the shared array keeps the previous call's contents
        got = [x.cpu().numpy() for x in _noalloc(g, torch, net, q, p, kind, param)]
        torch.cuda.synchronize()
        assert metrics.rel_err_scalar(got[0], ref[0]).max() <= TOL
        assert metrics.rel_err_vector(got[1], ref[1]).max() <= TOL
        assert np.array_equal(got[2], ref[2])


def test_noalloc_point_lists_and_shift_twice():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    q = random_traj(17, 9, 21, -3, 3)
    rng = synth.SplitMix64(22)
    p = synth.uniform_points(rng, 800, [-3, -3, 0], [3, 3, 2])
    off, idx = synth.random_partitions(rng, 17, 800, 500, p_empty=0.2)
    shift = synth.random_shift(rng, q)
    net = g.create_net(9, 256, 4, w, "bf16")
    args = [to_dev(torch, a) for a in (q, p, off, idx, shift)]
    ref = [x.cpu().numpy() for x in g.collision_cost(net, args[0], args[1], "softmin", 0.1, part_offsets=args[2],
                                                      part_idx=args[3], shift=args[4])]
    for _ in range(2):
        got = [x.cpu().numpy() for x in _noalloc(g, torch, net, args[0], args[1], "softmin", 0.1, args[2], args[3],
                                                  args[4])]
        empty = np.diff(off) == 0
        assert np.all(np.isinf(got[0][empty])) and np.array_equal(got[2], ref[2])
        assert metrics.rel_err_scalar(got[0][~empty], ref[0][~empty]).max() <= TOL
        assert metrics.rel_err_vector(got[1], ref[1]).max() <= TOL


def test_noalloc_rejects_requests_beyond_its_array():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    net = g.create_net(9, 256, 4, w, "bf16")
    q = to_dev(torch, random_traj(70000, 9, 3))  # 70000 x 256 floats of terms + the stash > 96 MiB
    p = to_dev(torch, synth.uniform_points(synth.SplitMix64(4), 10, [0, 0, 0], [1, 1, 1]))
    raw = g._lib.load()
    cost = torch.empty(70000, device="cuda")
    grad = torch.empty(70000, 9, device="cuda")
    rc = raw.gcdf_collision_cost_noalloc(net.handle, ctypes.c_void_p(q.data_ptr()), 70000,
                                         ctypes.c_void_p(p.data_ptr()), 10, None, None, 0, None, 1, 0.1,
                                         ctypes.c_void_p(cost.data_ptr()), ctypes.c_void_p(grad.data_ptr()), None,
                                         None)
    assert rc == g._lib.GCDF_EINVAL
    assert "scratch" in g.last_error()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_after_a_larger_call_with_other_values(prec):
    """The shared array keeps what the previous call left in it.  A larger call
    with other inputs and another reduction fills more of the array with other
    values first; the checked call must still match gcdf_collision_cost, which
    shows that it writes every word it reads."""
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=40, n_points=3000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, prec)
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    big_q = to_dev(torch, random_traj(300, 9, 77, -5, 5))
    big_p = to_dev(torch, synth.uniform_points(synth.SplitMix64(78), 5000, [-5, -5, 0], [5, 5, 2]))
    ref = [x.cpu().numpy() for x in g.collision_cost(net, q, p, "softmin", 0.02)]
    _noalloc(g, torch, net, big_q, big_p, "hinge", 0.3)
    torch.cuda.synchronize()
    got = [x.cpu().numpy() for x in _noalloc(g, torch, net, q, p, "softmin", 0.02)]
    assert metrics.rel_err_scalar(got[0], ref[0]).max() <= TOL
    assert metrics.rel_err_vector(got[1], ref[1]).max() <= TOL
    assert np.array_equal(got[2], ref[2])
