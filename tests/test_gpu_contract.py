"""The header's device-side contracts, on the GPU.

* NaN / Inf inputs propagate to the affected outputs and nothing traps: a NaN
  or infinite configuration, or a NaN point, changes only the outputs of the
  pairs and waypoints that use it, which follow the FP64 oracle's NaN pattern
  (a NaN pair makes the waypoint's cost NaN in every reduction; MIN ranks NaN
  first; HINGE's gradient sums only pairs with f < delta), while every other
  output stays bit-identical to a clean run.  FP32 and BF16 paths.
* A bounded device wait that expires sets the net's status word: the
  self-test launch waits, with the tensor-core kernel's own wait routines, on a
  barrier nothing arrives on; both waits give up, the abort flag is raised,
  gcdf_device_status reports bit 0 and clears it, and the context stays usable.
"""
import numpy as np
import pytest

import synth

from _helpers import lib, need_gpu, oracle_cost, random_traj, small_net, to_dev

pytestmark = pytest.mark.gpu

KINDS = [("min", 0.0), ("softmin", 0.05), ("hinge", 0.3)]


def _cost(g, torch, net, q, p, kind, param, off=None, idx=None):
    out = g.collision_cost(net, to_dev(torch, q), to_dev(torch, p), kind, param,
                           part_offsets=None if off is None else to_dev(torch, off),
                           part_idx=None if idx is None else to_dev(torch, idx))
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out]


def _same_nan_pattern(a, b):
    return np.array_equal(np.isnan(a), np.isnan(b))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_nan_and_inf_configurations_poison_only_their_waypoints(prec):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9, 256, 4, seed=7)
    q = random_traj(7, 9, 31)
    p = synth.uniform_points(synth.SplitMix64(32), 700, [-2, -2, 0], [2, 2, 2])
    bad = q.copy()
    bad[2, 2] = np.nan      # yaw of waypoint 2
    bad[4, 0] = np.inf      # x of waypoint 4
    bad[5, 6] = -np.inf     # an arm joint of waypoint 5
    affected = [2, 4, 5]
    clean = [i for i in range(7) if i not in affected]
    net = g.create_net(9, 256, 4, w, prec)
    # query mode: the affected waypoints' pairs are not finite, the rest unchanged
    f0, g0 = [x.cpu().numpy() for x in g.query(net, to_dev(torch, q), to_dev(torch, p))]
    f1, g1 = [x.cpu().numpy() for x in g.query(net, to_dev(torch, bad), to_dev(torch, p))]
    torch.cuda.synchronize()
    assert g.device_status(net) == 0
    M = p.shape[0]
    f0, f1 = f0.reshape(7, M), f1.reshape(7, M)
    g0, g1 = g0.reshape(7, M, 9), g1.reshape(7, M, 9)
    assert np.array_equal(f1[clean], f0[clean]) and np.array_equal(g1[clean], g0[clean])
    assert not np.isfinite(f1[affected]).any()
    for kind, param in KINDS:
        c0, gc0, a0 = _cost(g, torch, net, q, p, kind, param)
        c1, gc1, a1 = _cost(g, torch, net, bad, p, kind, param)
        assert g.device_status(net) == 0
        assert np.array_equal(c1[clean], c0[clean]) and np.array_equal(gc1[clean], gc0[clean])
        assert np.array_equal(a1[clean], a0[clean])
        cr, gr, ar = oracle_cost(shape, w, bad, p, kind, param, waypoints=affected)
        print(prec, kind, "affected costs", c1[affected], "oracle", cr)
        assert np.isnan(c1[affected]).all() and np.isnan(cr).all()
        assert _same_nan_pattern(gc1[affected], gr), (kind, gc1[affected], gr)
        if kind == "min":
            assert np.array_equal(a1[affected], ar)  # the first NaN pair of the list


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_nan_point_poisons_only_the_lists_that_hold_it(prec):
    torch = need_gpu()
    g = lib()
    shape, w = small_net(9, 256, 4, seed=8)
    N, M = 6, 400
    q = random_traj(N, 9, 41)
    p = synth.uniform_points(synth.SplitMix64(42), M, [-2, -2, 0], [2, 2, 2])
    bad_p = p.copy()
    bad_p[137, 1] = np.nan
    # waypoints 1 and 3 list point 137; the others do not
    lists = []
    for i in range(N):
        js = [j for j in range(0, M, 1 + i) if j != 137]
        if i in (1, 3):
            js = sorted(js + [137])
        lists.append(js)
    off = np.concatenate([[0], np.cumsum([len(l) for l in lists])]).astype(np.int32)
    idx = np.concatenate(lists).astype(np.int32)
    net = g.create_net(9, 256, 4, w, prec)
    for kind, param in KINDS:
        c0, gc0, a0 = _cost(g, torch, net, q, p, kind, param, off, idx)
        c1, gc1, a1 = _cost(g, torch, net, q, bad_p, kind, param, off, idx)
        assert g.device_status(net) == 0
        clean = [0, 2, 4, 5]
        assert np.array_equal(c1[clean], c0[clean]) and np.array_equal(gc1[clean], gc0[clean])
        assert np.isnan(c1[[1, 3]]).all()
        cr, gr, ar = oracle_cost(shape, w, q, bad_p, kind, param, off, idx, waypoints=[1, 3])
        assert _same_nan_pattern(gc1[[1, 3]], gr), (kind, gc1[[1, 3]], gr)
        if kind == "min":
            assert np.array_equal(a1[[1, 3]], ar) and np.all(ar == 137)
        else:  # not NaN in the gradient: HINGE skips the NaN pair, SOFTMIN does not
            assert np.isnan(gc1[[1, 3]]).all() == (kind == "softmin")
    # query mode over the lists: only the pairs of point 137 change
    f0, _ = g.query(net, to_dev(torch, q), to_dev(torch, p), to_dev(torch, off), to_dev(torch, idx))
    f1, _ = g.query(net, to_dev(torch, q), to_dev(torch, bad_p), to_dev(torch, off), to_dev(torch, idx))
    f0, f1 = f0.cpu().numpy(), f1.cpu().numpy()
    hit = idx == 137
    assert np.isnan(f1[hit]).all() and np.array_equal(f1[~hit], f0[~hit])


def test_expired_wait_sets_the_status_word_and_the_context_survives():
    torch = need_gpu()
    g = lib()
    shape, w = small_net()
    net = g.create_net(9, 256, 4, w, "bf16")
    assert g.device_status(net) == 0
    seen = g.selftest_wait_expiry(net, 200000)   # ~0.1 ms at GB300 clocks
    assert seen == [1, 1, 1], seen
    assert g.device_status(net) == 1             # bit 0: a wait gave up
    assert g.device_status(net) == 0             # the read cleared it
    # the context is still usable: a normal call runs and reports no expiry
    q = to_dev(torch, random_traj(3, 9, 5))
    p = to_dev(torch, synth.uniform_points(synth.SplitMix64(6), 300, [-2, -2, 0], [2, 2, 2]))
    c, gc, am = g.collision_cost(net, q, p, "softmin", 0.1)
    torch.cuda.synchronize()
    assert np.isfinite(c.cpu().numpy()).all()
    assert g.device_status(net) == 0


def test_temporary_pool_trim_keeps_results_identical():
    """The temporaries come from a library-owned pool that keeps freed memory;
    trimming it between calls changes nothing in the results."""
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=9, n_points=3000)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "bf16")
    q, p = to_dev(torch, wl.q), to_dev(torch, wl.p)
    a = [x.cpu().numpy() for x in g.collision_cost(net, q, p, "softmin", 0.02)]
    torch.cuda.synchronize()
    g.release_cached_memory()
    b = [x.cpu().numpy() for x in g.collision_cost(net, q, p, "softmin", 0.02)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert g.device_status(net) == 0
