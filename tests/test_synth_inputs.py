"""The seeded input generators (synth/) that both the oracle and the CUDA path
are fed from: the published SplitMix64 sequence, and the structure each
workload recipe states (weight bounds, configuration ranges, boxes inside the
room, points on the box surfaces with area weighting, linear waypoints)."""
import math

import numpy as np

import synth


def test_splitmix64_matches_the_published_sequence():
    # first outputs of Vigna's splitmix64 from state 0 (the reference C generator)
    r = synth.SplitMix64(0)
    assert [int(x) for x in r.next_u64(4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F, 0xF88BB8A8724C81EC]
    # the stream continues where it stopped, whatever the chunking
    a = synth.SplitMix64(12345)
    b = synth.SplitMix64(12345)
    assert np.array_equal(np.concatenate([a.next_u64(3), a.next_u64(5)]), b.next_u64(8))
    u = synth.SplitMix64(7).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3


def test_he_uniform_weights_bounds_and_order():
    shape = synth.NetShape(9, 256, 4)
    w = synth.he_uniform_weights(shape, seed=0)
    assert w.dtype == np.float32 and w.size == shape.n_params()
    assert np.array_equal(w, synth.he_uniform_weights(shape, seed=0))
    assert not np.array_equal(w, synth.he_uniform_weights(shape, seed=1))
    off = 0
    for (fo, fi) in shape.layer_dims():
        W = w[off: off + fo * fi]
        b = w[off + fo * fi: off + fo * fi + fo]
        wb, bb = math.sqrt(6.0 / fi), 1.0 / math.sqrt(fi)
        assert np.abs(W).max() <= wb * (1 + 1e-7) and np.abs(b).max() <= bb * (1 + 1e-7)
        if W.size > 1000:  # uniform: the spread fills the interval
            assert np.abs(W).max() > 0.99 * wb and abs(float(np.mean(W))) < 0.05 * wb
        off += fo * fi + fo
    assert off == w.size


def test_random_config_ranges():
    r = synth.SplitMix64(1)
    qs = np.stack([synth.random_config(r, 10, -2.0, 2.0) for _ in range(2000)])
    assert qs.shape == (2000, 10)
    assert qs[:, :2].min() >= -2.0 and qs[:, :2].max() <= 2.0
    assert qs[:, 2:].min() >= -math.pi and qs[:, 2:].max() <= math.pi
    assert qs[:, 2:].max() > 3.0 and qs[:, 2:].min() < -3.0


def test_box_scene_points_lie_on_box_surfaces_with_area_weighting():
    rs = synth.SplitMix64(3)
    centres, halves = synth.random_boxes(rs, 20, [-5, -5, 0], [5, 5, 2])
    edges = 2 * halves
    assert edges.min() >= 0.1 and edges.max() <= 1.0
    assert np.all(centres - halves >= np.array([-5, -5, 0]) - 1e-12)
    assert np.all(centres + halves <= np.array([5, 5, 2]) + 1e-12)
    m = 40000
    p = synth.box_surface_points(rs, centres, halves, m).astype(np.float64)
    # distance of every point to the surface of its nearest box: zero (FP32 storage)
    d = np.abs(p[:, None, :] - centres[None]) - halves[None]   # (m, boxes, 3)
    inside = np.all(d <= 1e-5, axis=2)                          # within the closed box
    on_face = np.any(np.abs(d) <= 1e-5, axis=2)                 # on one of its faces
    hit = inside & on_face
    assert hit.any(axis=1).all()
    # area weighting: the share of points on each box follows its surface area
    # (counting every box a point lies on, the overlaps are rare and small)
    area = 2 * (edges[:, 0] * edges[:, 1] + edges[:, 1] * edges[:, 2] + edges[:, 0] * edges[:, 2])
    first = np.argmax(hit, axis=1)
    share = np.bincount(first, minlength=20) / m
    expect = area / area.sum()
    assert np.abs(share - expect).max() < 0.01


def test_box_scene_workload_recipe():
    wl = synth.box_scene(n_waypoints=128, n_points=4096)
    assert wl.q.shape == (128, 9) and wl.p.shape == (4096, 3)
    assert wl.q.dtype == np.float32 and wl.p.dtype == np.float32
    assert wl.reduction == "softmin" and wl.param == 0.02
    # waypoints are equally spaced along a straight line in configuration space
    dq = np.diff(wl.q.astype(np.float64), axis=0)
    assert np.allclose(dq, dq[0], atol=1e-5)
    assert np.all(wl.p[:, :2] >= -5) and np.all(wl.p[:, :2] <= 5)
    assert np.all(wl.p[:, 2] >= 0) and np.all(wl.p[:, 2] <= 2)
    # the same seeds give the same scene
    again = synth.box_scene(n_waypoints=128, n_points=4096)
    assert np.array_equal(wl.p, again.p) and np.array_equal(wl.q, again.q) and np.array_equal(wl.weights, again.weights)
