"""Shared helpers for the GPU parity tests: inputs from `synth`, expected values
from `oracle`, results from the C ABI through the Python binding."""
import numpy as np
import pytest

import synth
from oracle import metrics, mlp, reduce as red


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    return g


def to_dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def oracle_query(shape, w, q, p, offsets=None, idx=None, shift=None):
    return mlp.query(shape.n_dof, shape.hidden, shape.n_layers, w, q, p, offsets, idx, shift)


def oracle_cost(shape, w, q, p, kind, param, offsets=None, idx=None, shift=None, waypoints=None):
    return red.collision_cost(shape.n_dof, shape.hidden, shape.n_layers, w, q, p, kind, param,
                              offsets, idx, shift, waypoints)


def errs(f, g, f_ref, g_ref):
    ef = metrics.rel_err_scalar(f, f_ref)
    eg = metrics.rel_err_vector(g, g_ref)
    return metrics.summary(ef), metrics.summary(eg)


def small_net(n_dof=9, hidden=256, n_layers=4, seed=0):
    shape = synth.NetShape(n_dof, hidden, n_layers)
    return shape, synth.he_uniform_weights(shape, seed)


def random_traj(n_wp, n_dof, seed, lo=-2.0, hi=2.0):
    r = synth.SplitMix64(seed)
    qs = synth.random_config(r, n_dof, lo, hi)
    qg = synth.random_config(r, n_dof, lo, hi)
    return synth.linear_trajectory(qs, qg, n_wp)
