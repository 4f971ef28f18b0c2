"""FP64 oracle: per-waypoint collision cost and gradient (test infrastructure only).

The paper imposes f(p_j, q_i) - delta >= 0 for every waypoint i and every
point j of its partition (Eq. 11 and the stacked vector of Eq. 14) and, inside
the l1-penalty subproblem (Eq. 12), penalises each violated constraint
linearly.  The trajectory optimizer consumes one cost and one gradient per
waypoint, obtained by reducing the per-pair values over that waypoint's
points.  Three reductions are provided:

  MIN      c_i = min_j f_ij; argmin = first list position attaining it;
           grad_i = df/dq at that pair.
  SOFTMIN  c_i = -T log sum_j exp(-f_ij / T), evaluated with the minimum as
           shift; grad_i = sum_j w_ij df_ij/dq with w = softmax(-f_i / T).
  HINGE    c_i = sum_j max(0, delta - f_ij); grad_i = -sum_{f_ij < delta} df_ij/dq
           (the l1 penalty of Eq. 12 for the GCDF rows, summed per waypoint).

An empty partition gives MIN/SOFTMIN cost +inf, HINGE cost 0, a zero gradient
and argmin -1.
"""
from __future__ import annotations

import numpy as np

from . import mlp

MIN, SOFTMIN, HINGE = "min", "softmin", "hinge"


def reduce_waypoint(kind: str, param: float, f: np.ndarray, dq: np.ndarray, pidx: np.ndarray):
    """Reduce one waypoint's pairs.  f (m,), dq (m, n), pidx (m,) point indices."""
    n = dq.shape[1]
    if f.size == 0:
        cost = 0.0 if kind == HINGE else np.inf
        return cost, np.zeros(n), -1
    if kind == MIN:
        k = int(np.argmin(f))  # first occurrence of the minimum
        return float(f[k]), dq[k].copy(), int(pidx[k])
    if kind == SOFTMIN:
        T = float(param)
        m = float(np.min(f))
        e = np.exp(-(f - m) / T)
        s = float(np.sum(e))
        cost = m - T * np.log(s)
        grad = (e[:, None] * dq).sum(axis=0) / s
        return cost, grad, int(pidx[int(np.argmin(f))])
    if kind == HINGE:
        d = float(param)
        act = f < d
        cost = float(np.sum(np.maximum(0.0, d - f)))
        grad = -dq[act].sum(axis=0)
        return cost, grad, int(pidx[int(np.argmin(f))])
    raise ValueError(kind)


def collision_cost(n_dof, hidden, n_layers, weights, q, p, kind, param,
                   offsets=None, idx=None, shift=None, waypoints=None):
    """cost (N,), grad (N, n), argmin (N,) for every waypoint (or the listed ones)."""
    N, M = q.shape[0], p.shape[0]
    if offsets is None:
        offsets = np.arange(N + 1, dtype=np.int64) * M
        idx = np.tile(np.arange(M), N)
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    wps = np.arange(N) if waypoints is None else np.asarray(waypoints)
    cost = np.empty(wps.size)
    grad = np.empty((wps.size, n_dof))
    amin = np.empty(wps.size, dtype=np.int64)
    for r, i in enumerate(wps):
        jj = idx[offsets[i]: offsets[i + 1]]
        ii = np.full(jj.size, i)
        f, dq = mlp.eval_pairs(n_dof, hidden, n_layers, weights, q, p, ii, jj, shift)
        cost[r], grad[r], amin[r] = reduce_waypoint(kind, param, f, dq, jj)
    return cost, grad, amin
