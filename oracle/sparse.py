"""FP64 oracle: spatial partition, dense->sparse GCDF Jacobian and the
single-step projection (test infrastructure only).

Partition (Sec. IV-A).  Waypoint i considers the obstacle points within a
range of its reference base position b_i; the range is not given in the
paper.  Reading: planar distance, I_{M,i} = { j : (p_jx - b_ix)^2 +
(p_jy - b_iy)^2 <= R^2 }, in increasing point order.  The test is evaluated
in FP64 on the FP32 inputs: dx = p_x - b_x, dy = p_y - b_y, d2 = dx*dx + dy*dy
(two products rounded, then their sum), compared with R*R.

Jacobian (Eq. 17 and the projection matrices of Eq. 18).  Row k of the dense
(sum m_i) x n gradient block belongs to waypoint i_k; the sparse Jacobian of
the stacked constraints with respect to the state vector [x_1; ...; x_N],
x_i = [q_i, v_i] in R^{2n}, is the block product with P_i, which places the
identity I_n at the columns of q_i.  Reading: those columns start at
2n(i-1) (the printed offset 2Nn(i-1) exceeds the 2Nn columns for i >= 2;
x_i has 2n entries).

Projection (Theorem 1, property 2): q_z = q_0 - f(p, q_0) M^{-1} grad_q f(p, q_0).
"""
from __future__ import annotations

import numpy as np

from . import mlp


def partition(base_xy, points, radius):
    """CSR lists (offsets (N+1,), idx) of the points within planar range R."""
    b = np.asarray(base_xy, dtype=np.float32).astype(np.float64).reshape(-1, 2)
    p = np.asarray(points, dtype=np.float32).astype(np.float64).reshape(-1, 3)
    r2 = float(np.float64(np.float32(radius)) * np.float64(np.float32(radius)))
    offsets = [0]
    idx = []
    for i in range(b.shape[0]):
        dx = p[:, 0] - b[i, 0]
        dy = p[:, 1] - b[i, 1]
        d2 = dx * dx + dy * dy
        sel = np.nonzero(d2 <= r2)[0]
        idx.append(sel)
        offsets.append(offsets[-1] + sel.size)
    idx = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    return np.asarray(offsets, dtype=np.int64), idx.astype(np.int64)


def projection_matrix(i, n, N):
    """P_i in R^{n x 2Nn} (Eq. 18, with the column offset 2n(i-1), i 1-based)."""
    P = np.zeros((n, 2 * N * n))
    P[:, 2 * n * (i - 1): 2 * n * (i - 1) + n] = np.eye(n)
    return P


def jacobian_dense(grad, offsets, n, N):
    """Eq. (17) written out: the stacked blocks grad_i P_i, as a dense matrix."""
    grad = np.asarray(grad, dtype=np.float64).reshape(-1, n)
    offsets = np.asarray(offsets, dtype=np.int64)
    rows = []
    for i in range(1, N + 1):
        blk = grad[offsets[i - 1]: offsets[i]]
        rows.append(blk @ projection_matrix(i, n, N))
    return np.concatenate(rows, axis=0) if rows else np.zeros((0, 2 * N * n))


def jacobian_csr(grad, offsets, n):
    """The same Jacobian in CSR form: every row holds its n entries in column
    order (row_ptr, col_idx, values)."""
    grad = np.asarray(grad, dtype=np.float64).reshape(-1, n)
    offsets = np.asarray(offsets, dtype=np.int64)
    K = grad.shape[0]
    row_ptr = np.arange(K + 1, dtype=np.int64) * n
    col = np.empty(K * n, dtype=np.int64)
    for i in range(offsets.size - 1):
        for k in range(offsets[i], offsets[i + 1]):
            col[k * n: (k + 1) * n] = 2 * n * i + np.arange(n)
    return row_ptr, col, grad.reshape(-1).copy()


def project(q0, f, grad, m_diag=None):
    """Theorem 1: q_z = q_0 - f M^{-1} grad (per row)."""
    q0 = np.asarray(q0, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64).reshape(-1, 1)
    minv = 1.0 if m_diag is None else 1.0 / np.asarray(m_diag, dtype=np.float64)
    return q0 - f * (minv * grad)


def project_pairs(n_dof, hidden, n_layers, weights, q, p, offsets=None, idx=None, shift=None, m_diag=None):
    """Projected configuration of every pair (stacked order of Eq. 14) through
    the FP64 MLP oracle."""
    f, g = mlp.query(n_dof, hidden, n_layers, weights, q, p, offsets, idx, shift)
    if offsets is None:
        ii, _ = mlp.dense_pairs(q.shape[0], p.shape[0])
    else:
        ii, _ = mlp.csr_pairs(offsets, idx)
    return project(np.asarray(q, np.float64)[ii], f, g, m_diag)
