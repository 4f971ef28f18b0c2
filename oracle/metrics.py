"""Relative-error measures for parity tests (test infrastructure only).

f can be close to zero, so a plain relative error is ill-conditioned.  Each
error is normalised by the larger of the reference's own magnitude and the
batch RMS of the reference:

    err_f = |f - f*| / max(|f*|, rms(f*))
    err_g = ||g - g*||_2 / max(||g*||_2, rms_k ||g*_k||_2)
"""
from __future__ import annotations

import numpy as np


def rel_err_scalar(x, ref):
    x = np.asarray(x, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if ref.size == 0:
        return np.zeros(0)
    rms = np.sqrt(np.mean(ref ** 2))
    den = np.maximum(np.abs(ref), rms)
    den = np.where(den > 0, den, 1.0)
    return np.abs(x - ref) / den


def rel_err_vector(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.shape[0] == 0:
        return np.zeros(0)
    x = x.reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    nr = np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(nr ** 2))
    den = np.maximum(nr, rms)
    den = np.where(den > 0, den, 1.0)
    return np.linalg.norm(x - ref, axis=1) / den


def summary(err):
    err = np.asarray(err)
    if err.size == 0:
        return {"max": 0.0, "p99": 0.0}
    return {"max": float(err.max()), "p99": float(np.quantile(err, 0.99))}
