"""Shared test helpers: conversions between the oracle's FP64 projection and
the library's FP32 record layout, and the spectrum comparison rule."""
import math

import numpy as np

HALF_LOG2E = 0.5 / math.log(2.0)  # log2(e)/2


def oracle_proj_to_records(proj):
    """Oracle rows (mx, my, A, B, C, w, rx, ry) -> library records (FP32) with
    the inverse covariance scaled by log2(e)/2."""
    rec = np.array(proj, dtype=np.float64, copy=True)
    rec[..., 2:5] *= HALF_LOG2E
    return rec.astype(np.float32)


def spectrum_error(gpu, ref, slack, rel_tol):
    """Per-query check |gpu - ref| <= rel_tol * peak_q + slack (slack = the
    oracle's sum over Gaussians whose q lies in the FP32/FP64 cutoff band,
    where either decision is correct).  Returns (ok, worst error / peak net of
    the band slack, pixels whose difference needed the slack)."""
    gpu = np.asarray(gpu, np.float64)
    Q = ref.shape[0]
    worst, used, ok = 0.0, 0, True
    for q in range(Q):
        peak = max(float(np.abs(ref[q]).max()), 1e-30)
        d = np.abs(gpu[q] - ref[q])
        tol = rel_tol * peak
        used += int(np.count_nonzero((d > tol) & (d <= tol + slack[q])))
        if np.any(d > tol + slack[q]):
            ok = False
        worst = max(worst, float(np.maximum(d - slack[q], 0.0).max()) / peak)
    return ok, worst, used

