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



def grad_error(gpu, ref, rel=1e-3, floor=1e-3, slack=None):
    """Element-wise gradient check of one parameter group:
    |g - g_ref| <= rel * |g_ref| + floor * max|g_ref| (+ slack) for every
    element (the floor keeps the bound defined where a component is ~0; the
    oracle's slack covers ReLU decisions an FP32 forward may take either
    way).  Returns (ok, worst ratio |g - g_ref| / bound (<= 1 passes), flat
    index of the worst element, its GPU value, its oracle value)."""
    a = np.asarray(gpu, np.float64).ravel()
    b = np.asarray(ref, np.float64).ravel()
    assert a.shape == b.shape, (a.shape, b.shape)
    if b.size == 0:
        return True, 0.0, -1, 0.0, 0.0
    bound = rel * np.abs(b) + floor * float(np.abs(b).max())
    if slack is not None:
        bound = bound + np.asarray(slack, np.float64).ravel()
    d = np.abs(a - b)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(bound > 0, d / np.where(bound > 0, bound, 1.0), np.where(d > 0, np.inf, 0.0))
    i = int(np.argmax(ratio))
    worst = float(ratio[i])
    return bool(worst <= 1.0), worst, i, float(a[i]), float(b[i])


def check_grads(named, tag, rel=1e-3, floor=1e-3):
    """Runs grad_error over (name, gpu, ref[, slack]) groups, prints each
    group's worst element and returns the worst ratio over all groups (<= 1
    passes)."""
    worst = 0.0
    for entry in named:
        name, a, b = entry[:3]
        sl = entry[3] if len(entry) > 3 else None
        ok, r, i, ga, gb = grad_error(a, b, rel, floor, sl)
        print(f"{tag} {name}: worst element {i}: gpu {ga:.6e} oracle {gb:.6e} "
              f"(|diff| / bound = {r:.2e})")
        worst = max(worst, r)
    print(f"{tag}: worst over all groups {worst:.2e} (<= 1 passes)")
    return worst
