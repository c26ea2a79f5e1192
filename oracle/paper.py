"""FP64 oracle of the paper's own primitive and deformation head (Sec. 4.1-4.2,
Sec. 6.1).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the product never
imports it.  Plain numpy for the head, the C oracle's render for the sums.

Primitive n (Sec. 4.1): raw angular centre (u, v) normalised by the
hyperbolic map, Cholesky factor l = (l1, l2, l3) of the covariance
(Sec. 3.2: Sigma = L L^T, L = [[l1, 0], [l2, l3]]), attenuation
delta = sigmoid(a), complex response psi = (re, im).
Deformation (Sec. 4.2, Eq. 10-14): residuals (dmu_x, dmu_y, dpsi_re,
dpsi_im, ddelta) = F(gamma(mu), gamma(s)); the frame at s is
(mu + dmu, Sigma, psi + dpsi, delta + ddelta) (no covariance residual).
Spectrum (Eq. 13): A = sum_n psi_n K_n with K = delta exp(-q/2), per channel,
decomposed into magnitude and phase (Sec. 6.1).

Readings (the paper is silent or garbled):
  * centre -> pixels: the map with range [0, 2 pi] is the azimuth,
    x = W (tanh u + 1) / 2; the one with range [0, pi/2] the elevation,
    y = H (tanh v + 1) / 2; dmu is in pixels, added after the map;
  * Sigma in pixel units from the raw Cholesky entries (no exp);
  * the MLP input: gamma of the reference centre normalised to the unit
    square (x/W, y/H) with L_mean bands and of the TX position normalised by
    the room with L_tx bands (10 and 6 in Sec. 6.1);
  * "an eight-layer MLP with skip connections every two layers and a hidden
    width of 156" (Sec. 6.1): 8 hidden Linear+ReLU layers of width 156, the
    encoded input concatenated to the activations entering hidden layers 3, 5
    and 7, then a Linear output layer of width 5;
  * delta + ddelta is used as it comes (no clamp).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

SKIPS = (2, 4, 6)  # 0-based hidden layers whose input includes the encoding


def centres(u, v, H: int, W: int):
    """Reference-frame centres in pixels from the raw (u, v)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    return W * (np.tanh(u) + 1.0) / 2.0, H * (np.tanh(v) + 1.0) / 2.0


def covariance(l1, l2, l3):
    """Sigma = L L^T with L = [[l1, 0], [l2, l3]]: (Sxx, Sxy, Syy)."""
    l1, l2, l3 = (np.asarray(a, np.float64) for a in (l1, l2, l3))
    return l1 * l1, l1 * l2, l2 * l2 + l3 * l3


def mlp(feat: np.ndarray, Ws, bs) -> np.ndarray:
    """feat [R, din] -> [R, 5]: hidden layers with ReLU, the input features
    concatenated to the activations entering the layers listed in SKIPS."""
    h = feat
    n_hidden = len(Ws) - 1
    for l in range(n_hidden):
        x = np.concatenate([h, feat], 1) if l in SKIPS else h
        h = np.maximum(x @ np.asarray(Ws[l], np.float64).T + np.asarray(bs[l], np.float64), 0.0)
    return h @ np.asarray(Ws[-1], np.float64).T + np.asarray(bs[-1], np.float64)


def residuals(pscene, pmlp, tx, H: int, W: int) -> np.ndarray:
    """[Q, N, 5] = (dmu_x, dmu_y, dpsi_re, dpsi_im, ddelta) (Eq. 14)."""
    tx = np.atleast_2d(np.asarray(tx, np.float64))
    x0, y0 = centres(pscene.mu[:, 0], pscene.mu[:, 1], H, W)
    gm = np.stack([oracle.pe(np.array([x / W, y / H]), pmlp.L_mean) for x, y in zip(x0, y0)])
    rmin = np.asarray(pmlp.room_min, np.float64)
    rsz = np.asarray(pmlp.room_size, np.float64)
    gt = np.stack([oracle.pe((t - rmin) / rsz, pmlp.L_tx) for t in tx])
    Q, N = tx.shape[0], x0.shape[0]
    out = np.zeros((Q, N, 5))
    for q in range(Q):
        feat = np.concatenate([gm, np.repeat(gt[q:q + 1], N, 0)], 1)
        out[q] = mlp(feat, pmlp.W, pmlp.b)
    return out


def project(pscene, resid, H: int, W: int, q_cut: float):
    """Oracle records [Q, N, 8] for the real and the imaginary channel
    (mx, my, A, B, C, w, rx, ry; conic unscaled, w = delta psi_c)."""
    x0, y0 = centres(pscene.mu[:, 0], pscene.mu[:, 1], H, W)
    sxx, sxy, syy = covariance(pscene.chol[:, 0], pscene.chol[:, 1], pscene.chol[:, 2])
    det = sxx * syy - sxy * sxy
    A, B, C = syy / det, -sxy / det, sxx / det
    delta0 = 1.0 / (1.0 + np.exp(-np.asarray(pscene.attn_logit, np.float64)))
    psi0 = np.asarray(pscene.psi, np.float64)
    Q, N = resid.shape[0], x0.shape[0]
    recs = []
    for c in range(2):
        p = np.zeros((Q, N, 8))
        p[..., 0] = x0[None] + resid[..., 0]
        p[..., 1] = y0[None] + resid[..., 1]
        p[..., 2], p[..., 3], p[..., 4] = A[None], B[None], C[None]
        p[..., 5] = (delta0[None] + resid[..., 4]) * (psi0[None, :, c] + resid[..., 2 + c])
        p[..., 6] = np.sqrt(q_cut * sxx)[None]
        p[..., 7] = np.sqrt(q_cut * syy)[None]
        recs.append(p)
    return recs


def forward(pscene, pmlp, tx, H: int, W: int, q_cut: float, band: float = 1e-4,
            wrap: bool = False):
    """(magnitude, phase, re, im, slack, resid) of Eq. 13 with the paper's head;
    pmlp = None: no deformation."""
    tx = np.atleast_2d(np.asarray(tx, np.float64))
    N = pscene.mu.shape[0]
    resid = residuals(pscene, pmlp, tx, H, W) if pmlp is not None else np.zeros((tx.shape[0], N, 5))
    pre, pim = project(pscene, resid, H, W, q_cut)
    re, s_re = oracle.render(pre, H, W, q_cut, band, wrap=wrap)
    im, s_im = oracle.render(pim, H, W, q_cut, band, wrap=wrap)
    return np.hypot(re, im), np.arctan2(im, re), re, im, np.maximum(s_re, s_im), resid
