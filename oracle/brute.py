"""Dense numpy brute force for tiny cases (TEST INFRASTRUCTURE ONLY).

An implementation of the forward path that is independent of oracle.c: the
covariance is assembled as R diag(sigma^2) R^T and inverted with
numpy.linalg.inv, the MLP is applied as whole-batch matrix products, and the
spectrum is evaluated for every pixel against every Gaussian by broadcasting
(no bounding boxes).  Memory grows as Q*N*H*W, so keep it to a few hundred
thousand pixel-Gaussian pairs per query.
"""
from __future__ import annotations

import numpy as np


def pe_batch(x: np.ndarray, L: int) -> np.ndarray:
    """Eq. 15 on rows of x [R,d]: [x, sin(2^k pi x)_{k<L}, cos(2^k pi x)_{k<L}]."""
    x = np.asarray(x, np.float64)
    freqs = (2.0 ** np.arange(L)) * np.pi                     # [L]
    ang = x[:, None, :] * freqs[None, :, None]                 # [R,L,d]
    R = x.shape[0]
    return np.concatenate([x, np.sin(ang).reshape(R, -1), np.cos(ang).reshape(R, -1)], axis=1)


def mlp_batch(feat: np.ndarray, Ws, bs) -> np.ndarray:
    h = np.asarray(feat, np.float64)
    for i, (W, b) in enumerate(zip(Ws, bs)):
        h = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if i + 1 < len(Ws):
            h = np.maximum(h, 0.0)
    return h


def deform(scene, mlp, tx, H, W):
    tx = np.atleast_2d(np.asarray(tx, np.float64))
    N, Q = scene.n, tx.shape[0]
    mu = np.asarray(scene.mean, np.float64) / np.array([W, H], np.float64)
    s = (tx - np.asarray(mlp.room_min)) / np.asarray(mlp.room_size)
    gm = pe_batch(mu, mlp.L_mean)                              # [N, 26]
    gs = pe_batch(s, mlp.L_tx)                                 # [Q, 63]
    feat = np.concatenate([np.broadcast_to(gm[None], (Q, N, gm.shape[1])),
                           np.broadcast_to(gs[:, None], (Q, N, gs.shape[1]))], axis=2)
    out = mlp_batch(feat.reshape(Q * N, -1), mlp.W, mlp.b)
    return out.reshape(Q, N, -1)


def render(scene, resid, H, W, q_cut, Q=1):
    """Dense evaluation of Eq. 13 for every pixel and Gaussian."""
    N = scene.n
    if resid is None:
        resid = np.zeros((Q, N, 5))
    Q = resid.shape[0]
    mean = np.asarray(scene.mean, np.float64)[None] + resid[..., 0:2]      # [Q,N,2]
    th = np.asarray(scene.rot, np.float64)[None] + resid[..., 2]
    ls = np.asarray(scene.log_scale, np.float64)[None] + resid[..., 3:5]
    c, s = np.cos(th), np.sin(th)
    Rm = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)       # [Q,N,2,2]
    D2 = np.zeros(Rm.shape)
    D2[..., 0, 0] = np.exp(2 * ls[..., 0])
    D2[..., 1, 1] = np.exp(2 * ls[..., 1])
    Sigma = Rm @ D2 @ np.swapaxes(Rm, -1, -2)
    Sinv = np.linalg.inv(Sigma)
    w = np.asarray(scene.amp, np.float64) / (1.0 + np.exp(-np.asarray(scene.opacity_logit, np.float64)))
    ys, xs = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    pix = np.stack([xs, ys], -1).reshape(-1, 2)                            # [P,2]
    out = np.zeros((Q, H * W))
    for q in range(Q):
        d = pix[None, :, :] - mean[q][:, None, :]                          # [N,P,2]
        qq = np.einsum("npi,nij,npj->np", d, Sinv[q], d)
        k = np.where(qq <= q_cut, np.exp(-0.5 * qq), 0.0)
        out[q] = (w[:, None] * k).sum(0)
    return out.reshape(Q, H, W)


def bin_brute(rec32, H, W, tw, th):
    """Every tile tested against every record rectangle, in FP32 as the
    records are stored; returns {(q, t): [ids ascending]}."""
    rec32 = np.asarray(rec32, np.float32)
    Q, N = rec32.shape[:2]
    ntx, nty = (W + tw - 1) // tw, (H + th - 1) // th
    f = np.float32
    mx, my, rx, ry = rec32[..., 0], rec32[..., 1], rec32[..., 6], rec32[..., 7]
    with np.errstate(invalid="ignore", over="ignore"):
        xlo, xhi = (mx - rx).astype(f), (mx + rx).astype(f)
        ylo, yhi = (my - ry).astype(f), (my + ry).astype(f)
        ok = (xhi >= 0) & (xlo <= f(W - 1)) & (yhi >= 0) & (ylo <= f(H - 1))
        px0 = np.ceil(np.maximum(xlo, f(0)))
        px1 = np.floor(np.minimum(xhi, f(W - 1)))
        py0 = np.ceil(np.maximum(ylo, f(0)))
        py1 = np.floor(np.minimum(yhi, f(H - 1)))
    ok &= (px0 <= px1) & (py0 <= py1)
    lists = {}
    for q in range(Q):
        for ty in range(nty):
            for tx in range(ntx):
                # tile pixel span intersects the pixel span of the footprint
                a0, a1 = tx * tw, min(W - 1, tx * tw + tw - 1)
                b0, b1 = ty * th, min(H - 1, ty * th + th - 1)
                hit = ok[q] & (px0[q] <= a1) & (px1[q] >= a0) & (py0[q] <= b1) & (py1[q] >= b0)
                ids = np.nonzero(hit)[0]
                if ids.size:
                    lists[(q, ty * ntx + tx)] = ids.astype(np.uint32)
    return lists
