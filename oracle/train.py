"""FP64 oracle of the training protocol's parts (Sec. 4.4).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the product never
imports it.  Plain numpy, written for checking by eye.

  loss          Eq. 16: lambda_1 * mean |A_hat - A| + (1 - lambda_1) * (1 - SSIM)
  ssim          the SSIM index the paper names in Eq. 16, in its standard form
                (Wang, Bovik, Sheikh, Simoncelli 2004): local means, variances
                and covariance under an 11 x 11 Gaussian window (sigma 1.5,
                weights summing to 1), constants C1 = (0.01 L)^2,
                C2 = (0.03 L)^2, averaged over the map.  Readings (the paper is
                silent): zero padding outside the map ("same" size), data range
                L = 1, and over a batch of Q maps the mean of the Q indices.
  ssim_grad     d SSIM / d A_hat, derived by hand from the definition above
  adam          one Adam step (Kingma & Ba 2015, Algorithm 1; the paper trains
                with PyTorch's Adam, whose defaults beta = (0.9, 0.999),
                eps = 1e-8 are taken), learning rates from Table I
  anneal_noise  Eq. 18: n_i = gamma * N3(0,1) * 2 / cbrt(N_s) * (1 - i / tau) for
                i < tau and 0 afterwards, added to the TX position in the unit
                cube of the normalised room (Eq. 17); the normal draws are
                passed in
"""
from __future__ import annotations

import math

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """11 x 11 Gaussian weights, sigma 1.5, normalised to sum 1."""
    r = np.arange(WIN) - WIN // 2
    g = np.exp(-(r ** 2) / (2 * SIGMA ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _filter(x: np.ndarray) -> np.ndarray:
    """(G * x)(p) = sum_d G(d) x(p + d) over the 11 x 11 window, zero outside
    the map.  x: [H, W]."""
    H, W = x.shape
    G = window()
    h = WIN // 2
    pad = np.zeros((H + 2 * h, W + 2 * h))
    pad[h:h + H, h:h + W] = x
    out = np.zeros((H, W))
    for dy in range(WIN):
        for dx in range(WIN):
            out += G[dy, dx] * pad[dy:dy + H, dx:dx + W]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two [H, W] maps."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    num = (2 * mx * my + C1) * (2 * sxy + C2)
    den = (mx * mx + my * my + C1) * (sxx + syy + C2)
    return num / den


def ssim(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM index of each map pair: x, y [Q, H, W] (or [H, W]) -> [Q] (or scalar)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.ndim == 2:
        return float(ssim_map(x, y).mean())
    return np.array([ssim_map(x[q], y[q]).mean() for q in range(x.shape[0])])


def ssim_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d SSIM(x, y) / d x for one [H, W] pair.

    With a = 2 mx my + C1, b = 2 sxy + C2, c = mx^2 + my^2 + C1,
    d = sxx + syy + C2 and s = a b / (c d) at every pixel p, the mean over the
    P pixels depends on x through mx = G*x, sxx = G*(x^2) - mx^2 and
    sxy = G*(x y) - mx my.  Per pixel
      ds/dmx  = (2 my b) / (c d) - s (2 mx) / c
      ds/dsxx = -s / d
      ds/dsxy = 2 a / (c d)
    so, with the adjoint of the zero-padded window sum (the same sum, since G
    is symmetric),
      dSSIM/dx = (1/P) [ G*(ds/dmx - 2 mx ds/dsxx - my ds/dsxy)
                         + 2 x G*(ds/dsxx) + y G*(ds/dsxy) ]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    a = 2 * mx * my + C1
    b = 2 * sxy + C2
    c = mx * mx + my * my + C1
    d = sxx + syy + C2
    s = a * b / (c * d)
    d_mx = 2 * my * b / (c * d) - s * 2 * mx / c
    d_sxx = -s / d
    d_sxy = 2 * a / (c * d)
    P = x.size
    g = _filter(d_mx - 2 * mx * d_sxx - my * d_sxy) + 2 * x * _filter(d_sxx) + y * _filter(d_sxy)
    return g / P


def loss(x: np.ndarray, y: np.ndarray, lam: float = 0.7) -> float:
    """Eq. 16 over a batch [Q, H, W]: lam * mean |x - y| + (1 - lam) * (1 - mean_q SSIM_q)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return float(lam * np.abs(x - y).mean() + (1 - lam) * (1 - ssim(x, y).mean()))


def loss_grad(x: np.ndarray, y: np.ndarray, lam: float = 0.7) -> np.ndarray:
    """d loss / d x for Eq. 16 (sign(0) = 0 for the L1 term)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    Q = x.shape[0]
    g = lam * np.sign(x - y) / x.size
    for q in range(Q):
        g[q] -= (1 - lam) * ssim_grad(x[q], y[q]) / Q
    return g


def adam(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step at step number t >= 1; returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    m_hat = m / (1 - beta1 ** t)
    v_hat = v / (1 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def anneal_noise(normals: np.ndarray, i: int, n_positions: int, gamma: float = 1.0,
                 tau: int = 10000) -> np.ndarray:
    """Eq. 18: noise on the normalised TX position at iteration i; normals
    [..., 3] are the N3(0,1) draws."""
    if i >= tau:
        return np.zeros_like(np.asarray(normals, np.float64))
    return gamma * np.asarray(normals, np.float64) * (2.0 / n_positions ** (1.0 / 3.0)) * \
        (1.0 - i / tau)
