"""Pins of the training-protocol oracle (Sec. 4.4: Eq. 16 loss with SSIM,
Eq. 17-18 anneal smoothing, Adam with Table I learning rates) against values
fixed outside it: the published SSIM window, closed forms on constant maps,
scipy's correlation, finite differences and torch's Adam on the CPU."""
import math

import numpy as np
import pytest
import torch
from scipy import ndimage

from oracle import train



def test_ssim_window_is_the_standard_one():
    """11-tap Gaussian, sigma 1.5, normalised: the 1-D weights used by every
    SSIM implementation since Wang et al. (2004)."""
    G = train.window()
    g1 = G.sum(axis=0)
    assert G.shape == (11, 11) and G.sum() == pytest.approx(1.0, abs=1e-15)
    want = [0.00102838, 0.00759876, 0.03600077, 0.10936069, 0.21300554, 0.26601172]
    assert g1[:6] == pytest.approx(want, abs=1e-8)
    assert np.allclose(G, np.outer(g1, g1), rtol=0, atol=1e-17)


def test_ssim_of_identical_maps_is_one():
    x = np.random.default_rng(0).uniform(0, 1, (20, 33))
    assert train.ssim(x, x) == pytest.approx(1.0, abs=1e-14)


def test_ssim_constant_maps_closed_form():
    """Constant maps alpha, beta: away from the zero-padded border every local
    variance vanishes and SSIM = (2 alpha beta + C1) / (alpha^2 + beta^2 + C1)."""
    a, b = 0.8, 0.3
    s = train.ssim_map(np.full((30, 40), a), np.full((30, 40), b))
    inner = s[5:-5, 5:-5]
    want = (2 * a * b + 0.01 ** 2) / (a * a + b * b + 0.01 ** 2)
    assert np.allclose(inner, want, rtol=1e-12, atol=0)


def test_ssim_matches_scipy_correlation():
    """The same index with the local statistics from scipy.ndimage.correlate
    (zero padding): an independent evaluation of the window sums."""
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (17, 29))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    G = train.window()

    def f(z):
        return ndimage.correlate(z, G, mode="constant", cval=0.0)

    mx, my = f(x), f(y)
    sxx, syy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    assert train.ssim(x, y) == pytest.approx(s.mean(), rel=1e-12)
    assert train.ssim(x, y) == pytest.approx(train.ssim(y, x), rel=1e-12)


def test_ssim_grad_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (12, 14))
    y = rng.uniform(0, 1, (12, 14))
    g = train.ssim_grad(x, y)
    h = 1e-6
    for (i, j) in [(0, 0), (5, 7), (11, 13), (3, 12), (6, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j] += h
        xm[i, j] -= h
        fd = (train.ssim(xp, y) - train.ssim(xm, y)) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-11)


def test_loss_eq16_and_its_gradient():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (2, 10, 12))
    y = rng.uniform(0, 1, (2, 10, 12))
    L = train.loss(x, y, 0.7)
    assert L == pytest.approx(0.7 * np.abs(x - y).mean() + 0.3 * (1 - train.ssim(x, y).mean()))
    g = train.loss_grad(x, y, 0.7)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 5), (0, 9, 11)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (train.loss(xp, y) - train.loss(xm, y)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-11)
    assert train.loss(y, y) == 0.0


def test_adam_first_step_and_torch():
    """Step 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps).
    Several steps agree with torch.optim.Adam (CPU, FP64)."""
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    t1, m, v = train.adam(th, g, np.zeros(50), np.zeros(50), 1, 1e-2)
    assert np.allclose(t1, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    p = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=8e-3)
    ours, m, v = th.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        gt = rng.normal(size=50)
        p.grad = torch.tensor(gt, dtype=torch.float64)
        opt.step()
        ours, m, v = train.adam(ours, gt, m, v, t, 8e-3)
    assert np.allclose(ours, p.detach().numpy(), rtol=0, atol=1e-14)


def test_anneal_noise_schedule():
    """Eq. 18: scale gamma * 2 / cbrt(N_s) at i = 0, half of it at tau / 2,
    zero from tau on; with N_s = 8 the i = 0 noise is the normal draw itself."""
    z = np.random.default_rng(5).normal(size=(4, 3))
    assert np.array_equal(train.anneal_noise(z, 0, 8), z)
    assert np.allclose(train.anneal_noise(z, 5000, 8, tau=10000), 0.5 * z, rtol=0, atol=1e-15)
    assert np.all(train.anneal_noise(z, 10000, 8) == 0)
    assert np.allclose(train.anneal_noise(z, 0, 1000, gamma=2.0), z * 2.0 * 2.0 / 10.0,
                       rtol=1e-14)
