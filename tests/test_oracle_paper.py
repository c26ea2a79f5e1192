"""Pins of the paper-head oracle (Sec. 4.1-4.2, Sec. 6.1) against closed forms
and constructed cases: the tanh centre map, the Cholesky covariance, one
primitive's magnitude / phase / lattice sum, the skip wiring of the 8 x 156
MLP, and each residual's effect."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import paper


def one(u, v, l1, l2, l3, a, psi):
    return synth.PaperScene(np.array([[u, v]]), np.array([[l1, l2, l3]]), np.array([a]),
                            np.array([psi]))


def test_centre_map():
    """x = W (tanh u + 1) / 2, y = H (tanh v + 1) / 2: u = v = 0 is the map's
    centre, the map is odd about it and saturates at the edges."""
    x, y = paper.centres(np.array([0.0, 0.7, -0.7, 30.0]), np.array([0.0, -1.3, 1.3, -30.0]), 90, 360)
    assert x[0] == 180.0 and y[0] == 45.0
    assert x[1] + x[2] == pytest.approx(360.0, abs=1e-12) and y[1] + y[2] == pytest.approx(90.0, abs=1e-12)
    assert x[3] == pytest.approx(360.0, abs=1e-9) and y[3] == pytest.approx(0.0, abs=1e-9)


def test_cholesky_covariance():
    rng = np.random.default_rng(0)
    l1, l2, l3 = rng.uniform(0.5, 4, 20), rng.normal(0, 1, 20), rng.uniform(0.5, 4, 20)
    sxx, sxy, syy = paper.covariance(l1, l2, l3)
    for i in range(20):
        L = np.array([[l1[i], 0.0], [l2[i], l3[i]]])
        S = np.array([[sxx[i], sxy[i]], [sxy[i], syy[i]]])
        assert np.allclose(L @ L.T, S, rtol=1e-14, atol=1e-14)
        assert np.linalg.det(S) == pytest.approx((l1[i] * l3[i]) ** 2, rel=1e-12)


def test_one_primitive_closed_form():
    """Axis-aligned (l2 = 0) primitive, no deformation: magnitude
    delta |psi| exp(-q/2), phase arg psi inside the footprint, lattice sum of
    the magnitude 2 pi l1 l3 delta |psi| (q_cut 60: truncation e^-30)."""
    H, W = 64, 96
    r, ph, a = 0.8, -1.1, 0.4
    u = math.atanh(2 * 47.0 / W - 1)
    v = math.atanh(2 * 31.0 / H - 1)
    sc = one(u, v, 2.0, 0.0, 3.0, a, [r * math.cos(ph), r * math.sin(ph)])
    mag, phase, _, _, _, _ = paper.forward(sc, None, np.zeros((1, 3)), H, W, 60.0)
    delta = 1 / (1 + math.exp(-a))
    x0, y0 = paper.centres(np.array([u]), np.array([v]), H, W)
    yy, xx = np.mgrid[0:H, 0:W]
    qq = ((xx - x0[0]) / 2.0) ** 2 + ((yy - y0[0]) / 3.0) ** 2
    inside = qq <= 60.0
    assert np.allclose(mag[0][inside], delta * r * np.exp(-qq[inside] / 2), rtol=1e-12, atol=0)
    assert np.allclose(phase[0][inside], ph, rtol=0, atol=1e-12)
    assert mag.sum() == pytest.approx(2 * math.pi * 2.0 * 3.0 * delta * r, rel=1e-9)


def _zero_mlp(m):
    return synth.MLP([np.zeros_like(w) for w in m.W], [np.zeros_like(b) for b in m.b], m.L_mean,
                     m.L_tx)


def test_skip_wiring():
    """Only the encoding entering hidden layer 7 (0-based 6) is non-zero: its
    weight on input 156 + dm (the first TX feature, the normalised x) feeds a
    chain to dpsi_re, so dpsi_re = the normalised TX x for every Gaussian."""
    m = _zero_mlp(synth.make_paper_mlp(seed=0))
    dm = 2 * (2 * m.L_mean + 1)
    assert m.W[6].shape == (156, 156 + 81)
    m.W[6][0, 156 + dm] = 1.0
    m.W[7][0, 0] = 1.0
    m.W[8][2, 0] = 1.0
    sc = synth.make_paper_scene(7, 20, 40, seed=1)
    tx = synth.make_tx(3, seed=2)
    res = paper.residuals(sc, m, tx, 20, 40)
    want = (tx[:, 0].astype(np.float64) - m.room_min[0]) / m.room_size[0]
    assert np.allclose(res[..., 2], want[:, None], rtol=0, atol=1e-15)
    assert np.all(res[..., [0, 1, 3, 4]] == 0)


def test_residuals_move_and_scale():
    """An output bias dmu_x = 3 shifts the map by 3 columns exactly (away from
    the edges); ddelta = 0.25 scales the magnitude by (delta + 0.25) / delta."""
    H, W = 40, 80
    sc = synth.make_paper_scene(20, H, W, seed=3)
    x0, _ = paper.centres(sc.mu[:, 0], sc.mu[:, 1], H, W)
    keep = (x0 > 15) & (x0 < W - 20)
    sc = synth.PaperScene(sc.mu[keep], sc.chol[keep], sc.attn_logit[keep], sc.psi[keep])
    m = _zero_mlp(synth.make_paper_mlp(seed=3))
    base, _, _, _, _, _ = paper.forward(sc, m, np.zeros((1, 3)), H, W, 9.0)
    m.b[8][0] = 3.0
    moved, _, _, _, _, _ = paper.forward(sc, m, np.zeros((1, 3)), H, W, 9.0)
    assert np.allclose(moved[0][:, 3:], base[0][:, :-3], rtol=0, atol=1e-12)
    one_sc = synth.PaperScene(sc.mu[:1], sc.chol[:1], sc.attn_logit[:1], sc.psi[:1])
    m.b[8][0] = 0.0
    b1, _, _, _, _, _ = paper.forward(one_sc, m, np.zeros((1, 3)), H, W, 9.0)
    m.b[8][4] = 0.25
    b2, _, _, _, _, _ = paper.forward(one_sc, m, np.zeros((1, 3)), H, W, 9.0)
    d = 1 / (1 + math.exp(-float(one_sc.attn_logit[0])))
    assert np.allclose(b2, b1 * (d + 0.25) / d, rtol=1e-12, atol=0)
