"""Pins for the FP64 oracle (CPU only).

The oracle is only trusted after it is tied to something other than itself:
closed forms (exact trigonometric values, Gaussian lattice sums), invariants of
the order-free sum (Eq. 9/13), an independent dense numpy brute force, a
brute-force tile test, and central finite differences for the gradients.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SAFE = {"sqrt": math.sqrt, "sin": math.sin, "cos": math.cos, "pi": math.pi,
        "inf": math.inf, "nan": math.nan}


def _expr(s):
    return float(eval(s.strip(), {"__builtins__": {}}, SAFE))


def _fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([p.strip() for p in line.split("|")])
    return rows


# ------------------------------------------------------------------ PE ----
def test_pe_closed_form():
    """Eq. 15 against exact trig values, including the feature order."""
    rows = _fixture("pe_closed_form.txt")
    assert len(rows) >= 6
    for xs, L, exp in rows:
        x = np.array([_expr(v) for v in xs.split(",")])
        want = np.array([_expr(v) for v in exp.split(",")])
        got = oracle.pe(x, int(L))
        assert got.shape == (x.size * (2 * int(L) + 1),)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_pe_dimension_of_the_mlp_input():
    # d(2L+1): 2 mean components with L=6 plus 3 TX components with L=10.
    assert oracle.pe(np.zeros(2), 6).size + oracle.pe(np.zeros(3), 10).size == 89
    assert synth.mlp_dims()[0] == 89


# ----------------------------------------------------------------- MLP ----
def _selector_mlp(feature, out_j, scale=1.0, L_mean=6, L_tx=10):
    """An MLP whose output j is scale * ReLU(feature value): hidden unit 0
    carries the selected feature through every layer."""
    m = synth.zero_mlp(L_mean, L_tx)
    m.W[0][0, feature] = 1.0
    for l in range(1, len(m.W) - 1):
        m.W[l][0, 0] = 1.0
    m.W[-1][out_j, 0] = scale
    return m


def test_mlp_routes_each_feature_to_the_output():
    """Closed form: out_j = scale*ReLU(gamma_f), for mean features and TX
    features; catches a wrong concatenation order, a transposed weight or a
    dropped layer."""
    H, W = 90, 360
    sc = synth.make_scene(3, H, W, seed=1)
    tx = np.array([[1.3, 4.1, 0.7], [3.9, 0.2, 2.6]], np.float32)
    mu = sc.mean.astype(np.float64) / np.array([W, H])
    s = (tx.astype(np.float64) - np.array(synth.ROOM_MIN)) / np.array(synth.ROOM_SIZE)
    for f in [0, 1, 2, 5, 13, 25, 26, 27, 28, 29, 40, 58, 59, 88]:
        m = _selector_mlp(f, out_j=f % 5, scale=2.0)
        r = oracle.deform(sc, m, tx, H, W)
        for q in range(2):
            for n in range(3):
                feat = np.concatenate([oracle.pe(mu[n], 6), oracle.pe(s[q], 10)])
                want = np.zeros(5)
                want[f % 5] = 2.0 * max(feat[f], 0.0)
                np.testing.assert_allclose(r[q, n], want, atol=1e-14)
    # the feature value itself, from the closed form for index 29 = sin(2 pi s_x)
    # within gamma(tx): 26 + 3 + 0 -> sin(2^0 pi s_x) is index 29
    m = _selector_mlp(29, out_j=0)
    r = oracle.deform(sc, m, tx, H, W)
    np.testing.assert_allclose(r[:, 0, 0], np.maximum(np.sin(np.pi * s[:, 0]), 0), atol=1e-14)


def test_mlp_biases_and_relu():
    m = synth.zero_mlp()
    m.b[-1][:] = [0.5, -1.0, 0.25, 0.0, 2.0]
    sc = synth.make_scene(4, 90, 360, seed=2)
    r = oracle.deform(sc, m, synth.make_tx(2), 90, 360)
    np.testing.assert_array_equal(r, np.broadcast_to(m.b[-1], r.shape))
    m2 = synth.zero_mlp()
    m2.b[0][3] = -1.0  # negative pre-activation is cut by ReLU
    m2.W[1][0, 3] = 1.0
    m2.W[-1][0, 0] = 1.0
    m2.b[1][0] = 0.75   # positive bias passes
    r2 = oracle.deform(sc, m2, synth.make_tx(2), 90, 360)
    # unit 0 of layer 2 = ReLU(0.75 + 1*ReLU(-1)) = 0.75 -> layers 3,4 have no path -> 0
    np.testing.assert_array_equal(r2, 0.0)
    m2.W[2][0, 0] = 1.0
    m2.W[3][0, 0] = 1.0
    r3 = oracle.deform(sc, m2, synth.make_tx(2), 90, 360)
    np.testing.assert_allclose(r3[..., 0], 0.75, atol=1e-15)


def test_mlp_matches_dense_numpy():
    H, W = 16, 32
    sc = synth.make_scene(40, H, W, seed=3)
    m = synth.make_mlp(gain=2.0, bias_std=0.1, seed=3)
    tx = synth.make_tx(3, seed=3)
    np.testing.assert_allclose(oracle.deform(sc, m, tx, H, W), brute.deform(sc, m, tx, H, W),
                               rtol=1e-12, atol=1e-13)


def test_zero_mlp_leaves_gaussians_unchanged():
    H, W = 90, 360
    sc = synth.make_scene(200, H, W, seed=4)
    tx = synth.make_tx(3, seed=4)
    r = oracle.deform(sc, synth.zero_mlp(), tx, H, W)
    assert np.all(r == 0.0)
    A1, _, _, _ = oracle.forward(sc, synth.zero_mlp(), tx, H, W, 9.0)
    A0, _, _, _ = oracle.forward(sc, None, tx[:1], H, W, 9.0)
    for q in range(3):
        assert np.array_equal(A1[q], A0[0])


# ------------------------------------------------------------- project ----
def test_projection_conic_invariants():
    """The inverse covariance has eigenvalues exp(-2 ls_i) with eigenvector
    (cos th, sin th) for the first (Sec. 3.2 Sigma = L L^T is positive
    definite; here Sigma = R diag(sigma^2) R^T); the footprint half-widths are
    sqrt(q_cut * Sigma_xx), sqrt(q_cut * Sigma_yy)."""
    sc = synth.make_scene(300, 90, 360, ls_std=0.6, seed=5)
    p = oracle.project(sc, None, 9.0)[0]
    A, B, Cc = p[:, 2], p[:, 3], p[:, 4]
    ls = sc.log_scale.astype(np.float64)
    th = sc.rot.astype(np.float64)
    i1, i2 = np.exp(-2 * ls[:, 0]), np.exp(-2 * ls[:, 1])
    np.testing.assert_allclose(A + Cc, i1 + i2, rtol=1e-13)
    np.testing.assert_allclose(A * Cc - B * B, i1 * i2, rtol=1e-11)
    v = np.stack([np.cos(th), np.sin(th)], 1)
    Mv = np.stack([A * v[:, 0] + B * v[:, 1], B * v[:, 0] + Cc * v[:, 1]], 1)
    np.testing.assert_allclose(Mv, i1[:, None] * v, rtol=1e-11, atol=1e-14)
    det = A * Cc - B * B
    np.testing.assert_allclose(p[:, 6] ** 2, 9.0 * Cc / det, rtol=1e-11)
    np.testing.assert_allclose(p[:, 7] ** 2, 9.0 * A / det, rtol=1e-11)
    sg = 1 / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    np.testing.assert_allclose(p[:, 5], sc.amp * sg, rtol=1e-14)


def test_projection_applies_residuals():
    sc = synth.make_scene(50, 90, 360, seed=6)
    g = synth.rng(6)
    resid = g.normal(0, 0.3, size=(2, 50, 5))
    p = oracle.project(sc, resid, 9.0)
    np.testing.assert_allclose(p[..., 0:2], sc.mean[None] + resid[..., 0:2], rtol=1e-15)
    shifted = synth.Scene(sc.mean, sc.log_scale + resid[1, :, 3:5], sc.rot + resid[1, :, 2],
                          sc.opacity_logit, sc.amp)
    p2 = oracle.project(shifted, None, 9.0)[0]
    np.testing.assert_allclose(p[1, :, 2:5], p2[:, 2:5], rtol=1e-6)


# -------------------------------------------------------------- render ----
def _one(mx, my, ls1, ls2=None, rot=0.0, o=50.0, amp=1.0):
    ls2 = ls1 if ls2 is None else ls2
    return synth.Scene(np.array([[mx, my]], np.float64), np.array([[ls1, ls2]], np.float64),
                       np.array([rot], np.float64), np.array([o], np.float64),
                       np.array([amp], np.float64))


def test_single_gaussian_peak_is_its_weight():
    sc = _one(20.0, 11.0, math.log(3.0), o=0.3, amp=0.8)
    A, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), 24, 40, 9.0)
    w = 0.8 / (1 + math.exp(-0.3))
    assert A[0, 11, 20] == pytest.approx(w, rel=0, abs=1e-15)
    assert A.max() == A[0, 11, 20]


@pytest.mark.parametrize("sigma", [1.5, 3.0, 4.0])
def test_isotropic_integral_closed_form(sigma):
    """Lattice sum of an untruncated Gaussian = 2 pi sigma^2 w (Poisson
    summation error ~exp(-2 pi^2 sigma^2), negligible here); with the 3-sigma
    cutoff the integral is 2 pi sigma^2 w (1 - exp(-q_cut/2))."""
    sc = _one(40.3, 39.6, math.log(sigma), amp=1.0)
    A, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), 80, 80, math.inf)
    assert A.sum() == pytest.approx(2 * math.pi * sigma ** 2, rel=1e-9)
    A9, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), 80, 80, 9.0)
    assert A9.sum() == pytest.approx(2 * math.pi * sigma ** 2 * (1 - math.exp(-4.5)), rel=6e-3)
    assert 1 - math.exp(-4.5) == pytest.approx(0.98889, abs=1e-5)


def test_anisotropic_rotated_integral():
    sc = _one(40.0, 40.0, math.log(2.0), math.log(5.0), rot=0.7, amp=0.5)
    A, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), 80, 80, math.inf)
    assert A.sum() == pytest.approx(2 * math.pi * 2.0 * 5.0 * 0.5, rel=1e-9)


def test_render_matches_dense_brute_force():
    """64 Gaussians on a 32x16 grid, every pixel against every Gaussian."""
    H, W = 16, 32
    sc = synth.make_scene(64, H, W, seed=7)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=7)
    tx = synth.make_tx(3, seed=7)
    for q_cut in (9.0, 4.0, math.inf):
        A, _, _, resid = oracle.forward(sc, m, tx, H, W, q_cut)
        Bd = brute.render(sc, brute.deform(sc, m, tx, H, W), H, W, q_cut)
        np.testing.assert_allclose(A, Bd, rtol=0, atol=1e-12 * max(1.0, Bd.max()))


def test_order_free_invariants():
    """Eq. 9 is a plain sum: permutation-invariant, additive over disjoint
    sets, linear in amplitude, and shift-equivariant for integer shifts."""
    H, W = 40, 80
    sc = synth.make_scene(120, H, W, seed=8)
    A, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), H, W, 9.0)
    perm = synth.rng(8).permutation(120)
    sp = synth.Scene(*(a[perm] for a in sc.arrays()))
    Ap, _, _, _ = oracle.forward(sp, None, np.zeros((1, 3)), H, W, 9.0)
    np.testing.assert_allclose(Ap, A, rtol=1e-13, atol=1e-14)
    s1 = synth.Scene(*(a[:50] for a in sc.arrays()))
    s2 = synth.Scene(*(a[50:] for a in sc.arrays()))
    A1, _, _, _ = oracle.forward(s1, None, np.zeros((1, 3)), H, W, 9.0)
    A2, _, _, _ = oracle.forward(s2, None, np.zeros((1, 3)), H, W, 9.0)
    np.testing.assert_allclose(A1 + A2, A, rtol=1e-13, atol=1e-14)
    sk = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, sc.amp.astype(np.float64) * 3.0)
    Ak, _, _, _ = oracle.forward(sk, None, np.zeros((1, 3)), H, W, 9.0)
    np.testing.assert_allclose(Ak, 3.0 * A, rtol=1e-13, atol=1e-14)
    # integer shift of an interior Gaussian shifts its image
    one = _one(30.4, 17.2, math.log(2.5), math.log(1.5), rot=0.4)
    sh = _one(30.4 + 7.0, 17.2 - 5.0, math.log(2.5), math.log(1.5), rot=0.4)
    Ao, _, _, _ = oracle.forward(one, None, np.zeros((1, 3)), H, W, 9.0)
    As, _, _, _ = oracle.forward(sh, None, np.zeros((1, 3)), H, W, 9.0)
    # As[y, x] = Ao[y + 5, x - 7]
    np.testing.assert_allclose(As[0, :-5, 7:], Ao[0, 5:, :-7], rtol=1e-12, atol=1e-15)
    assert As.sum() == pytest.approx(Ao.sum(), rel=1e-12)


def test_slack_covers_only_the_cutoff_band():
    H, W = 30, 60
    sc = synth.make_scene(80, H, W, seed=9)
    A, S, proj, _ = oracle.forward(sc, None, np.zeros((1, 3)), H, W, 9.0, band=1e-2)
    assert np.all(S >= 0)
    # tiny band -> nearly no slack; the band sum is bounded by w*exp(-4.5*(1-band))
    _, S0, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), H, W, 9.0, band=0.0)
    assert S0.sum() <= 1e-12 + S.sum()
    assert S.max() <= proj[0, :, 5].sum() * math.exp(-4.5 * (1 - 1e-2))


# ----------------------------------------------------------------- bin ----
def _parse_f(v):
    return np.float32(_expr(v))


def test_bin_hand_worked_edges():
    rows = _fixture("bin_edges.txt")
    for geo, recs, exp in rows:
        H, W, tw, th = (int(v) for v in geo.split())
        mx, my, rx, ry = (_parse_f(v) for v in recs.split())
        rec = np.zeros((1, 1, 8), np.float32)
        rec[0, 0, 0], rec[0, 0, 1], rec[0, 0, 6], rec[0, 0, 7] = mx, my, rx, ry
        counts, gids, offs, nk = oracle.bin_f32(rec, H, W, tw, th)
        ntx, nty = oracle.tiles(H, W, tw, th)
        got = [t for t in range(ntx * nty) if offs[t + 1] > offs[t]]
        want = [] if exp == "none" else [int(v) for v in exp.split()]
        assert got == want, (geo, recs, got, want)
        assert int(counts[0, 0]) == len(want) == nk


@pytest.mark.parametrize("geo", [(90, 360, 16, 16), (36, 40, 16, 16), (90, 360, 8, 8),
                                 (16, 32, 32, 16), (17, 45, 8, 4)])
def test_bin_matches_brute_force(geo):
    H, W, tw, th = geo
    rec = synth.random_rects_records(3, 150, H, W, r_max=W / 6, seed=sum(geo))
    counts, gids, offs, nk = oracle.bin_f32(rec, H, W, tw, th)
    lists = brute.bin_brute(rec, H, W, tw, th)
    ntx, nty = oracle.tiles(H, W, tw, th)
    T = ntx * nty
    total = 0
    for q in range(3):
        for t in range(T):
            seg = gids[offs[q * T + t]: offs[q * T + t + 1]]
            want = lists.get((q, t), np.zeros(0, np.uint32))
            assert np.array_equal(seg, want), (q, t)
            total += want.size
    assert total == nk == offs[-1]
    per = np.zeros((3, 150), np.int64)
    for (q, t), ids in lists.items():
        per[q, ids] += 1
    assert np.array_equal(per, counts)


def test_bin_capacity_overflow_reports_required():
    rec = synth.random_rects_records(2, 100, 90, 360, r_max=40, seed=11)
    _, _, _, need = oracle.bin_f32(rec, 90, 360, 16, 16)
    counts, gids, offs, nk = oracle.bin_f32(rec, 90, 360, 16, 16, cap=need - 1)
    assert gids is None and nk == need
    _, g2, _, nk2 = oracle.bin_f32(rec, 90, 360, 16, 16, cap=need)
    assert g2 is not None and nk2 == need


def test_bin_empty_scene():
    rec = np.zeros((2, 0, 8), np.float32)
    counts, gids, offs, nk = oracle.bin_f32(rec, 90, 360, 16, 16)
    assert nk == 0 and np.all(offs == 0) and offs.size == 2 * 23 * 6 + 1


# ------------------------------------------------------------ gradients ---
def _loss(sc, m, tx, H, W, c):
    A, _, _, _ = oracle.forward(sc, m, tx, H, W, math.inf)
    return float((A * c).sum())


def test_gradients_match_finite_differences():
    """64 Gaussians on 32x16, no cutoff (the cutoff makes A discontinuous),
    L = sum(c * A) with random c; central differences, h = 1e-6."""
    H, W = 16, 32
    sc = synth.make_scene(64, H, W, seed=12)
    sc = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()))
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=12)
    m.W = [w.astype(np.float64) for w in m.W]
    m.b = [b.astype(np.float64) for b in m.b]
    tx = synth.make_tx(2, seed=12).astype(np.float64)
    c = synth.rng(12).normal(size=(2, H, W))
    g = oracle.grad(sc, m, tx, H, W, math.inf, c)
    h = 1e-6
    rs = synth.rng(13)

    def check(arr, idx, analytic):
        old = arr[idx]
        arr[idx] = old + h
        lp = _loss(sc, m, tx, H, W, c)
        arr[idx] = old - h
        lm = _loss(sc, m, tx, H, W, c)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        assert analytic == pytest.approx(fd, rel=2e-5, abs=2e-7), (idx, analytic, fd)

    for n in rs.choice(64, 10, replace=False):
        for i in range(2):
            check(sc.mean, (n, i), g["d_mean"][n, i])
            check(sc.log_scale, (n, i), g["d_log_scale"][n, i])
        check(sc.rot, (n,), g["d_rot"][n])
        check(sc.opacity_logit, (n,), g["d_opacity"][n])
        check(sc.amp, (n,), g["d_amp"][n])
    for l in range(len(m.W)):
        for _ in range(6):
            j = rs.integers(0, m.W[l].shape[0]); k = rs.integers(0, m.W[l].shape[1])
            check(m.W[l], (j, k), g["d_W"][l][j, k])
        j = rs.integers(0, m.b[l].shape[0])
        check(m.b[l], (j,), g["d_b"][l][j])


def test_stop_grad_mean_drops_only_the_encoding_path():
    H, W = 16, 32
    sc = synth.make_scene(20, H, W, seed=14)
    m = synth.make_mlp(gain=1.0, seed=14)
    tx = synth.make_tx(2, seed=14)
    c = synth.rng(14).normal(size=(2, H, W))
    g = oracle.grad(sc, m, tx, H, W, math.inf, c)
    gs = oracle.grad(sc, m, tx, H, W, math.inf, c, stop_grad_mean=True)
    np.testing.assert_allclose(gs["d_mean"], g["d_mean_direct"], rtol=1e-14)
    assert not np.allclose(g["d_mean"], g["d_mean_direct"])
    for a, b in zip(g["d_W"], gs["d_W"]):
        np.testing.assert_array_equal(a, b)


def _numpy_mlp_backward(m, x, g_out, masks):
    """Independent dense numpy back-propagation of one row with the ReLU
    decisions given explicitly (masks[l]: the on/off pattern of the units of
    hidden layer l); an 'off' unit contributes activation 0."""
    L = len(m.W)
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    for l in range(L - 1):
        z = m.W[l].astype(np.float64) @ h + m.b[l]
        h = np.where(masks[l], z, 0.0)
        acts.append(h)
    d = np.asarray(g_out, np.float64)
    dW, db = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = np.outer(d, acts[l])
        db[l] = d.copy()
        if l > 0:
            d = (m.W[l].astype(np.float64).T @ d) * masks[l - 1]
    return dW, db


def test_relu_slack_is_zero_without_ambiguous_decisions():
    """Biases of +10 put every hidden pre-activation far above zero: no ReLU
    decision is ambiguous and the slack is exactly zero."""
    H, W = 16, 32
    sc = synth.make_scene(30, H, W, seed=21)
    m = synth.make_mlp(gain=0.3, seed=21)
    m.b = [np.full_like(b, 10.0) for b in m.b]
    tx = synth.make_tx(2, seed=21)
    dr = synth.rng(21).normal(size=(2, 30, 5))
    _, _, _, sl = oracle.mlp_grad(sc, m, tx, H, W, dr)
    assert all(float(np.abs(a).max()) == 0.0 for a in sl["d_W"] + sl["d_b"])
    assert float(np.abs(sl["d_mean"]).max()) == 0.0


def test_relu_slack_equals_the_flipped_decision():
    """One row whose hidden unit j of the second layer is put exactly at zero
    pre-activation (by its bias): the slack of every parameter equals the
    absolute difference between the dense numpy back-propagations with that
    unit on and off, and the gradient itself is one of the two."""
    H, W = 16, 32
    sc = synth.make_scene(1, H, W, seed=22)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, n_hidden=3, seed=22)
    m.W = [w.astype(np.float64) for w in m.W]
    m.b = [b.astype(np.float64) for b in m.b]
    tx = synth.make_tx(1, seed=22)
    mu = sc.mean[0].astype(np.float64) / np.array([W, H])
    s = (tx[0] - np.array(m.room_min)) / np.array(m.room_size)
    x = np.concatenate([oracle.pe(mu, m.L_mean), oracle.pe(s, m.L_tx)])
    h0 = np.maximum(m.W[0] @ x + m.b[0], 0.0)
    z1 = m.W[1] @ h0 + m.b[1]
    j = int(np.argmax(np.abs(z1)))
    m.b[1][j] = 0.0
    m.b[1][j] = -float(m.W[1][j] @ h0)      # z1[j] = 0 up to rounding
    masks = []
    h = x
    for l in range(len(m.W) - 1):
        z = m.W[l] @ h + m.b[l]
        masks.append(z > 0.0)
        h = np.maximum(z, 0.0)
    dr = synth.rng(22).normal(size=(1, 1, 5))
    dW, db, _, sl = oracle.mlp_grad(sc, m, tx, H, W, dr, stop_grad_mean=True)
    on = [mk.copy() for mk in masks]
    off = [mk.copy() for mk in masks]
    on[1][j], off[1][j] = True, False
    dW_on, db_on = _numpy_mlp_backward(m, x, dr[0, 0], on)
    dW_off, db_off = _numpy_mlp_backward(m, x, dr[0, 0], off)
    close = lambda a, b: all(np.allclose(x, y, rtol=1e-9, atol=1e-12) for x, y in zip(a, b))
    assert close(dW, dW_on) or close(dW, dW_off)  # either decision at z = 0
    for l in range(len(m.W)):
        np.testing.assert_allclose(sl["d_W"][l], np.abs(dW_on[l] - dW_off[l]), rtol=1e-9,
                                   atol=1e-12)
        np.testing.assert_allclose(sl["d_b"][l], np.abs(db_on[l] - db_off[l]), rtol=1e-9,
                                   atol=1e-12)
    assert float(np.abs(sl["d_W"][0]).max()) > 0.0  # the flip reaches the first layer


# ---------------------------------------------------------------- rssi ----
@pytest.mark.parametrize("sigma", [1.5, 2.5])
def test_rssi_closed_form(sigma):
    """RSSI head (Sec. 7.2): the pooled map of one untruncated isotropic
    Gaussian far from the edges is its lattice sum 2 pi sigma^2 w over the
    H W pixels; with the zero MLP the residuals are exactly 0."""
    sc = _one(32.0, 31.0, math.log(sigma), o=0.4, amp=0.7)
    w = 0.7 / (1 + math.exp(-0.4))
    mlp = synth.zero_mlp()
    r, slack = oracle.rssi(sc, mlp, synth.make_tx(2, seed=3), 64, 64, math.inf)
    want = 2 * math.pi * sigma ** 2 * w / (64 * 64)
    assert r.shape == (2,) and slack.shape == (2,)
    assert r == pytest.approx([want, want], rel=1e-9)


def test_rssi_is_the_mean_magnitude():
    """Pooling is linear in the amplitudes, adds over disjoint scenes with
    non-negative maps, and takes the magnitude (Sec. 6.6): negating every
    amplitude leaves the RSSI unchanged while the map changes sign."""
    sc = synth.make_scene(40, 16, 16, seed=5)
    mlp = synth.make_mlp(seed=2, bias_std=0.05)
    tx = synth.make_tx(3, seed=4)
    r, _ = oracle.rssi(sc, mlp, tx, 16, 16, 9.0)
    A, _, _, _ = oracle.forward(sc, mlp, tx, 16, 16, 9.0)
    assert np.all(r > 0)
    k = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, sc.amp.astype(np.float64) * 2.5)
    rk, _ = oracle.rssi(k, mlp, tx, 16, 16, 9.0)
    assert rk == pytest.approx(2.5 * r, rel=1e-12)
    neg = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, -sc.amp.astype(np.float64))
    An, _, _, _ = oracle.forward(neg, mlp, tx, 16, 16, 9.0)
    rn, _ = oracle.rssi(neg, mlp, tx, 16, 16, 9.0)
    assert np.allclose(An, -A, rtol=0, atol=1e-15) and rn == pytest.approx(r, rel=1e-12)
    s1 = synth.Scene(*(a[:20] for a in sc.arrays()))
    s2 = synth.Scene(*(a[20:] for a in sc.arrays()))
    r1, _ = oracle.rssi(s1, mlp, tx, 16, 16, 9.0)
    r2, _ = oracle.rssi(s2, mlp, tx, 16, 16, 9.0)
    assert r1 + r2 == pytest.approx(r, rel=1e-12)


# --------------------------------------------------- azimuth wrap, 2 channels ----
def test_wrap_is_cyclic():
    """With wrap the map is periodic in azimuth: moving every Gaussian by k
    columns rolls the map by k columns (exactly, integer moves)."""
    H, W = 20, 48
    sc = synth.make_scene(60, H, W, seed=11)
    A, _, _, _ = oracle.forward(sc, None, np.zeros((1, 3)), H, W, 9.0, wrap=True)
    for k in (5, 31):
        m = sc.mean.astype(np.float64).copy()
        m[:, 0] = (m[:, 0] + k) % W
        sk = synth.Scene(m, sc.log_scale, sc.rot, sc.opacity_logit, sc.amp)
        Ak, _, _, _ = oracle.forward(sk, None, np.zeros((1, 3)), H, W, 9.0, wrap=True)
        assert np.allclose(Ak, np.roll(A, k, axis=2), rtol=0, atol=1e-12)


def test_wrap_seam_integral_and_interior():
    """A Gaussian on the 0 / W seam keeps its whole lattice sum 2 pi sigma^2 w
    with wrap (q_cut = 60: truncation e^-30) and loses about half without;
    away from the seam wrap changes nothing."""
    sigma = 2.0
    seam = _one(0.4, 30.0, math.log(sigma), amp=1.0)
    Aw, _, _, _ = oracle.forward(seam, None, np.zeros((1, 3)), 60, 72, 60.0, wrap=True)
    An, _, _, _ = oracle.forward(seam, None, np.zeros((1, 3)), 60, 72, 60.0)
    assert Aw.sum() == pytest.approx(2 * math.pi * sigma ** 2, rel=1e-9)
    assert 0.5 < An.sum() / Aw.sum() < 0.8  # centre at column 0.4: a bit over half at x >= 0
    mid = _one(36.2, 30.0, math.log(sigma), amp=0.5)
    Bw, _, _, _ = oracle.forward(mid, None, np.zeros((1, 3)), 60, 72, 9.0, wrap=True)
    Bn, _, _, _ = oracle.forward(mid, None, np.zeros((1, 3)), 60, 72, 9.0)
    assert np.array_equal(Bw, Bn)


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (32, 8)])
def test_bin_wrap_matches_brute_force(tile):
    """Tile lists with wrap: a Gaussian lists tile t when a column of t is
    congruent mod W to a pixel column of ceil(mx-rx)..floor(mx+rx) (FP32) and
    t's rows meet the clamped row range; W = 72 is not a multiple of 32."""
    tw, th = tile
    H, W = 24, 72
    rng = np.random.default_rng(12)
    Nn = 80
    rec = np.zeros((2, Nn, 8), np.float32)
    rec[..., 0] = rng.uniform(-5, W + 5, (2, Nn))
    rec[..., 1] = rng.uniform(-3, H + 3, (2, Nn))
    rec[..., 6] = rng.uniform(0.2, 12, (2, Nn))
    rec[..., 7] = rng.uniform(0.2, 6, (2, Nn))
    rec[0, 0, 6] = 40.0  # spans more than W - 1 columns: every column tile
    counts, gids, offs, nk = oracle.bin_f32(rec, H, W, tw, th, wrap=True)
    ntx, nty = oracle.tiles(H, W, tw, th)
    want = [[[] for _ in range(ntx * nty)] for _ in range(2)]
    for q in range(2):
        for n in range(Nn):
            mx, my, rx, ry = (np.float32(v) for v in rec[q, n, [0, 1, 6, 7]])
            lo, hi = np.ceil(np.float32(mx - rx)), np.floor(np.float32(mx + rx))
            ylo = np.ceil(max(np.float32(my - ry), np.float32(0)))
            yhi = np.floor(min(np.float32(my + ry), np.float32(H - 1)))
            if lo > hi or ylo > yhi:
                continue
            cols = set(int(c) % W for c in np.arange(lo, hi + 1)) if hi - lo + 1 < W else set(range(W))
            ct = sorted(set(c // tw for c in cols))
            for ty in range(int(ylo) // th, int(yhi) // th + 1):
                for tx in ct:
                    want[q][ty * ntx + tx].append(n)
    for q in range(2):
        for t in range(ntx * nty):
            got = list(gids[offs[q * ntx * nty + t]:offs[q * ntx * nty + t + 1]])
            assert got == want[q][t], (q, t)
    assert nk == sum(len(l) for w in want for l in w)


def test_two_channels_magnitude_and_phase():
    """One Gaussian of complex amplitude r e^{i phi}: magnitude
    r sigmoid(o) exp(-q/2), phase phi inside the footprint; opposite
    amplitudes at the same place cancel; a zero imaginary part gives the
    one-channel map's magnitude."""
    r, phi, o = 0.9, 2.3, 0.5
    sc = synth.Scene(np.array([[20.0, 11.0]]), np.array([[math.log(2.5)] * 2]), np.array([0.0]),
                     np.array([o]), np.array([[r * math.cos(phi), r * math.sin(phi)]]))
    re, im, mag, ph, _ = oracle.forward_complex(sc, None, np.zeros((1, 3)), 24, 40, 9.0)
    w = r / (1 + math.exp(-o))
    y, x = np.mgrid[0:24, 0:40]
    qq = ((x - 20.0) ** 2 + (y - 11.0) ** 2) / 2.5 ** 2
    inside = qq <= 9.0
    assert np.allclose(mag[0][inside], w * np.exp(-qq[inside] / 2), rtol=1e-12, atol=0)
    assert np.all(mag[0][~inside] == 0)
    assert np.allclose(ph[0][inside], phi, rtol=0, atol=1e-12)
    two = synth.Scene(np.array([[20.0, 11.0], [20.0, 11.0]]), np.array([[1.0, 1.0], [1.0, 1.0]]),
                      np.zeros(2), np.zeros(2), np.array([[0.3, -0.2], [-0.3, 0.2]]))
    _, _, mag2, _, _ = oracle.forward_complex(two, None, np.zeros((1, 3)), 24, 40, 9.0)
    assert np.all(np.abs(mag2) <= 1e-15)
    sc3 = synth.make_scene(30, 24, 40, seed=13)
    amp2 = np.stack([sc3.amp.astype(np.float64), np.zeros(30)], 1)
    c3 = synth.Scene(sc3.mean, sc3.log_scale, sc3.rot, sc3.opacity_logit, amp2)
    A, _, _, _ = oracle.forward(sc3, None, np.zeros((1, 3)), 24, 40, 9.0)
    _, _, mag3, _, _ = oracle.forward_complex(c3, None, np.zeros((1, 3)), 24, 40, 9.0)
    assert np.array_equal(mag3, np.abs(A))
