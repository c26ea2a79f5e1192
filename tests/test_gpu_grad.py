"""GPU gradients (render backward, project backward, MLP backward and the
autograd.Function over all of them) against the FP64 oracle's analytic
gradient, which the CPU suite pins to central finite differences.

Tolerance, element by element within each parameter group (a field of the
record or residual gradients, a weight matrix, a bias vector):
|g_gpu - g_oracle| <= 1e-3 |g_oracle| + 1e-3 max|g_oracle| (relative 1e-3,
with a floor of 1e-3 of the group's largest component where a component is
~0).  Every comparison prints its worst element.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import check_grads, grad_error

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def api():
    from paper_2506_12787_b300 import api, build
    build.build()
    assert torch.cuda.is_available()
    return api


def dev():
    return torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def params_of(m):
    out = []
    for W, b in zip(m.W, m.b):
        out += [T(W).requires_grad_(), T(b).requires_grad_()]
    return out


def run_autograd(api, sc, m, tx, H, W, q_cut, dA, stop_grad_mean=False, tile=(16, 16)):
    from paper_2506_12787_b300.autograd import SpectrumConfig, render_spectra
    cfg = SpectrumConfig(api.make_grid(H, W, tile[0], tile[1], q_cut),
                         stop_grad_mean=stop_grad_mean)
    leaves = [T(a).requires_grad_() for a in sc.arrays()]
    ps = params_of(m)
    out = render_spectra(cfg, T(tx), *leaves, ps)
    out.backward(T(dA))
    names = ["d_mean", "d_log_scale", "d_rot", "d_opacity", "d_amp"]
    g = {k: v.grad.cpu().numpy() for k, v in zip(names, leaves)}
    g["d_W"] = [p.grad.cpu().numpy() for p in ps[0::2]]
    g["d_b"] = [p.grad.cpu().numpy() for p in ps[1::2]]
    return out.detach().cpu().numpy(), g


def groups_of(g, ref):
    """(name, gpu, oracle) for every parameter group: each field of d_mean /
    d_log_scale, d_rot, d_opacity, d_amp, and every weight and bias."""
    out = []
    sl = ref.get("slack")
    for k in ["d_mean", "d_log_scale"]:
        for c in range(2):
            s_ = sl["d_mean"][:, c] if (sl is not None and k == "d_mean") else None
            out.append((f"{k}[:,{c}]", np.asarray(g[k])[:, c], ref[k][:, c], s_))
    for k in ["d_rot", "d_opacity", "d_amp"]:
        out.append((k, g[k], ref[k]))
    for l, (a, b) in enumerate(zip(g.get("d_W", []), ref.get("d_W", []))):
        out.append((f"d_W[{l}]", a, b, sl["d_W"][l] if sl is not None else None))
    for l, (a, b) in enumerate(zip(g.get("d_b", []), ref.get("d_b", []))):
        out.append((f"d_b[{l}]", a, b, sl["d_b"][l] if sl is not None else None))
    return out


def compare(g, ref, tag):
    return check_grads(groups_of(g, ref), tag)


@pytest.mark.parametrize("q_cut,tile", [(9.0, (16, 16)), (9.0, (8, 8)), (9.0, (32, 16)),
                                        (2.0, (16, 16)), (math.inf, (16, 16))])
def test_render_backward_matches_oracle(api, q_cut, tile):
    """Every record gradient against the oracle: the usual cutoff over three
    tile shapes (box rows split over the lanes of a warp), a tight cutoff
    (many box rows without in-cutoff pixels) and no cutoff (every row of
    every box in full)."""
    H, W = 90, 360
    sc = synth.make_scene(600 if q_cut < math.inf else 200, H, W, ls_std=0.4, seed=40)
    Q = 2
    tx = synth.make_tx(Q, seed=40)
    dA = synth.rng(40).normal(size=(Q, H, W))
    ref = oracle.grad(sc, None, tx, H, W, q_cut, dA)
    grid = api.make_grid(H, W, tile[0], tile[1], q_cut)
    ds = api.DeviceScene.from_host(sc, dev())
    r = api.Renderer(grid, dev())
    r.forward(ds, None, T(tx))
    L = r.last
    d_rec = api.wrf_render_backward(L["rec"], L["gids"], L["offs"], L["n_keys"], r.cap, sc.n, Q,
                                    grid, T(dA)).cpu().numpy()
    names = ["mx", "my", "A", "B", "C", "w"]
    worst = check_grads([(f"d_{nm}", d_rec[..., c], ref["d_proj"][..., c])
                         for c, nm in enumerate(names)],
                        f"render backward q_cut={q_cut} tile={tile[0]}x{tile[1]}")
    assert worst <= 1.0


def test_project_backward_matches_oracle(api):
    H, W = 90, 360
    sc = synth.make_scene(500, H, W, seed=41)
    Q = 3
    resid = synth.rng(41).normal(0, 0.3, size=(Q, sc.n, 5))
    d_proj = synth.rng(42).normal(size=(Q, sc.n, 6))
    # oracle chain rule of the projection only: feed d_proj through or_project_grad
    import ctypes as C
    L = oracle.lib()
    arrs = [oracle._d(a) for a in sc.arrays()]
    dres = np.zeros((Q, sc.n, 5)); dm = np.zeros((sc.n, 2)); dls = np.zeros((sc.n, 2))
    drot = np.zeros(sc.n); dop = np.zeros(sc.n); damp = np.zeros(sc.n)
    r64, pr = oracle._d(resid)
    dp, pdp = oracle._d(d_proj)
    D = oracle.D
    L.or_project_grad(sc.n, arrs[1][1], arrs[2][1], arrs[3][1], arrs[4][1], Q, pr, pdp,
                      dres.ctypes.data_as(D), dm.ctypes.data_as(D), dls.ctypes.data_as(D),
                      drot.ctypes.data_as(D), dop.ctypes.data_as(D), damp.ctypes.data_as(D))
    g = api.wrf_project_backward(api.DeviceScene.from_host(sc, dev()), T(resid), Q, T(d_proj))
    for k, ref in [("d_resid", dres), ("d_mean", dm), ("d_log_scale", dls), ("d_rot", drot),
                   ("d_opacity", dop), ("d_amp", damp)]:
        a = g[k].cpu().numpy()
        if a.ndim >= 2:
            grp = [(f"{k}[...,{c}]", a[..., c], ref[..., c]) for c in range(a.shape[-1])]
        else:
            grp = [(k, a, ref)]
        assert check_grads(grp, "project backward") <= 1.0, k


@pytest.mark.parametrize("case", [
    # (Gaussians, queries, hidden layers): ragged 64-row tiles (700 = 10 x 64 + 60);
    # a model of five 128 x 128 layers (two passes of at most three weight
    # gradients); a model without hidden 128 x 128 layers; and the training
    # workload's 20k Gaussians over 8 queries (2,504 tiles: every CTA flushes
    # its tensor-memory accumulators more than once)
    (700, 3, 4), (700, 3, 6), (300, 2, 1), (20000, 8, 4)])
@pytest.mark.parametrize("stop", [False, True])
def test_deform_backward_matches_oracle(api, stop, case):
    H, W = 90, 360
    n, Q, n_hidden = case
    sc = synth.make_scene(n, H, W, seed=43)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, n_hidden=n_hidden, seed=43)
    tx = synth.make_tx(Q, seed=43)
    d_resid = synth.rng(44).normal(size=(Q, sc.n, 5))
    # FP64 oracle gradient, with the slack of ReLU decisions that an FP32
    # forward may take either way
    dW_ref, db_ref, dmean, sl = oracle.mlp_grad(sc, m, tx, H, W, d_resid, stop_grad_mean=stop)
    ds, dmlp = api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev())
    grid = api.make_grid(H, W)
    dW, db, d_mean = api.wrf_deform_backward(ds, dmlp, grid, T(tx), T(d_resid),
                                             stop_grad_mean=stop)
    # the same with the hidden activations saved by the forward (no recompute)
    resid, acts = api.wrf_deform_acts(ds, dmlp, grid, T(tx))
    assert torch.equal(resid, api.wrf_deform(ds, dmlp, grid, T(tx)))
    dW2, db2, d_mean2 = api.wrf_deform_backward(ds, dmlp, grid, T(tx), T(d_resid),
                                                stop_grad_mean=stop, acts=acts)
    for tag, gw, gb in [("recomputed", dW, db), ("saved activations", dW2, db2)]:
        grp = []
        for l in range(len(m.W)):
            grp += [(f"d_W[{l}]", gw[l].cpu().numpy(), dW_ref[l], sl["d_W"][l]),
                    (f"d_b[{l}]", gb[l].cpu().numpy(), db_ref[l], sl["d_b"][l])]
        assert check_grads(grp, f"deform backward ({tag})") <= 1.0
    if stop:
        assert np.all(d_mean.cpu().numpy() == 0)
    else:
        for tag, dmg in [("recomputed", d_mean), ("saved activations", d_mean2)]:
            dmg = dmg.cpu().numpy()
            grp = [(f"d_mean[:,{c}]", dmg[:, c], dmean[:, c], sl["d_mean"][:, c])
                   for c in range(2)]
            assert check_grads(grp, f"deform backward d_mean through gamma(mean) ({tag})") <= 1.0


@pytest.mark.parametrize("case", ["64x32x16", "800x90x360"])
def test_autograd_matches_oracle(api, case):
    n, H, W = (int(v) for v in case.split("x"))
    sc = synth.make_scene(n, H, W, ls_mean=math.log(2.0 if n == 64 else 3.0), seed=n)
    m = synth.make_mlp(gain=0.5, bias_std=0.02, seed=n)
    Q = 2
    tx = synth.make_tx(Q, seed=n)
    dA = synth.rng(n + 1).normal(size=(Q, H, W))
    out, g = run_autograd(api, sc, m, tx, H, W, 9.0, dA)
    ref = oracle.grad(sc, m, tx, H, W, 9.0, dA)
    assert compare(g, ref, f"autograd {case}") <= 1.0


def test_autograd_stop_grad_mean(api):
    H, W = 16, 32
    sc = synth.make_scene(64, H, W, ls_mean=math.log(2.0), seed=5)
    m = synth.make_mlp(gain=0.5, bias_std=0.02, seed=5)
    tx = synth.make_tx(2, seed=5)
    dA = synth.rng(6).normal(size=(2, H, W))
    _, g = run_autograd(api, sc, m, tx, H, W, 9.0, dA, stop_grad_mean=True)
    ref = oracle.grad(sc, m, tx, H, W, 9.0, dA, stop_grad_mean=True)
    assert compare(g, ref, "autograd stop-grad") <= 1.0


def test_training_step_workload(api):
    """The training-step workload: 20k Gaussians, 64 TX, 360x90; targets
    rendered by the oracle from a copy with means jittered by N(0, 2 px);
    mean L1 loss.  Gradients of 2 of the queries against the oracle, then one
    gradient step on all 64 must lower the loss."""
    from paper_2506_12787_b300.autograd import SpectrumConfig, render_spectra
    H, W, N, Q = 90, 360, 20000, 64
    sc = synth.make_scene(N, H, W, seed=0)
    m = synth.make_mlp(seed=0)
    tx = synth.make_tx(Q, seed=3)
    tgt_scene = synth.jitter_means(sc, 2.0, seed=4)
    A_tgt, _, _, _ = oracle.forward(tgt_scene, m, tx, H, W, 9.0)
    A_tgt_t = T(A_tgt)
    # gradient parity on 2 queries (L1 sign from the GPU forward)
    sub = [0, 37]
    out, _ = run_autograd(api, sc, m, tx[sub], H, W, 9.0, np.zeros((2, H, W)))
    dA = np.sign(out - A_tgt[sub]) / (2 * H * W)
    _, g = run_autograd(api, sc, m, tx[sub], H, W, 9.0, dA)
    ref = oracle.grad(sc, m, tx[sub], H, W, 9.0, dA)
    assert compare(g, ref, "training step (2 queries)") <= 1.0
    # full step: loss decreases after a small step along -grad of the Gaussians
    cfg = SpectrumConfig(api.make_grid(H, W, 16, 16, 9.0))
    leaves = [T(a).requires_grad_() for a in sc.arrays()]
    ps = params_of(m)
    loss0 = (render_spectra(cfg, T(tx), *leaves, ps) - A_tgt_t).abs().mean()
    loss0.backward()
    with torch.no_grad():
        for v in leaves + ps:
            assert torch.all(torch.isfinite(v.grad))
        stepped = [v - 1e-2 * v.grad / (v.grad.abs().max() + 1e-30) for v in leaves]
        loss1 = (render_spectra(cfg, T(tx), *stepped, [p.detach() for p in ps]) - A_tgt_t).abs().mean()
    print(f"training step: L1 {float(loss0):.6f} -> {float(loss1):.6f}")
    assert float(loss1) < float(loss0)


def edge_scene(n, H, W, tile, seed):
    """Gaussians centred on or within a pixel of tile edges (corners
    included), so that every footprint straddles two to four tiles."""
    sc = synth.make_scene(n, H, W, ls_std=0.3, seed=seed)
    r = synth.rng(seed + 7)
    tw, th = tile
    ex = tw * r.integers(1, max(2, W // tw), n) + r.choice([-1.0, -0.5, 0.0, 0.25, 0.5], n)
    ey = th * r.integers(1, max(2, H // th), n) + r.choice([-1.0, -0.5, 0.0, 0.25, 0.5], n)
    m = np.stack([np.clip(ex, 0, W - 1), np.clip(ey, 0, H - 1)], axis=1)
    return synth.Scene(m.astype(np.float32), sc.log_scale, sc.rot, sc.opacity_logit, sc.amp)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_gradients_straddling_tile_edges(api, tile):
    """Every Gaussian straddles tile edges: each tile renders part of its
    footprint and the backward adds the parts together; every gradient
    element against the oracle."""
    H, W = 90, 360
    sc = edge_scene(400, H, W, tile, seed=61)
    m = synth.make_mlp(gain=0.5, bias_std=0.02, seed=61)
    tx = synth.make_tx(2, seed=61)
    dA = synth.rng(62).normal(size=(2, H, W))
    _, g = run_autograd(api, sc, m, tx, H, W, 9.0, dA, tile=tile)
    ref = oracle.grad(sc, m, tx, H, W, 9.0, dA)
    assert compare(g, ref, f"tile edges {tile[0]}x{tile[1]}") <= 1.0
