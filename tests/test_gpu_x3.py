"""GPU parity of the FP32-level tensor-core deformation MLP (precision
WRF_BF16X3: every FP32 weight and activation split into BF16 hi + lo, every
product taken as hi hi + hi lo + lo hi with FP32 accumulation), through the
C ABI.

Two references:
  * a numpy emulation of the same splits (hi = bf16(x), lo = bf16(x - hi) of
    every weight, bias and activation; FP64 sums) pins the tensor-core
    arithmetic itself: the kernel differs from it by the FP32 accumulation
    order only (median <= 2e-6, max <= 3e-5 of max |resid|).  Dropping one of
    the three products or a lo term moves the error to ~1e-3;
  * the FP64 oracle pins the whole path: residuals within the emulation's own
    error plus that margin, spectra within the FP32 tolerance (1e-4 x peak),
    gradients within the gradient tolerance with the ReLU band widened to
    X3_BAND (below).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import check_grads, spectrum_error

pytestmark = pytest.mark.gpu

# ReLU decisions the three-product forward may take either way: a product
# a b = (ah + al + ea)(bh + bl + eb) taken as ah bh + ah bl + al bh misses
# al bl, ea b and a eb, each at most 2^-16 |a b| (BF16 keeps 8 significant
# bits, so |x - hi| <= 2^-8 |x| and |x - hi - lo| <= 2^-16 |x|), so a
# pre-activation may be off by 3 x 2^-16 ~ 4.6e-5 of its terms' magnitude,
# plus FP32 accumulation (< 1e-5) and what the previous layer carried in;
# the band is twice the single-layer bound.
X3_BAND = 1e-4


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


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split(x):
    """(hi, lo) = (bf16(x), bf16(x - hi)) of float32 values, as float64
    (x - hi is exact in FP32)."""
    x = np.asarray(x, np.float32)
    hi = bf16(x)
    return hi, bf16((x.astype(np.float64) - hi).astype(np.float32))


def x3_layer(h, Wl, bl):
    hh, hl = split(h)
    wh, wl = split(Wl)
    b_hi, b_lo = split(bl)
    return hh @ wh.T + hh @ wl.T + hl @ wh.T + (b_hi + b_lo)


def emulate_x3_mlp(sc, m, tx, H, W):
    """Residuals [Q,N,5] and hidden activations [n_layers-1][Q*N][128] with
    the kernel's splitting points.  Layer 1 is FP32 (U[n] + V[q], Eq. 14-15);
    every later layer takes its input and weights as hi + lo pairs."""
    N, Q = sc.n, tx.shape[0]
    gm = np.stack([oracle.pe(np.array([x / W, y / H]), m.L_mean) for x, y in sc.mean])
    s = (np.asarray(tx, np.float64) - np.asarray(m.room_min)) / np.asarray(m.room_size)
    gt = np.stack([oracle.pe(v, m.L_tx) for v in s])
    W0 = np.asarray(m.W[0], np.float64)
    dm = gm.shape[1]
    U = (gm @ W0[:, :dm].T).astype(np.float32)
    V = (gt @ W0[:, dm:].T + m.b[0]).astype(np.float32)
    h = np.maximum(U[None, :, :] + V[:, None, :], np.float32(0)).reshape(Q * N, -1)
    acts = [h]
    for l in range(1, len(m.W) - 1):
        h = np.maximum(x3_layer(h, m.W[l], m.b[l]), 0).astype(np.float32)
        acts.append(h)
    out = x3_layer(h, m.W[-1], m.b[-1])
    return out.reshape(Q, N, -1), acts


def x3_mlp(api, m):
    return api.DeviceMLP.from_host(m, dev(), precision=api.WRF_BF16X3)


@pytest.mark.parametrize("N,Q,n_hidden", [(1000, 3, 4), (5, 1, 4), (128, 1, 4), (2048, 2, 4),
                                          (300, 7, 4), (700, 3, 1), (257, 2, 2), (129, 3, 3)])
def test_deform_x3_matches_emulation_and_oracle(api, N, Q, n_hidden):
    """Residuals and saved activations: ragged last tiles (5, 129, 257, 300,
    700 rows per query), whole tiles (128, 1000 = 7 x 128 + 104, 2048), and
    networks with 0 to 3 hidden 128 x 128 layers."""
    H, W = 90, 360
    sc = synth.make_scene(N, H, W, seed=N)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, n_hidden=n_hidden, seed=N)
    tx = synth.make_tx(Q, seed=N)
    ref, ref_acts = emulate_x3_mlp(sc, m, tx, H, W)
    ds, dmlp = api.DeviceScene.from_host(sc, dev()), x3_mlp(api, m)
    grid = api.make_grid(H, W)
    resid, acts = api.wrf_deform_acts(ds, dmlp, grid, T(tx))
    got = resid.cpu().numpy()
    assert torch.equal(resid, api.wrf_deform(ds, dmlp, grid, T(tx)))
    scale = np.abs(ref).max()
    rel = np.abs(got - ref) / scale
    p50 = np.percentile(rel, 50)
    fp64 = oracle.deform(sc, m, tx, H, W)
    err64 = np.abs(got - fp64).max() / np.abs(fp64).max()
    emu64 = np.abs(ref - fp64).max() / np.abs(fp64).max()
    print(f"deform x3 N={N} Q={Q} hidden={n_hidden}: vs emulation p50 {p50:.1e} "
          f"max {rel.max():.1e}; vs FP64 oracle {err64:.2e} (emulation {emu64:.2e})")
    assert p50 <= 2e-6
    assert rel.max() <= 3e-5
    assert err64 <= emu64 + 3e-5
    a = acts.cpu().numpy()
    assert a.shape == (len(m.W) - 1, Q * N, 128)
    for l, ra in enumerate(ref_acts):
        e = np.abs(a[l] - ra).max() / max(np.abs(ra).max(), 1e-30)
        print(f"  activation {l}: max err / max {e:.1e}")
        assert e <= 3e-5
    assert api.wrf_status_read() == 0


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("gain", [0.1, 1.0])
def test_forward_x3_matches_oracle(api, gain, fused):
    """Spectra within the FP32 tolerance (1e-4 x peak)."""
    H, W = 90, 360
    sc = synth.make_scene(1024, H, W, seed=0)
    m = synth.make_mlp(gain=gain, bias_std=0.02 if gain > 0.5 else 0.0, seed=0)
    tx = synth.make_tx(3, seed=0)
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, 9.0)
    r = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev(), fused=fused)
    out = r.forward(api.DeviceScene.from_host(sc, dev()), x3_mlp(api, m), T(tx))
    ok, worst, used = spectrum_error(out.cpu().numpy(), A, slack, 1e-4)
    print(f"forward x3 gain={gain} fused={fused}: max err/peak {worst:.2e} (slack px {used})")
    assert ok


def test_fused_equals_unfused_x3(api):
    """deform_project (the MLP epilogue projects) == deform then project."""
    H, W = 90, 360
    sc = synth.make_scene(3000, H, W, seed=12)
    m = x3_mlp(api, synth.make_mlp(gain=1.0, seed=12))
    tx = T(synth.make_tx(3, seed=12))
    ds = api.DeviceScene.from_host(sc, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    rec_f, _ = api.wrf_deform_project(ds, m, grid, tx)
    resid = api.wrf_deform(ds, m, grid, tx)
    rec_u, _ = api.wrf_project(ds, resid, 3, grid)
    assert torch.equal(rec_f, rec_u)


def test_zero_mlp_x3_is_identity(api):
    H, W = 90, 360
    sc = synth.make_scene(1500, H, W, seed=6)
    tx = T(synth.make_tx(2, seed=6))
    ds = api.DeviceScene.from_host(sc, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    a = api.Renderer(grid, dev()).forward(ds, x3_mlp(api, synth.zero_mlp()), tx)
    b = api.Renderer(grid, dev()).forward(ds, None, tx)
    assert torch.equal(a, b)


def test_x3_query_alone_equals_query_in_batch(api):
    H, W = 90, 360
    sc = synth.make_scene(3001, H, W, seed=7)
    m = x3_mlp(api, synth.make_mlp(seed=7))
    tx = T(synth.make_tx(9, seed=7))
    ds = api.DeviceScene.from_host(sc, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    batch = api.Renderer(grid, dev()).forward(ds, m, tx)
    for q in (0, 5, 8):
        alone = api.Renderer(grid, dev()).forward(ds, m, tx[q:q + 1])
        assert torch.equal(alone[0], batch[q])


@pytest.mark.parametrize("case", [(700, 3, 4), (300, 2, 1), (20000, 8, 4)])
@pytest.mark.parametrize("stop", [False, True])
def test_deform_backward_from_x3_activations(api, stop, case):
    """The MLP backward from the activations the three-product forward saved:
    every weight, bias and (stop = False) d_mean element against the FP64
    oracle, with the ReLU band widened to X3_BAND."""
    H, W = 90, 360
    n, Q, n_hidden = case
    sc = synth.make_scene(n, H, W, seed=43)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, n_hidden=n_hidden, seed=43)
    tx = synth.make_tx(Q, seed=43)
    d_resid = synth.rng(44).normal(size=(Q, sc.n, 5))
    dW_ref, db_ref, dmean, sl = oracle.mlp_grad(sc, m, tx, H, W, d_resid, stop_grad_mean=stop,
                                                band=X3_BAND)
    ds, dmlp = api.DeviceScene.from_host(sc, dev()), x3_mlp(api, m)
    grid = api.make_grid(H, W)
    _, acts = api.wrf_deform_acts(ds, dmlp, grid, T(tx))
    dW, db, d_mean = api.wrf_deform_backward(ds, dmlp, grid, T(tx), T(d_resid),
                                             stop_grad_mean=stop, acts=acts)
    grp = []
    for l in range(len(m.W)):
        grp += [(f"d_W[{l}]", dW[l].cpu().numpy(), dW_ref[l], sl["d_W"][l]),
                (f"d_b[{l}]", db[l].cpu().numpy(), db_ref[l], sl["d_b"][l])]
    if not stop:
        dmg = d_mean.cpu().numpy()
        grp += [(f"d_mean[:,{c}]", dmg[:, c], dmean[:, c], sl["d_mean"][:, c]) for c in range(2)]
    assert check_grads(grp, "deform backward (x3 activations)") <= 1.0


def test_autograd_x3_matches_oracle(api):
    """render_spectra with the three-product forward MLP: every gradient
    element against the oracle."""
    from paper_2506_12787_b300.autograd import SpectrumConfig, render_spectra
    H, W, n = 90, 360, 800
    sc = synth.make_scene(n, H, W, ls_mean=math.log(3.0), seed=n)
    m = synth.make_mlp(gain=0.5, bias_std=0.02, seed=n)
    Q = 2
    tx = synth.make_tx(Q, seed=n)
    dA = synth.rng(n + 1).normal(size=(Q, H, W))
    cfg = SpectrumConfig(api.make_grid(H, W, 16, 16, 9.0), mlp_precision=api.WRF_BF16X3)
    leaves = [T(a).requires_grad_() for a in sc.arrays()]
    ps = []
    for Wt, b in zip(m.W, m.b):
        ps += [T(Wt).requires_grad_(), T(b).requires_grad_()]
    out = render_spectra(cfg, T(tx), *leaves, ps)
    out.backward(T(dA))
    ref = oracle.grad(sc, m, tx, H, W, 9.0, dA, band=X3_BAND)
    sl = ref["slack"]
    grp = []
    names = ["d_mean", "d_log_scale", "d_rot", "d_opacity", "d_amp"]
    for k, lv in zip(names, leaves):
        a = lv.grad.cpu().numpy()
        if a.ndim == 2:
            grp += [(f"{k}[:,{c}]", a[:, c], ref[k][:, c],
                     sl["d_mean"][:, c] if k == "d_mean" else None) for c in range(2)]
        else:
            grp.append((k, a, ref[k]))
    for l, p in enumerate(ps[0::2]):
        grp.append((f"d_W[{l}]", p.grad.cpu().numpy(), ref["d_W"][l], sl["d_W"][l]))
    for l, p in enumerate(ps[1::2]):
        grp.append((f"d_b[{l}]", p.grad.cpu().numpy(), ref["d_b"][l], sl["d_b"][l]))
    assert check_grads(grp, "autograd x3") <= 1.0


def test_x3_training_workload_sampled(api):
    """The training workload's forward at full size (20k Gaussians, 64 TX,
    activations saved, as the training step launches it): residuals of 4
    sampled queries against the FP64 oracle, all 64 against the emulation's
    error level, and the saved activations of layer 0 against U + V."""
    H, W, N, Q = 90, 360, 20000, 64
    sc = synth.make_scene(N, H, W, seed=0)
    m = synth.make_mlp(seed=0)
    tx = synth.make_tx(Q, seed=3)
    ds, dmlp = api.DeviceScene.from_host(sc, dev()), x3_mlp(api, m)
    grid = api.make_grid(H, W, 16, 16, 9.0)
    resid, acts = api.wrf_deform_acts(ds, dmlp, grid, T(tx))
    torch.cuda.synchronize()
    assert api.wrf_status_read() == 0
    got = resid.cpu().numpy()
    sub = [0, 21, 37, 63]
    fp64 = oracle.deform(sc, m, tx[sub], H, W)
    err = np.abs(got[sub] - fp64).max() / np.abs(fp64).max()
    ref, _ = emulate_x3_mlp(sc, m, tx[sub], H, W)
    emu = np.abs(ref - fp64).max() / np.abs(fp64).max()
    print(f"x3 training workload, queries {sub}: max err / max|resid| {err:.2e} "
          f"(emulation {emu:.2e})")
    assert err <= emu + 3e-5
    assert np.all(np.isfinite(got))
    assert acts.shape == (len(m.W) - 1, Q * N, 128)
    assert bool(torch.all(acts >= 0)) and bool(torch.all(torch.isfinite(acts)))


def test_x3_rejects_deep_networks_and_bf16_acts(api):
    H, W = 90, 360
    sc = synth.make_scene(64, H, W, seed=2)
    ds = api.DeviceScene.from_host(sc, dev())
    tx = T(synth.make_tx(1, seed=2))
    deep = x3_mlp(api, synth.make_mlp(n_hidden=5, seed=2))
    with pytest.raises(api.WrfError):
        api.wrf_deform(ds, deep, api.make_grid(H, W), tx)
    bf = api.DeviceMLP.from_host(synth.make_mlp(seed=2), dev(), precision=api.WRF_BF16)
    with pytest.raises(api.WrfError):
        api.wrf_deform_acts(ds, bf, api.make_grid(H, W), tx)
