"""GPU parity of the azimuth-wrap option (0 and W columns the same
direction) against the FP64 oracle: wrapped tile lists bit-exact, spectra
within 1e-4 x peak (FP32 MLP) or 2e-3 x peak (BF16 MLP) plus the cutoff-band
slack, gradients element by element within 1e-3 relative (floor 1e-3 of
the group's largest component), the RSSI head with wrap, and the
reported limit (a footprint as wide as W - tile width)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import check_grads, oracle_proj_to_records, spectrum_error
from paper_2506_12787_b300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2506_12787_b300 import api, build
    build.build()
    assert torch.cuda.is_available()
    return api


def dev():
    return torch.device("cuda:0")


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev())


def seam_scene(n, H, W, seed):
    """Half of the Gaussians within 12 px of the 0 / W seam."""
    sc = synth.make_scene(n, H, W, seed=seed)
    m = sc.mean.astype(np.float64).copy()
    rng = np.random.default_rng(seed + 50)
    k = n // 2
    m[:k, 0] = rng.uniform(-12, 12, k) % W
    return synth.Scene(m.astype(np.float32), sc.log_scale, sc.rot, sc.opacity_logit, sc.amp)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8), (32, 16)])
def test_wrapped_tile_lists_bit_exact(api, tile):
    tw, th = tile
    H, W = 90, 360
    sc = seam_scene(1500, H, W, 1)
    proj = oracle.project(sc, None, 9.0, Q=2)
    rec32 = oracle_proj_to_records(proj)
    counts, gids_o, offs_o, nk_o = oracle.bin_f32(rec32, H, W, tw, th, wrap=True)
    grid = api.make_grid(H, W, tw, th, 9.0, wrap=True)
    gids, nk, offs = api.wrf_bin(T(rec32), 1500, 2, grid, nk_o)
    torch.cuda.synchronize()
    assert int(nk.item()) == nk_o
    assert np.array_equal(offs.cpu().numpy().view(np.uint32), offs_o)
    assert np.array_equal(gids.cpu().numpy().view(np.uint32)[:nk_o], gids_o)
    # wrapping adds keys for the seam Gaussians
    _, _, _, nk_flat = oracle.bin_f32(rec32, H, W, tw, th)
    print(f"wrap tile {tw}x{th}: {nk_o} keys (flat plane {nk_flat})")
    assert nk_o > nk_flat


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 2e-3)])
def test_wrapped_forward_matches_oracle(api, precision, tol):
    H, W = 90, 360
    sc = seam_scene(2000, H, W, 2)
    m = synth.make_mlp(gain=0.1, seed=2)
    tx = synth.make_tx(3, seed=2)
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, 9.0, wrap=True)
    prec = api.WRF_BF16 if precision == "bf16" else api.WRF_FP32
    r = api.Renderer(api.make_grid(H, W, 16, 16, 9.0, wrap=True), dev())
    out = r.forward(api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev(), precision=prec),
                    T(tx))
    ok, worst, used = spectrum_error(out.cpu().numpy(), A, slack, tol)
    Aflat, _, _, _ = oracle.forward(sc, m, tx, H, W, 9.0)
    seam_mass = float(np.abs(A - Aflat)[:, :, :16].sum() + np.abs(A - Aflat)[:, :, -16:].sum())
    print(f"wrap forward {precision}: max err/peak {worst:.2e} (slack px {used}); "
          f"mass moved across the seam {seam_mass:.2f}")
    assert ok and seam_mass > 1.0


def test_wrapped_gradients(api):
    from paper_2506_12787_b300.autograd import SpectrumConfig, render_spectra
    H, W = 30, 64
    sc = seam_scene(200, H, W, 3)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=3)
    tx = synth.make_tx(3, seed=3)
    dA = np.random.default_rng(3).normal(size=(3, H, W)) / (3 * H * W)
    cfg = SpectrumConfig(api.make_grid(H, W, 16, 16, 9.0, wrap=True))
    leaves = [T(a).requires_grad_() for a in sc.arrays()]
    ps = []
    for Wt, b in zip(m.W, m.b):
        ps += [T(Wt).requires_grad_(), T(b).requires_grad_()]
    out = render_spectra(cfg, T(tx), *leaves, ps)
    out.backward(T(dA))
    ref = oracle.grad(sc, m, tx, H, W, 9.0, dA, wrap=True)
    names = ["d_mean", "d_log_scale", "d_rot", "d_opacity", "d_amp"]
    grp = []
    for k, lv in zip(names, leaves):
        a = lv.grad.cpu().numpy()
        if a.ndim == 2:
            grp += [(f"{k}[:,{c}]", a[:, c], ref[k][:, c]) for c in range(a.shape[1])]
        else:
            grp.append((k, a, ref[k]))
    sl = ref["slack"]  # ReLU decisions an FP32 forward may take either way
    for l, (p, rW) in enumerate(zip(ps[0::2], ref["d_W"])):
        grp.append((f"d_W[{l}]", p.grad.cpu().numpy(), rW, sl["d_W"][l]))
    for l, (p, rb) in enumerate(zip(ps[1::2], ref["d_b"])):
        grp.append((f"d_b[{l}]", p.grad.cpu().numpy(), rb, sl["d_b"][l]))
    assert check_grads(grp, "wrap grad") <= 1.0


def test_wrapped_rssi(api):
    H = W = 16
    sc = seam_scene(50, H, W, 4)
    sc = synth.Scene(sc.mean, sc.log_scale - np.float32(math.log(2.0)), sc.rot, sc.opacity_logit,
                     sc.amp)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=4)
    tx = synth.make_tx(16, seed=4)
    grid = api.make_grid(H, W, 16, 16, 9.0, wrap=True)
    r = api.wrf_rssi(api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev()), grid,
                     T(tx))
    ro, rslack = oracle.rssi(sc, m, tx, H, W, 9.0, wrap=True)
    A, _, _, _ = oracle.forward(sc, m, tx, H, W, 9.0, wrap=True)
    peak = np.abs(A).reshape(16, -1).max(1)
    d = np.abs(r.cpu().numpy().astype(np.float64) - ro)
    print(f"wrap rssi: max err/peak {float((d / peak).max()):.2e}")
    assert np.all(d <= 1e-4 * peak + rslack)


def test_wrap_limits(api):
    """A footprint as wide as W - tile width is reported (status word), and
    wrap with an infinite cutoff is refused."""
    H, W = 32, 64
    rec = np.zeros((1, 2, 8), np.float32)
    rec[0, :, 0] = [10.0, 40.0]
    rec[0, :, 1] = [16.0, 16.0]
    rec[0, :, 2:5] = [0.01, 0.0, 0.01]
    rec[0, :, 5] = 1.0
    rec[0, :, 6] = [3.0, 25.0]   # 2 * 25 >= 64 - 16
    rec[0, :, 7] = [3.0, 3.0]
    api.wrf_status_read()
    grid = api.make_grid(H, W, 16, 16, 9.0, wrap=True)
    api.wrf_bin(T(rec), 2, 1, grid, 64)
    assert api.wrf_status_read() == _lib.WRF_EUNSUPPORTED
    rec[0, 1, 6] = 3.0
    api.wrf_bin(T(rec), 2, 1, grid, 64)
    assert api.wrf_status_read() == _lib.WRF_OK
    with pytest.raises(api.WrfError) as e:
        api.wrf_bin(T(rec), 2, 1, api.make_grid(H, W, 16, 16, math.inf, wrap=True), 64)
    assert e.value.status == _lib.WRF_EINVAL
