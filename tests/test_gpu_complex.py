"""GPU parity of the two-channel path (Sec. 6.1: the real and imaginary parts
rendered as separate channels and decomposed into magnitude and phase)
against the FP64 oracle, through the C ABI.

The comparison is on the complex value reconstructed from the GPU's
(magnitude, phase), mag (cos phase, sin phase), against the oracle's (re,
im) per channel, within 1e-4 x the channel peak (FP32 MLP) or 2e-3 (BF16
MLP) plus the cutoff-band slack: phase alone is ill-conditioned where the
magnitude vanishes.  The magnitude itself is compared within the same bound.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import spectrum_error
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


def complex_scene(n, H, W, seed):
    sc = synth.make_scene(n, H, W, seed=seed)
    rng = np.random.default_rng(seed + 70)
    ph = rng.uniform(-math.pi, math.pi, n)
    amp = np.stack([sc.amp * np.cos(ph), sc.amp * np.sin(ph)], 1).astype(np.float32)
    return synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, amp)


def check(name, out, sc, m, tx, H, W, tol, wrap=False):
    re, im, mag, ph, slack = oracle.forward_complex(sc, m, tx, H, W, 9.0, wrap=wrap)
    gm, gp = out[:, 0].astype(np.float64), out[:, 1].astype(np.float64)
    ok_re, e_re, _ = spectrum_error(gm * np.cos(gp), re, slack, tol)
    ok_im, e_im, _ = spectrum_error(gm * np.sin(gp), im, slack, tol)
    ok_m, e_m, used = spectrum_error(gm, mag, slack, tol)
    print(f"{name}: re {e_re:.2e}, im {e_im:.2e}, magnitude {e_m:.2e} (x peak; slack px {used})")
    assert ok_re and ok_im and ok_m


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 2e-3), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_two_channel_forward_matches_oracle(api, precision, tol, tile):
    H, W = 90, 360
    sc = complex_scene(2000, H, W, 1)
    m = synth.make_mlp(gain=0.1, seed=1)
    tx = synth.make_tx(3, seed=1)
    prec = {"fp32": api.WRF_FP32, "bf16": api.WRF_BF16, "bf16x3": api.WRF_BF16X3}[precision]
    r = api.Renderer(api.make_grid(H, W, tile[0], tile[1], 9.0), dev())
    out = r.forward(api.DeviceScene.from_host(sc, dev()),
                    api.DeviceMLP.from_host(m, dev(), precision=prec), T(tx))
    assert tuple(out.shape) == (3, 2, H, W)
    check(f"2-channel {precision} {tile}", out.cpu().numpy(), sc, m, tx, H, W, tol)


def test_two_channel_with_wrap_and_projection_only(api):
    """No MLP (wrf_project), azimuth wrap, a small grid with ragged tiles."""
    H, W = 40, 72
    sc = complex_scene(300, H, W, 2)
    tx = np.zeros((2, 3))
    r = api.Renderer(api.make_grid(H, W, 16, 16, 9.0, wrap=True), dev())
    out = r.forward(api.DeviceScene.from_host(sc, dev()), None, T(tx))
    check("2-channel, wrap, no MLP", out.cpu().numpy(), sc, None, tx, H, W, 1e-4, wrap=True)


def test_two_channel_records_tail(api):
    """The imaginary weights follow the records: sigmoid(opacity) amp_im."""
    H, W = 40, 72
    sc = complex_scene(50, H, W, 3)
    ds = api.DeviceScene.from_host(sc, dev())
    rec, _ = api.wrf_project(ds, None, 2, api.make_grid(H, W, 16, 16, 9.0))
    tail = api.record_tail(rec, 2, 50).cpu().numpy()
    want = sc.amp[:, 1].astype(np.float64) / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    assert np.allclose(tail, np.broadcast_to(want, (2, 50)), rtol=1e-6, atol=1e-7)
    re_w = rec[..., 5].cpu().numpy()
    want_re = sc.amp[:, 0].astype(np.float64) / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    assert np.allclose(re_w, np.broadcast_to(want_re, (2, 50)), rtol=1e-6, atol=1e-7)


def test_two_channel_reduces_to_one(api):
    """A zero imaginary part: the magnitude equals |one-channel map| bit for
    bit, the phase is 0 or pi."""
    H, W = 90, 360
    sc = synth.make_scene(1500, H, W, seed=4)
    amp2 = np.stack([sc.amp, np.zeros_like(sc.amp)], 1)
    sc2 = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, amp2)
    m = synth.make_mlp(seed=4)
    tx = T(synth.make_tx(2, seed=4))
    grid = api.make_grid(H, W, 16, 16, 9.0)
    one = api.Renderer(grid, dev()).forward(api.DeviceScene.from_host(sc, dev()),
                                            api.DeviceMLP.from_host(m, dev()), tx)
    two = api.Renderer(grid, dev()).forward(api.DeviceScene.from_host(sc2, dev()),
                                            api.DeviceMLP.from_host(m, dev()), tx)
    assert torch.equal(two[:, 0], one.abs())
    ph = two[:, 1]
    assert bool(torch.all((ph == 0) | (ph.abs() == math.pi)))


def test_two_channel_rssi_and_backward_limit(api):
    H = W = 16
    sc = complex_scene(50, H, W, 5)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=5)
    tx = synth.make_tx(8, seed=5)
    ds, dm = api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev())
    r = api.wrf_rssi(ds, dm, api.make_grid(H, W, 16, 16, 9.0), T(tx)).cpu().numpy()
    ro, rslack = oracle.rssi(sc, m, tx, H, W, 9.0)
    _, _, mag, _, _ = oracle.forward_complex(sc, m, tx, H, W, 9.0)
    peak = mag.reshape(8, -1).max(1)
    d = np.abs(r.astype(np.float64) - ro)
    print(f"2-channel rssi: max err/peak {float((d / peak).max()):.2e}")
    assert np.all(d <= 1e-4 * peak + rslack)
    with pytest.raises(api.WrfError) as e:
        api.wrf_project_backward(ds, None, 1, torch.zeros((1, 50, 6), device=dev()))
    assert e.value.status == _lib.WRF_EUNSUPPORTED


@pytest.mark.parametrize("cfg", [(16, 8, 4, 1, 0), (32, 16, 4, 2, 1), (32, 8, 2, 2, 0),
                                 (16, 16, 4, 1, 1), (32, 16, 4, 1, 1)],
                         ids=lambda c: "%dx%dp%db%d%s" % (c[:4] + ("t" if c[4] else "",)))
def test_two_channel_launch_knobs(api, cfg):
    """Every rasteriser knob on the two-channel path: magnitude and phase
    bit-identical to the default knobs of the same tile (the same per-pixel
    arithmetic and order), and the complex value within 1e-4 x peak of the
    oracle (FP32 MLP); one case with azimuth wrap."""
    tw, th, px, bf, tma = cfg
    H, W = 90, 360
    wrap = cfg[:4] == (16, 16, 4, 1)
    sc = complex_scene(2500, H, W, 3)
    m = synth.make_mlp(gain=0.1, seed=3)
    tx = synth.make_tx(2, seed=3)
    ds = api.DeviceScene.from_host(sc, dev())
    dm = api.DeviceMLP.from_host(m, dev(), precision=api.WRF_FP32)
    outs = []
    for p, b, t in ((px, bf, tma), (2, 1, 0)):
        r = api.Renderer(api.make_grid(H, W, tw, th, 9.0, wrap=wrap, px_per_thread=p,
                                       batch_factor=b, tma_staging=t), dev())
        outs.append(r.forward(ds, dm, T(tx)).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    check(f"2-channel knobs {cfg} wrap={wrap}", outs[0], sc, m, tx, H, W, 1e-4, wrap=wrap)
