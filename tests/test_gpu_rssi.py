"""GPU parity of the RSSI head (Sec. 7.2: global average pool of the rendered
map's magnitude, Sec. 6.6) against the FP64 oracle, through the C ABI.

Tolerances: the un-pooled map within 1e-4 x its peak (plus the cutoff-band
slack, helpers.spectrum_error), as for the FP32 forward path; the pooled value
within 1e-4 x the map's peak plus the pooled slack (pooling averages the
per-pixel errors).  The paper's setting is 50 Gaussians on a 16 x 16 map.
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


def _run(api, sc, m, tx, H, W, q_cut=9.0, with_map=True):
    grid = api.make_grid(H, W, 16, 16, q_cut)
    Q = tx.shape[0]
    mp = torch.full((Q, H, W), float("nan"), device=dev()) if with_map else None
    r = api.wrf_rssi(api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev()), grid,
                     T(tx), map_out=mp)
    torch.cuda.synchronize()
    return r.cpu().numpy(), (mp.cpu().numpy() if with_map else None)


def _check(name, r, mp, sc, m, tx, H, W, q_cut=9.0):
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, q_cut)
    ro, rslack = oracle.rssi(sc, m, tx, H, W, q_cut)
    ok_map, worst_map, used = spectrum_error(mp, A, slack, 1e-4)
    peak = np.abs(A).reshape(len(tx), -1).max(1)
    d = np.abs(r.astype(np.float64) - ro)
    worst = float((np.maximum(d - rslack, 0) / np.maximum(peak, 1e-30)).max())
    print(f"{name}: map max err/peak {worst_map:.2e} (slack px {used}); "
          f"pooled max err/peak {worst:.2e}; rssi[0] gpu {r[0]:.6e} oracle {ro[0]:.6e}")
    assert ok_map
    assert np.all(d <= 1e-4 * peak + rslack)


@pytest.mark.parametrize("seed", [0, 1])
def test_rssi_paper_setting(api, seed):
    """50 Gaussians, 16 x 16 map (Sec. 7.2), 64 TX positions, MLP with
    non-zero biases so the residuals move every Gaussian."""
    H = W = 16
    sc = synth.make_scene(50, H, W, ls_mean=math.log(1.5), ls_std=0.3, seed=seed)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=seed)
    tx = synth.make_tx(64, seed=seed + 10)
    r, mp = _run(api, sc, m, tx, H, W)
    _check(f"rssi 50 x 16x16 seed {seed}", r, mp, sc, m, tx, H, W)


def test_rssi_limits_and_shapes(api):
    """The largest scene (64 Gaussians), a non-square 40 x 24 map (960
    pixels: a ragged last pass of the 256 threads), an MLP with one hidden
    128 x 128 layer (n_layers = 3), and the untruncated kernel (q_cut = inf)."""
    H, W = 24, 40
    sc = synth.make_scene(64, H, W, ls_mean=math.log(2.0), seed=3)
    m = synth.make_mlp(n_hidden=2, gain=1.0, bias_std=0.05, seed=3)
    tx = synth.make_tx(5, seed=3)
    r, mp = _run(api, sc, m, tx, H, W)
    _check("rssi 64 x 24x40, 1 hidden layer", r, mp, sc, m, tx, H, W)
    r, mp = _run(api, sc, m, tx, H, W, q_cut=math.inf)
    _check("rssi 64 x 24x40, q_cut inf", r, mp, sc, m, tx, H, W, q_cut=math.inf)


def test_rssi_takes_the_magnitude(api):
    """Negative amplitudes: the map changes sign, the pooled magnitude does
    not (Sec. 6.6)."""
    H = W = 16
    sc = synth.make_scene(50, H, W, ls_mean=math.log(1.5), seed=7)
    neg = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, -sc.amp)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=7)
    tx = synth.make_tx(8, seed=7)
    r, mp = _run(api, sc, m, tx, H, W)
    rn, mpn = _run(api, neg, m, tx, H, W)
    _check("rssi negative amplitudes", rn, mpn, neg, m, tx, H, W)
    assert np.array_equal(mpn, -mp) and np.array_equal(rn, r)


def test_rssi_map_equals_the_tiled_path(api):
    """The fused head's map agrees with wrf_deform_project + wrf_bin +
    wrf_render (FP32 MLP) within FP32 rounding order."""
    H = W = 16
    sc = synth.make_scene(50, H, W, ls_mean=math.log(1.5), seed=2)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=2)
    tx = synth.make_tx(16, seed=2)
    _, mp = _run(api, sc, m, tx, H, W)
    out = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev()).forward(
        api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev()), T(tx))
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, 9.0)
    ok, worst, used = spectrum_error(mp, out.cpu().numpy().astype(np.float64), slack, 1e-5)
    print(f"rssi map vs tiled path: max diff/peak {worst:.2e} (slack px {used})")
    assert ok


def test_rssi_query_alone_equals_in_batch(api):
    """A query's value and map do not depend on the other queries."""
    H = W = 16
    sc = synth.make_scene(50, H, W, ls_mean=math.log(1.5), seed=4)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=4)
    tx = synth.make_tx(32, seed=4)
    r, mp = _run(api, sc, m, tx, H, W)
    for i in (0, 17, 31):
        ri, mpi = _run(api, sc, m, tx[i:i + 1], H, W)
        assert ri[0] == r[i] and np.array_equal(mpi[0], mp[i])


def test_rssi_edge_cases(api):
    H = W = 16
    m = synth.make_mlp(seed=1)
    tx = synth.make_tx(4, seed=1)
    # empty scene: zero RSSI and map
    empty = synth.make_scene(0, H, W, seed=1)
    r, mp = _run(api, empty, m, tx, H, W)
    assert np.all(r == 0) and np.all(mp == 0)
    # no queries: a no-op
    grid = api.make_grid(H, W, 16, 16, 9.0)
    sc = synth.make_scene(50, H, W, seed=1)
    ds, dm = api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev())
    out = api.wrf_rssi(ds, dm, grid, T(np.zeros((0, 3))))
    assert out.numel() == 0
    # limits: more than 64 Gaussians, more than 65536 pixels
    big = api.DeviceScene.from_host(synth.make_scene(65, H, W, seed=1), dev())
    with pytest.raises(api.WrfError) as e:
        api.wrf_rssi(big, dm, grid, T(tx))
    assert e.value.status == _lib.WRF_EUNSUPPORTED
    with pytest.raises(api.WrfError) as e:
        api.wrf_rssi(ds, dm, api.make_grid(257, 256, 16, 16, 9.0), T(tx))
    assert e.value.status == _lib.WRF_EUNSUPPORTED
