"""GPU parity of the rasteriser's launch knobs (pixels per thread 2 or 4,
records per thread per shared-memory batch 1 or 2, records staged by
per-thread cp.async or by TMA gathers) on every tile shape, and of the
autotuner that searches them.

A pixel's terms are the same FP32 operations whatever the knobs (the same
row-pair coefficients, the same column offset from the tile centre, the
records summed in ascending order); only which records a warp considers
changes with its block width (8 or 16 columns), and a record outside a
pixel's warp block contributes nothing unless FP32 rounding puts the pixel
inside the cutoff.  So every configuration must equal the default one
except at pixels within the oracle's cutoff-band slack, and match the FP64
oracle at the render tolerance (1e-4 x peak plus that slack).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import oracle_proj_to_records, spectrum_error
from paper_2506_12787_b300 import autotune

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


def render(api, rec32, H, W, cfg, wrap=False):
    Q, N = rec32.shape[:2]
    r = api.Renderer(autotune.make_grid(H, W, cfg, 9.0, wrap), dev())
    out = r.bin_and_render(T(rec32), N, Q)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def records():
    """Oracle-projected records on two geometries (one with ragged tiles on
    both axes), with the oracle's spectra and cutoff-band slack."""
    out = {}
    for H, W, n in ((90, 360, 6000), (37, 45, 700)):
        sc = synth.make_scene(n, H, W, ls_mean=math.log(2.5), ls_std=0.5, seed=H + W)
        resid = synth.rng(W).normal(0, 0.3, size=(3, n, 5))
        proj = oracle.project(sc, resid, 9.0)
        A, slack = oracle.render(proj, H, W, 9.0)
        out[(H, W)] = (oracle_proj_to_records(proj), A, slack)
    return out


@pytest.mark.parametrize("geo", [(90, 360), (37, 45)])
@pytest.mark.parametrize("cfg", autotune.space(), ids=lambda c: autotune.config_name(*c))
def test_knobs_match_default_and_oracle(api, records, geo, cfg):
    H, W = geo
    rec32, A, slack = records[geo]
    out = render(api, rec32, H, W, cfg)
    ok, worst, used = spectrum_error(out, A, slack, 1e-4)
    base = render(api, rec32, H, W, (cfg[0], cfg[1], 2, 1))
    d = np.abs(out.astype(np.float64) - base)
    peak = np.abs(A).reshape(A.shape[0], -1).max(axis=1)[:, None, None]
    differ = int(np.count_nonzero(d))
    print(f"{autotune.config_name(*cfg)} {H}x{W}: err/peak {worst:.2e} (slack pixels {used}), "
          f"pixels differing from the default knobs: {differ} of {d.size}")
    assert ok
    assert np.all(d <= 1e-6 * peak + slack)
    assert differ <= max(4, d.size // 10000)


def test_knobs_with_azimuth_wrap(api):
    H, W = 90, 360
    sc = synth.make_scene(2500, H, W, ls_mean=math.log(2.5), ls_std=0.4, seed=5)
    m = sc.mean.astype(np.float64).copy()
    m[:1000, 0] = synth.rng(6).uniform(-12, 12, 1000) % W  # Gaussians on the seam
    sc = synth.Scene(m.astype(np.float32), sc.log_scale, sc.rot, sc.opacity_logit, sc.amp)
    proj = oracle.project(sc, None, 9.0, Q=2)
    A, slack = oracle.render(proj, H, W, 9.0, wrap=True)
    rec32 = oracle_proj_to_records(proj)
    for cfg in ((32, 8, 4, 2, 0), (16, 16, 4, 1, 1), (32, 16, 2, 2, 1)):
        out = render(api, rec32, H, W, cfg, wrap=True)
        ok, worst, used = spectrum_error(out, A, slack, 1e-4)
        print(f"wrap {autotune.config_name(*cfg)}: err/peak {worst:.2e}")
        assert ok


def test_batched_forward_with_knobs(api):
    """The batched, graph-replayed forward (the path the autotuner times) at
    the 20000-Gaussian scene: every knob setting equals the default up to
    the cutoff band; two queries against the FP64 oracle."""
    from paper_2506_12787_b300.batched import BatchedForward
    H, W, N, Q = 90, 360, 20000, 16
    sc = synth.make_scene(N, H, W, seed=21)
    m = synth.make_mlp(seed=21)
    tx_np = synth.make_tx(Q, seed=21)
    ds, dm = api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev(),
                                                                        precision=api.WRF_BF16)
    tx = T(tx_np)
    stream = torch.cuda.Stream()
    outs = {}
    for cfg in ((32, 8, 2, 1), (32, 8, 2, 2), (32, 8, 4, 1), (32, 8, 4, 2), (32, 16, 2, 1),
                (32, 16, 4, 2), (32, 16, 4, 1, 1), (32, 8, 2, 2, 1)):
        fw = BatchedForward(ds, dm, autotune.make_grid(H, W, cfg, 9.0), Q, dev())
        with torch.cuda.stream(stream):
            fw.reserve(tx, stream)
        g = fw.graph(tx, stream)
        with torch.cuda.stream(stream):
            g.replay()
        stream.synchronize()
        fw.check(stream)
        outs[cfg] = fw.out.cpu().numpy().copy()
    A, slack, _, _ = oracle.forward(sc, m, tx_np[:2], H, W, 9.0)
    for cfg, o in outs.items():
        base = outs[(cfg[0], cfg[1], 2, 1)]  # the same tile shape, default knobs
        ok, worst, _ = spectrum_error(o[:2], A, slack, 2e-3)
        d = np.abs(o[:2].astype(np.float64) - base[:2])
        peak = np.abs(A).reshape(2, -1).max(axis=1)[:, None, None]
        differ = int(np.count_nonzero(o != base))
        print(f"batched {autotune.config_name(*cfg)}: err/peak {worst:.2e}, "
              f"differing pixels {differ} of {o.size}")
        assert ok
        assert np.all(d <= 1e-6 * peak + slack)
        assert differ <= o.size // 10000


def test_autotune_searches_and_caches(api, tmp_path):
    H, W, N, Q = 90, 360, 5000, 8
    sc = synth.make_scene(N, H, W, seed=31)
    m = synth.make_mlp(seed=31)
    ds, dm = api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev(),
                                                                        precision=api.WRF_BF16)
    tx = T(synth.make_tx(Q, seed=31))
    cand = [(32, 8, 2, 1, 0), (32, 8, 4, 2, 0), (16, 16, 2, 2, 1), (16, 8, 4, 1, 1)]
    path = str(tmp_path / "cache.json")
    best, times = autotune.tune(ds, dm, H, W, tx, 9.0, reps=2, cache_path=path, candidates=cand,
                                verbose=True)
    assert best in cand
    assert set(times) == {autotune.config_name(*c) for c in cand}
    assert all(t > 0 for t in times.values())
    assert times[autotune.config_name(*best)] == min(times.values())
    # the same search again is served from the cache; another space is not
    best2, times2 = autotune.tune(ds, dm, H, W, tx, 9.0, cache_path=path, candidates=cand)
    assert best2 == best and times2 == times
    best3, times3 = autotune.tune(ds, dm, H, W, tx, 9.0, reps=2, cache_path=path,
                                  candidates=cand[:2])
    assert set(times3) == {autotune.config_name(*c) for c in cand[:2]}
