"""GPU parity of the forward path against the FP64 oracle (through the C ABI).

Tolerances: tile and key lists bit-exact; FP32 spectra within 1e-4 x the
spectrum's peak; BF16-MLP spectra within 2e-3 x peak (plus the oracle's
cutoff-band slack, see helpers.spectrum_error).  Every comparison prints its
error.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import oracle_proj_to_records, spectrum_error

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (8, 8), (16, 8), (32, 8), (32, 16)]


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


def _bin_gpu(api, rec32, H, W, tw, th, cap=None):
    Q, N = rec32.shape[:2]
    grid = api.make_grid(H, W, tw, th, 9.0)
    _, _, _, need = oracle.bin_f32(rec32, H, W, tw, th)
    cap = need if cap is None else cap
    gids, nk, offs = api.wrf_bin(T(rec32), N, Q, grid, cap)
    torch.cuda.synchronize()
    return gids.cpu().numpy().view(np.uint32), int(nk.item()), offs.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------ bin ----
@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("geo", [(90, 360), (37, 45), (180, 720)])
def test_bin_bit_exact(api, tile, geo):
    H, W = geo
    tw, th = tile
    rec = synth.random_rects_records(5, 2500, H, W, r_max=W / 10, seed=H + tw)
    counts, g_or, o_or, nk_or = oracle.bin_f32(rec, H, W, tw, th)
    g, nk, o = _bin_gpu(api, rec, H, W, tw, th)
    assert nk == nk_or
    assert np.array_equal(o, o_or)
    assert np.array_equal(g[:nk], g_or)
    print(f"bin {geo} tile {tile}: {nk} keys bit-exact")


def test_bin_full_size_batched_workload(api):
    """20k Gaussians x 256 queries (projected by the oracle without MLP,
    perturbed per query), tile lists bit-exact."""
    H, W = 90, 360
    sc = synth.make_scene(20000, H, W, seed=0)
    proj = oracle.project(sc, None, 9.0)[0]
    g = synth.rng(99)
    rec = np.repeat(oracle_proj_to_records(proj)[None], 256, axis=0)
    rec[..., 0:2] += g.normal(0, 1.5, size=(256, 20000, 2)).astype(np.float32)
    counts, g_or, o_or, nk_or = oracle.bin_f32(rec, H, W, 16, 16)
    gg, nk, o = _bin_gpu(api, rec, H, W, 16, 16)
    assert nk == nk_or and np.array_equal(o, o_or) and np.array_equal(gg[:nk], g_or)
    print(f"bin 20k x 256: {nk} keys bit-exact ({nk / (256 * 20000):.2f} tiles/Gaussian)")


def test_bin_edge_cases(api):
    H, W = 90, 360
    # empty scene
    g, nk, o = _bin_gpu(api, np.zeros((3, 0, 8), np.float32), H, W, 16, 16, cap=16)
    assert nk == 0 and np.all(o == 0)
    # everything off-grid
    rec = synth.random_rects_records(2, 300, H, W, seed=5)
    rec[..., 0] += 10 * W
    g, nk, o = _bin_gpu(api, rec, H, W, 16, 16, cap=16)
    assert nk == 0 and np.all(o == 0)
    # single Gaussian, N = 1; footprint exactly on tile boundaries
    rec = np.zeros((1, 1, 8), np.float32)
    rec[0, 0, [0, 1, 6, 7]] = [32.0, 16.0, 16.0, 0.0]
    counts, g_or, o_or, nk_or = oracle.bin_f32(rec, H, W, 16, 16)
    g, nk, o = _bin_gpu(api, rec, H, W, 16, 16)
    assert nk == nk_or == 3 and np.array_equal(o, o_or)
    # infinite footprint covers every tile
    rec[0, 0, 6:8] = np.inf
    g, nk, o = _bin_gpu(api, rec, H, W, 16, 16)
    assert nk == 23 * 6


def test_bin_overflow_reports_required_count(api):
    H, W = 90, 360
    rec = synth.random_rects_records(4, 1000, H, W, r_max=30, seed=8)
    _, _, _, need = oracle.bin_f32(rec, H, W, 16, 16)
    g, nk, o = _bin_gpu(api, rec, H, W, 16, 16, cap=need - 1)
    assert nk == need
    assert api.wrf_status_read() == -2  # WRF_ENOSPC, then cleared
    assert api.wrf_status_read() == 0


# --------------------------------------------------------------- project ---
def test_project_matches_oracle(api):
    H, W = 90, 360
    sc = synth.make_scene(3000, H, W, ls_std=0.5, seed=3)
    resid = synth.rng(3).normal(0, 0.5, size=(4, 3000, 5)).astype(np.float32)
    ref = oracle_proj_to_records(oracle.project(sc, resid.astype(np.float64), 9.0))
    grid = api.make_grid(H, W, 16, 16, 9.0)
    rec, cnt = api.wrf_project(api.DeviceScene.from_host(sc, dev()), T(resid), 4, grid)
    rec = rec.cpu().numpy()
    np.testing.assert_allclose(rec[..., 0:2], ref[..., 0:2], rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(rec[..., 2:5], ref[..., 2:5], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(rec[..., 5], ref[..., 5], rtol=1e-5)
    np.testing.assert_allclose(rec[..., 6:8], ref[..., 6:8], rtol=1e-5)
    # tile counts: the same integer function of the GPU's own records
    c_or, _, _, _ = oracle.bin_f32(rec, H, W, 16, 16)
    assert np.array_equal(cnt.cpu().numpy().view(np.uint32), c_or)


# ---------------------------------------------------------------- render ---
def _render_records(api, rec32, H, W, tile, q_cut=9.0):
    Q, N = rec32.shape[:2]
    grid = api.make_grid(H, W, tile[0], tile[1], q_cut)
    r = api.Renderer(grid, dev())
    out = r.bin_and_render(T(rec32), N, Q)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("geo", [(90, 360), (16, 32), (37, 45)])
def test_render_matches_oracle(api, tile, geo):
    H, W = geo
    n = 64 if geo == (16, 32) else 800
    sc = synth.make_scene(n, H, W, ls_mean=math.log(2.5), ls_std=0.4, seed=W)
    resid = synth.rng(W).normal(0, 0.3, size=(3, n, 5))
    proj = oracle.project(sc, resid, 9.0)
    A, slack = oracle.render(proj, H, W, 9.0)
    out = _render_records(api, oracle_proj_to_records(proj), H, W, tile)
    ok, worst, used = spectrum_error(out, A, slack, 1e-4)
    print(f"render {geo} tile {tile}: max err/peak {worst:.2e}, slack pixels {used}")
    assert ok


def test_render_without_cutoff(api):
    H, W = 16, 32
    sc = synth.make_scene(64, H, W, seed=1)
    proj = oracle.project(sc, None, math.inf)
    A, slack = oracle.render(proj, H, W, math.inf)
    out = _render_records(api, oracle_proj_to_records(proj), H, W, (16, 16), q_cut=math.inf)
    ok, worst, _ = spectrum_error(out, A, slack, 1e-4)
    print(f"render no cutoff: max err/peak {worst:.2e}")
    assert ok


def test_render_single_gaussian_closed_form(api):
    """Peak = w at an integer centre; lattice sum = 2 pi sigma^2 w (1 - e^-4.5)."""
    H, W = 90, 360
    sc = synth.Scene(np.array([[100.0, 40.0]], np.float32), np.log([[3.0, 3.0]]).astype(np.float32),
                     np.zeros(1, np.float32), np.array([40.0], np.float32),
                     np.array([0.75], np.float32))
    proj = oracle.project(sc, None, 9.0)
    out = _render_records(api, oracle_proj_to_records(proj), H, W, (16, 16))
    assert out[0, 40, 100] == pytest.approx(0.75, rel=1e-6)
    assert out.sum() == pytest.approx(2 * math.pi * 9 * 0.75 * (1 - math.exp(-4.5)), rel=6e-3)


def test_render_edge_cases(api):
    H, W = 90, 360
    out = _render_records(api, np.zeros((2, 0, 8), np.float32), H, W, (16, 16))
    assert np.all(out == 0)
    rec = oracle_proj_to_records(oracle.project(synth.make_scene(50, H, W, seed=2), None, 9.0))
    rec[..., 0] -= 1000.0
    assert np.all(_render_records(api, rec, H, W, (16, 16)) == 0)


def test_tile_shape_does_not_change_the_sum(api):
    H, W = 90, 360
    sc = synth.make_scene(2000, H, W, seed=11)
    rec = oracle_proj_to_records(oracle.project(sc, None, 9.0))
    outs = [_render_records(api, rec, H, W, t) for t in TILES]
    for o in outs[1:]:
        np.testing.assert_allclose(o, outs[0], rtol=0, atol=2e-6 * outs[0].max())


# ------------------------------------------------------------- full path ---
@pytest.mark.parametrize("gain", [0.1, 1.0])
@pytest.mark.parametrize("fused", [True, False])
def test_forward_fp32_matches_oracle(api, gain, fused):
    H, W = 90, 360
    sc = synth.make_scene(1024, H, W, seed=0)
    m = synth.make_mlp(gain=gain, bias_std=0.02 if gain > 0.5 else 0.0, seed=0)
    tx = synth.make_tx(3, seed=0)
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, 9.0)
    r = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev(), fused=fused)
    out = r.forward(api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev()), T(tx))
    ok, worst, used = spectrum_error(out.cpu().numpy(), A, slack, 1e-4)
    print(f"forward fp32 gain={gain} fused={fused}: max err/peak {worst:.2e} (slack px {used})")
    assert ok


def test_deform_fp32_residuals(api):
    H, W = 90, 360
    sc = synth.make_scene(700, H, W, seed=4)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=4)
    tx = synth.make_tx(5, seed=4)
    ref = oracle.deform(sc, m, tx, H, W)
    got = api.wrf_deform(api.DeviceScene.from_host(sc, dev()), api.DeviceMLP.from_host(m, dev()),
                         api.make_grid(H, W), T(tx)).cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"deform fp32 max err / max|resid| = {err:.2e}")
    assert err < 5e-6  # the encoding phase is reduced exactly (no 2^k-amplified rounding)


def test_zero_mlp_is_identity_on_gpu(api):
    H, W = 90, 360
    sc = synth.make_scene(1500, H, W, seed=6)
    tx = synth.make_tx(2, seed=6)
    ds = api.DeviceScene.from_host(sc, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    a = api.Renderer(grid, dev()).forward(ds, api.DeviceMLP.from_host(synth.zero_mlp(), dev()), T(tx))
    b = api.Renderer(grid, dev()).forward(ds, None, T(tx))
    assert torch.equal(a, b)


def test_query_alone_equals_query_in_batch(api):
    H, W = 90, 360
    sc = synth.make_scene(3000, H, W, seed=7)
    m = api.DeviceMLP.from_host(synth.make_mlp(seed=7), dev())
    tx = T(synth.make_tx(9, seed=7))
    ds = api.DeviceScene.from_host(sc, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    batch = api.Renderer(grid, dev()).forward(ds, m, tx)
    for q in (0, 4, 8):
        alone = api.Renderer(grid, dev()).forward(ds, m, tx[q:q + 1])
        assert torch.equal(alone[0], batch[q])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x3"])
def test_zero_queries(api, precision):
    """Q = 0 through the whole path (deform + project, bin, render): empty
    spectra, no device error; the next non-empty call is unaffected."""
    H, W = 90, 360
    prec = {"fp32": api.WRF_FP32, "bf16": api.WRF_BF16, "bf16x3": api.WRF_BF16X3}[precision]
    ds = api.DeviceScene.from_host(synth.make_scene(300, H, W, seed=4), dev())
    m = api.DeviceMLP.from_host(synth.make_mlp(seed=4), dev(), precision=prec)
    r = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev())
    # the key count and offsets must be written even with nothing to bin:
    # poison the renderer's buffers so a missing write shows
    r._buf("nk", 256).fill_(0xFF)
    r._buf("offs", 256).fill_(0xFF)
    out = r.forward(ds, m, T(np.zeros((0, 3), np.float32)))
    torch.cuda.synchronize()
    assert tuple(out.shape) == (0, H, W)
    assert api.wrf_status_read() == 0
    tx = T(synth.make_tx(2, seed=4))
    again = r.forward(ds, m, tx)
    ref = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev()).forward(ds, m, tx)
    assert torch.equal(again, ref)
