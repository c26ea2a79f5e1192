"""GPU parity of the paper's own head (Sec. 4.1-4.2, Sec. 6.1: tanh-mapped
angular centres, Cholesky covariance, attenuation and complex response, the
deformation network with skips every two layers and outputs dmu, dpsi,
ddelta) against the FP64 oracle, through the C ABI.

Tolerances.  The network runs in FP32 (sums of <= 160 + 237 products per
output, 9 layers), and the centre enters the encoding through tanhf (a few
ulp of (tanh u + 1) / 2, i.e. <= ~1e-7 relative, raised by 2^9 pi at the top
band of L_mean = 10 to ~2e-4 rad of sin / cos).  With unit-gain weights that
phase error reaches the residuals attenuated by the network, so records
carry: centres within 2e-3 px, weights within 1e-4 x the largest |w|,
inverse covariance and footprint radii within FP32 rounding (2e-6 relative;
no network term).  Spectra: a centre error e moves a Gaussian of standard
deviation >= 1.5 px by at most ~0.6 e / 1.5 of its peak, so the measured
centre errors (<= 2e-4 px) allow 1e-4 x the channel peak, the bound of the
other FP32 paths, plus the cutoff-band slack."""
import math

import numpy as np
import pytest
import torch

import synth
from helpers import spectrum_error
from oracle import paper
from paper_2506_12787_b300 import _lib

pytestmark = pytest.mark.gpu

H, W = 90, 360


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


def paper_mlp(seed, width=156, n_hidden=8, move=10.0):
    """Unit-gain network; the centre outputs scaled so dmu is a few pixels."""
    m = synth.make_paper_mlp(gain=1.0, bias_std=0.05, width=width, n_hidden=n_hidden, seed=seed)
    m.W[-1][:2] *= np.float32(move)
    m.b[-1][:2] *= np.float32(move)
    return m


def gpu_records(api, sc, m, tx, grid):
    Q, N = tx.shape[0], sc.mu.shape[0]
    ds = api.DevicePaperScene.from_host(sc, dev())
    dm = None if m is None else api.DevicePaperMLP.from_host(m, dev())
    rec = api.wrf_paper_deform_project(ds, dm, grid, T(tx))
    torch.cuda.synchronize()
    return rec.cpu().numpy().astype(np.float64), api.record_tail(rec, Q, N).cpu().numpy()


def check_records(g, tail, sc, m, tx, q_cut=9.0):
    Q, N = tx.shape[0], sc.mu.shape[0]
    resid = paper.residuals(sc, m, tx, H, W) if m is not None else np.zeros((Q, N, 5))
    pre, pim = paper.project(sc, resid, H, W, q_cut)
    s = 0.72134752044448170368  # log2(e) / 2, the records' conic scale
    e_c = float(np.abs(g[..., :2] - pre[..., :2]).max())
    conic = pre[..., 2:5] * s
    e_q = float((np.abs(g[..., 2:5] - conic) / np.abs(conic).max(-1, keepdims=True)).max())
    e_r = float((np.abs(g[..., 6:8] - pre[..., 6:8]) / pre[..., 6:8]).max())
    wmax = max(float(np.abs(pre[..., 5]).max()), float(np.abs(pim[..., 5]).max()))
    e_w = max(float(np.abs(g[..., 5] - pre[..., 5]).max()),
              float(np.abs(tail - pim[..., 5]).max())) / wmax
    print(f"records: centre {e_c:.2e} px, conic {e_q:.2e}, radii {e_r:.2e}, weight {e_w:.2e} "
          f"(|dmu| up to {float(np.abs(resid[..., :2]).max()):.2f} px)")
    assert e_c <= 2e-3 and e_q <= 2e-6 and e_r <= 2e-6 and e_w <= 1e-4
    return resid


def test_paper_records_match_oracle(api):
    """The paper's network (8 x 156, skips every two layers); N = 1000 = 15 x
    64 + 40 Gaussians (a ragged last CTA), 3 TX."""
    sc = synth.make_paper_scene(1000, H, W, seed=1)
    m = paper_mlp(1)
    tx = synth.make_tx(3, seed=1)
    g, tail = gpu_records(api, sc, m, tx, api.make_grid(H, W, 16, 16, 9.0))
    resid = check_records(g, tail, sc, m, tx)
    assert float(np.abs(resid[..., :2]).max()) > 1.0  # the centres really move


@pytest.mark.parametrize("width,n_hidden", [(100, 3), (160, 1), (17, 5), (156, 7)])
def test_paper_network_shapes(api, width, n_hidden):
    """Other widths (padded to 160 inside) and depths (skips at 2, 4, 6 below
    n_hidden only)."""
    sc = synth.make_paper_scene(130, H, W, seed=2)
    m = paper_mlp(2, width=width, n_hidden=n_hidden)
    tx = synth.make_tx(2, seed=2)
    g, tail = gpu_records(api, sc, m, tx, api.make_grid(H, W, 16, 16, 9.0))
    check_records(g, tail, sc, m, tx)


def test_paper_no_deformation_records(api):
    sc = synth.make_paper_scene(77, H, W, seed=3)
    tx = np.zeros((2, 3))
    g, tail = gpu_records(api, sc, None, tx, api.make_grid(H, W, 16, 16, 9.0))
    check_records(g, tail, sc, None, tx)
    assert np.array_equal(g[0], g[1])


def check_spectra(out, sc, m, tx, grid_w, q_cut, wrap, Hs=H, Ws=W, tol=1e-4):
    mag, ph, re, im, slack, _ = paper.forward(sc, m, tx, Hs, Ws, q_cut, wrap=wrap)
    gm, gp = out[:, 0].astype(np.float64), out[:, 1].astype(np.float64)
    ok_re, e_re, _ = spectrum_error(gm * np.cos(gp), re, slack, tol)
    ok_im, e_im, _ = spectrum_error(gm * np.sin(gp), im, slack, tol)
    ok_m, e_m, used = spectrum_error(gm, mag, slack, tol)
    print(f"paper spectra ({grid_w}): re {e_re:.2e}, im {e_im:.2e}, magnitude {e_m:.2e} "
          f"(x peak; slack px {used})")
    assert ok_re and ok_im and ok_m


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_paper_spectra_match_oracle(api, tile):
    """Magnitude and phase of Eq. 13 with the paper's head, 2000 Gaussians,
    3 TX, through binning and the two-channel rasteriser."""
    sc = synth.make_paper_scene(2000, H, W, seed=4)
    m = paper_mlp(4)
    tx = synth.make_tx(3, seed=4)
    r = api.Renderer(api.make_grid(H, W, tile[0], tile[1], 9.0), dev())
    out = r.forward_paper(api.DevicePaperScene.from_host(sc, dev()),
                          api.DevicePaperMLP.from_host(m, dev()), T(tx))
    assert tuple(out.shape) == (3, 2, H, W)
    check_spectra(out.cpu().numpy(), sc, m, tx, tile, 9.0, False)


def test_paper_spectra_wrap_no_deformation(api):
    """The reference frame alone on a wrapped 40 x 72 grid (ragged tiles)."""
    Hs, Ws = 40, 72
    sc = synth.make_paper_scene(300, Hs, Ws, ls_mean=math.log(2.0), seed=5)
    tx = np.zeros((1, 3))
    r = api.Renderer(api.make_grid(Hs, Ws, 16, 16, 9.0, wrap=True), dev())
    out = r.forward_paper(api.DevicePaperScene.from_host(sc, dev()), None, T(tx))
    check_spectra(out.cpu().numpy(), sc, None, tx, (16, 16), 9.0, True, Hs, Ws)


def test_paper_single_gaussian_and_determinism(api):
    """N = 1 (one CTA row of 64 used) matches the one-primitive closed form's
    oracle; repeated calls are bit-identical."""
    sc = synth.make_paper_scene(1, H, W, seed=6)
    m = paper_mlp(6)
    tx = synth.make_tx(1, seed=6)
    g, tail = gpu_records(api, sc, m, tx, api.make_grid(H, W, 16, 16, 9.0))
    check_records(g, tail, sc, m, tx)
    sc = synth.make_paper_scene(500, H, W, seed=7)
    ds, dm = api.DevicePaperScene.from_host(sc, dev()), api.DevicePaperMLP.from_host(m, dev())
    grid = api.make_grid(H, W, 16, 16, 9.0)
    a = api.wrf_paper_deform_project(ds, dm, grid, T(synth.make_tx(5, seed=7)))
    b = api.wrf_paper_deform_project(ds, dm, grid, T(synth.make_tx(5, seed=7)))
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_paper_workspace_too_small(api):
    sc = synth.make_paper_scene(100, H, W, seed=8)
    m = paper_mlp(8)
    ds, dm = api.DevicePaperScene.from_host(sc, dev()), api.DevicePaperMLP.from_host(m, dev())
    ws = torch.empty(1024, dtype=torch.uint8, device=dev())
    with pytest.raises(api.WrfError) as e:
        api.wrf_paper_deform_project(ds, dm, api.make_grid(H, W, 16, 16, 9.0),
                                     T(synth.make_tx(2, seed=8)), ws=ws)
    assert e.value.status == _lib.WRF_EINVAL


# ---------------------------------------------------------------------------
# Tensor-core network (precision = WRF_BF16): BF16 weights, activations and
# gamma(mean), FP32 accumulation, the query's encoding term in FP32.


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def hilo(v):
    """An FP32 value as the kernel's BF16 pair hi + lo (lo = BF16 of v - hi)."""
    v = np.asarray(v, np.float32)
    hi = bf16(v)
    return hi + bf16((v - hi.astype(np.float32)).astype(np.float32))


def emulate_paper_bf16(sc, m, tx, Hs=H, Ws=W):
    """Residuals [Q,N,5] with the tensor-core kernel's rounding points: every
    product of a BF16 operand pair (activations, gamma(mean) and the weights
    that multiply them) summed in FP64 and rounded to FP32; the query's term
    W_s gamma(s) + b computed in FP32 and entering as BF16 hi + lo (as do the
    biases); ReLU, then BF16."""
    import oracle
    x0, y0 = paper.centres(sc.mu[:, 0], sc.mu[:, 1], Hs, Ws)
    gm = bf16(np.stack([oracle.pe(np.array([x / Ws, y / Hs]), m.L_mean) for x, y in zip(x0, y0)]))
    s = (np.asarray(tx, np.float64) - np.asarray(m.room_min)) / np.asarray(m.room_size)
    gt = np.stack([oracle.pe(v, m.L_tx) for v in s])
    dm, width = gm.shape[1], m.W[0].shape[0]
    Q, N = tx.shape[0], gm.shape[0]
    h = None
    for l in range(len(m.W) - 1):
        Wl = np.asarray(m.W[l], np.float64)
        if l == 0:
            z = gm @ bf16(Wl[:, :dm]).T
            vec = gt @ Wl[:, dm:].T + m.b[l]
            z = z[None, :, :]
        elif l in paper.SKIPS:
            z = h @ bf16(Wl[:, :width]).T + (gm @ bf16(Wl[:, width:width + dm]).T)[None]
            vec = gt @ Wl[:, width + dm:].T + m.b[l]
        else:
            z = h @ bf16(Wl).T
            vec = np.broadcast_to(np.asarray(m.b[l], np.float64), (Q, width))
        z = z.astype(np.float32) + hilo(vec.astype(np.float32)).astype(np.float32)[:, None, :]
        h = bf16(np.maximum(z, 0))
        if h.shape[0] != Q:
            h = np.broadcast_to(h, (Q, N, width))
    return (h @ bf16(m.W[-1]).T).astype(np.float32) + hilo(m.b[-1]).astype(np.float32)


def bf16_records(api, sc, m, tx, grid=None):
    grid = grid or api.make_grid(H, W, 16, 16, 9.0)
    ds = api.DevicePaperScene.from_host(sc, dev())
    dm = api.DevicePaperMLP.from_host(m, dev(), precision=api.WRF_BF16)
    rec = api.wrf_paper_deform_project(ds, dm, grid, T(tx))
    torch.cuda.synchronize()
    return rec, rec.cpu().numpy().astype(np.float64), \
        api.record_tail(rec, tx.shape[0], sc.mu.shape[0]).cpu().numpy()


def residuals_from_records(g, tail, sc, Hs=H, Ws=W):
    """(dmu_x, dmu_y, w_re, w_im) of the GPU records, for comparison."""
    x0, y0 = paper.centres(sc.mu[:, 0], sc.mu[:, 1], Hs, Ws)
    return np.stack([g[..., 0] - x0[None], g[..., 1] - y0[None], g[..., 5], tail], -1)


def emulated_records(sc, resid, Hs=H, Ws=W):
    pre, pim = paper.project(sc, resid.astype(np.float64), Hs, Ws, 9.0)
    x0, y0 = paper.centres(sc.mu[:, 0], sc.mu[:, 1], Hs, Ws)
    return np.stack([pre[..., 0] - x0[None], pre[..., 1] - y0[None], pre[..., 5], pim[..., 5]], -1)


@pytest.mark.parametrize("N,Q", [(1000, 3), (5, 1), (128, 1), (300, 7), (257, 2)])
def test_paper_bf16_matches_emulation(api, N, Q):
    """Ragged tiles, a single row, one exact tile, odd tile counts (the last
    pair of a CTA has one tile)."""
    sc = synth.make_paper_scene(N, H, W, seed=N)
    m = paper_mlp(N)
    tx = synth.make_tx(Q, seed=N)
    _, g, tail = bf16_records(api, sc, m, tx)
    got = residuals_from_records(g, tail, sc)
    want = emulated_records(sc, emulate_paper_bf16(sc, m, tx))
    scale = np.abs(want).max(axis=(0, 1))
    rel = np.abs(got - want) / scale
    ref64 = emulated_records(sc, paper.residuals(sc, m, tx, H, W))
    e64 = float((np.abs(got - ref64) / scale).max())
    p50, p99 = np.percentile(rel, [50, 99])
    print(f"paper bf16 N={N} Q={Q}: vs emulation p50 {p50:.1e} p99 {p99:.1e} max {rel.max():.1e}; "
          f"vs FP64 oracle {e64:.1e}")
    # bulk: FP32 accumulation order; a few rows: BF16 rounding flips of an
    # activation on a rounding boundary, carried through the later layers
    assert p50 <= 1e-5
    assert rel.max() <= 2e-2


def test_paper_bf16_spectra(api):
    """Magnitude / phase through binning and the two-channel rasteriser
    against the oracle's projection and render of the emulated residuals."""
    sc = synth.make_paper_scene(2000, H, W, seed=11)
    m = paper_mlp(11)
    tx = synth.make_tx(3, seed=11)
    resid = emulate_paper_bf16(sc, m, tx).astype(np.float64)
    pre, pim = paper.project(sc, resid, H, W, 9.0)
    import oracle
    re, s_re = oracle.render(pre, H, W, 9.0)
    im, s_im = oracle.render(pim, H, W, 9.0)
    slack = np.maximum(s_re, s_im)
    r = api.Renderer(api.make_grid(H, W, 32, 8, 9.0), dev())
    out = r.forward_paper(api.DevicePaperScene.from_host(sc, dev()),
                          api.DevicePaperMLP.from_host(m, dev(), precision=api.WRF_BF16),
                          T(tx)).cpu().numpy().astype(np.float64)
    gm, gp = out[:, 0], out[:, 1]
    # flip level: single BF16 rounding flips carried through eight layers move
    # a record by up to ~5e-3 of its scale (the emulation test's max), i.e.
    # a centre by up to ~0.05 px at |dmu| ~ 10 px, which bounds the spectrum
    # difference near 1e-2 x peak rather than at FP32 rounding level
    ok_re, e_re, _ = spectrum_error(gm * np.cos(gp), re, slack, 1e-2)
    ok_im, e_im, _ = spectrum_error(gm * np.sin(gp), im, slack, 1e-2)
    print(f"paper bf16 spectra vs emulated residuals: re {e_re:.2e}, im {e_im:.2e} (x peak)")
    assert ok_re and ok_im


@pytest.mark.parametrize("width,n_hidden", [(100, 3), (160, 1), (17, 5), (156, 7)])
def test_paper_bf16_network_shapes(api, width, n_hidden):
    sc = synth.make_paper_scene(200, H, W, seed=12)
    m = paper_mlp(12, width=width, n_hidden=n_hidden)
    tx = synth.make_tx(3, seed=12)
    _, g, tail = bf16_records(api, sc, m, tx)
    got = residuals_from_records(g, tail, sc)
    want = emulated_records(sc, emulate_paper_bf16(sc, m, tx))
    rel = np.abs(got - want) / np.abs(want).max(axis=(0, 1))
    print(f"paper bf16 {width} x {n_hidden}: p50 {np.median(rel):.1e} max {rel.max():.1e}")
    assert np.median(rel) <= 1e-5 and rel.max() <= 2e-2


def test_paper_bf16_query_alone_equals_batch_and_repeats(api):
    """A query's records do not depend on the other queries of the call, and
    calls repeat bit for bit."""
    sc = synth.make_paper_scene(700, H, W, seed=13)
    m = paper_mlp(13)
    tx = synth.make_tx(5, seed=13)
    rec, _, _ = bf16_records(api, sc, m, tx)
    rec2, _, _ = bf16_records(api, sc, m, tx)
    assert torch.equal(rec, rec2)
    one, _, _ = bf16_records(api, sc, m, tx[3:4])
    assert torch.equal(one[0], rec[3])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x3"])
def test_paper_workload_full_size_sampled(api, precision):
    """The bench's paper workload as the bench launches it (20,000 Gaussians,
    64 TX, 360x90, tile 32x8, unit-gain network with small biases): two whole
    queries of the batch against the oracle -- the FP64 head for FP32 and for
    the three-product BF16 network (both held to 1e-4 x peak), the
    projection and render of the BF16-emulated residuals for BF16."""
    import math as _m
    import oracle
    sc = synth.make_paper_scene(20000, H, W, ls_mean=_m.log(3.0), ls_std=0.3, seed=0)
    m = synth.make_paper_mlp(gain=1.0, bias_std=0.05, seed=0)
    tx = synth.make_tx(64, seed=1)
    prec = {"bf16": api.WRF_BF16, "bf16x3": api.WRF_BF16X3, "fp32": api.WRF_FP32}[precision]
    r = api.Renderer(api.make_grid(H, W, 32, 8, 9.0), dev())
    out = r.forward_paper(api.DevicePaperScene.from_host(sc, dev()),
                          api.DevicePaperMLP.from_host(m, dev(), precision=prec), T(tx))
    torch.cuda.synchronize()
    picks = [0, 37]
    g = out.cpu().numpy()[picks].astype(np.float64)
    if precision in ("fp32", "bf16x3"):
        mag, ph, re, im, slack, _ = paper.forward(sc, m, tx[picks], H, W, 9.0)
        tol = 1e-4
    else:
        resid = emulate_paper_bf16(sc, m, tx[picks]).astype(np.float64)
        pre, pim = paper.project(sc, resid, H, W, 9.0)
        re, s_re = oracle.render(pre, H, W, 9.0)
        im, s_im = oracle.render(pim, H, W, 9.0)
        slack = np.maximum(s_re, s_im)
        tol = 1e-2
    ok_re, e_re, _ = spectrum_error(g[:, 0] * np.cos(g[:, 1]), re, slack, tol)
    ok_im, e_im, _ = spectrum_error(g[:, 0] * np.sin(g[:, 1]), im, slack, tol)
    print(f"paper workload {precision}, queries {picks}: re {e_re:.2e}, im {e_im:.2e} (x peak)")
    assert ok_re and ok_im


@pytest.mark.parametrize("N,Q", [(1000, 3), (5, 1), (300, 7)])
@pytest.mark.parametrize("shape", [(156, 8), (100, 3), (17, 5)])
def test_paper_bf16x3_records_match_oracle(api, N, Q, shape):
    """Three-product BF16 network: records against the FP64 head (centres,
    weights) at the FP32 path's bound, for ragged / single-row / odd tile
    counts and several network shapes."""
    width, n_hidden = shape
    sc = synth.make_paper_scene(N, H, W, seed=N + width)
    m = paper_mlp(N, width=width, n_hidden=n_hidden)
    tx = synth.make_tx(Q, seed=N)
    ds = api.DevicePaperScene.from_host(sc, dev())
    dm = api.DevicePaperMLP.from_host(m, dev(), precision=api.WRF_BF16X3)
    rec = api.wrf_paper_deform_project(ds, dm, api.make_grid(H, W, 16, 16, 9.0), T(tx))
    torch.cuda.synchronize()
    g = rec.cpu().numpy().astype(np.float64)
    tail = api.record_tail(rec, Q, N).cpu().numpy()
    got = residuals_from_records(g, tail, sc)
    want = emulated_records(sc, paper.residuals(sc, m, tx, H, W))
    scale = np.abs(want).max(axis=(0, 1))
    rel = float((np.abs(got - want) / scale).max())
    print(f"paper bf16x3 N={N} Q={Q} {width}x{n_hidden}: records vs FP64 oracle {rel:.1e}")
    assert rel <= 1e-4


def test_paper_bf16x3_query_alone_equals_batch(api):
    sc = synth.make_paper_scene(700, H, W, seed=14)
    m = paper_mlp(14)
    tx = synth.make_tx(5, seed=14)
    ds = api.DevicePaperScene.from_host(sc, dev())
    dm = api.DevicePaperMLP.from_host(m, dev(), precision=api.WRF_BF16X3)
    grid = api.make_grid(H, W, 16, 16, 9.0)
    rec = api.wrf_paper_deform_project(ds, dm, grid, T(tx)).clone()
    one = api.wrf_paper_deform_project(ds, dm, grid, T(tx[2:3]))
    torch.cuda.synchronize()
    assert torch.equal(one[0], rec[2])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "none"])
def test_paper_host_pipeline_matches_forward_paper(api, precision):
    """HostPipeline over PaperForward (TX from pinned host memory, magnitude /
    phase back to pinned host memory, copies overlapped) returns exactly the
    output of Renderer.forward_paper for alternating TX batches."""
    from paper_2506_12787_b300.batched import HostPipeline, PaperForward
    H, W, N, Q = 90, 360, 2000, 8
    prec = _lib.WRF_BF16 if precision == "bf16" else _lib.WRF_FP32
    sc = synth.make_paper_scene(N, H, W, seed=21)
    ds = api.DevicePaperScene.from_host(sc, dev())
    dm = None if precision == "none" else api.DevicePaperMLP.from_host(paper_mlp(21), dev(),
                                                                        precision=prec)
    grid = api.make_grid(H, W, 32, 8, 9.0)
    txs = [synth.make_tx(Q, seed=50 + i) for i in range(2)]
    ref = [api.Renderer(grid, dev()).forward_paper(ds, dm, T(t)).cpu().numpy() for t in txs]
    fw = PaperForward(ds, dm, grid, Q, dev())
    assert fw.launches_per_run == {"fp32": 10, "bf16": 8, "none": 7}[precision]
    for t in txs:  # key capacity for both batches
        fw.reserve(T(t))
    pipe = HostPipeline(fw)
    hosts = [torch.as_tensor(t).pin_memory() for t in txs]
    for i in range(6):
        out = pipe.step(hosts[i % 2])
        if i >= 4:  # steps 4 and 5 land in different ring slots
            pipe.sync()
            assert np.array_equal(out.numpy(), ref[i % 2])
    fw.check()
