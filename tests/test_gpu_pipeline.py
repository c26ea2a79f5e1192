"""GPU checks of the library's host-to-host forward pipeline (wrf_pipeline_*).

The pipeline issues the same library calls as batched.BatchedForward (one
graph per slot of wrf_deform_project + wrf_bin + wrf_render), so every step's
spectra must equal, bit for bit, the batched forward of the same TX
positions; a step whose keys outgrow the capacity sized at the first step is
recomputed with a grown capacity and still equals it; one step is checked
against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import spectrum_error

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


def direct(api, ds, dm, grid, tx_np):
    """Spectra of tx_np [Q,3] through BatchedForward (sized for these TX)."""
    from paper_2506_12787_b300.batched import BatchedForward
    fw = BatchedForward(ds, dm, grid, tx_np.shape[0], dev())
    tx = torch.as_tensor(tx_np, dtype=torch.float32, device=dev())
    need = fw.reserve(tx)
    fw.run(tx)
    torch.cuda.synchronize()
    fw.check()
    return fw.out.cpu().numpy().copy(), need


@pytest.mark.parametrize("channels,precision", [(1, "BF16"), (2, "FP32")])
def test_pipeline_equals_batched_forward(api, channels, precision):
    from paper_2506_12787_b300.batched import NativePipeline
    Q, N = 8, 6000
    sc = synth.make_scene(N, H, W, seed=31)
    if channels == 2:
        amp2 = np.stack([sc.amp, synth.rng(32).normal(0, 0.5, N).astype(np.float32)], 1)
        sc = synth.Scene(sc.mean, sc.log_scale, sc.rot, sc.opacity_logit, amp2)
    m = synth.make_mlp(seed=31)
    prec = getattr(api, "WRF_" + precision)
    ds = api.DeviceScene.from_host(sc, dev())
    dm = api.DeviceMLP.from_host(m, dev(), precision=prec)
    grid = api.make_grid(H, W, 32, 16, 9.0, px_per_thread=4)
    pipe = NativePipeline(ds, dm, grid, Q)
    batches = [synth.make_tx(Q, seed=40 + i) for i in range(5)]
    outs = []
    for i, b in enumerate(batches):
        outs.append(pipe.step(torch.as_tensor(b, dtype=torch.float32).contiguous()))
        if i % 2 == 1:  # results of a slot stay valid until that slot is reused
            pipe.wait()
            for j in (i - 1, i):
                ref, _ = direct(api, ds, dm, grid, batches[j])
                got = outs[j].numpy()
                assert got.shape == ref.shape
                assert np.array_equal(got, ref), f"step {j} differs from the batched forward"
    pipe.wait()
    ref, _ = direct(api, ds, dm, grid, batches[4])
    assert np.array_equal(outs[4].numpy(), ref)
    pipe.close()
    print(f"pipeline {channels} channel(s) {precision}: 5 steps bit-identical to BatchedForward")


def test_pipeline_recovers_from_key_overflow(api):
    """key_margin = 1: the capacity is the first step's key count + 1024; a
    later step with more keys is recomputed into its own host buffer."""
    from paper_2506_12787_b300.batched import NativePipeline
    Q, N = 4, 20000
    sc = synth.make_scene(N, H, W, seed=33)
    m = synth.make_mlp(gain=1.0, bias_std=0.05, seed=33)
    ds = api.DeviceScene.from_host(sc, dev())
    dm = api.DeviceMLP.from_host(m, dev(), precision=api.WRF_BF16)
    grid = api.make_grid(H, W, 16, 16, 9.0)
    cands = [synth.make_tx(Q, seed=100 + i) for i in range(12)]
    needs = [direct(api, ds, dm, grid, c)[1] for c in cands]
    lo, hi = int(np.argmin(needs)), int(np.argmax(needs))
    if needs[hi] <= needs[lo] + 1024:
        pytest.skip(f"key counts too close to force an overflow: {min(needs)}..{max(needs)}")
    pipe = NativePipeline(ds, dm, grid, Q, key_margin=1.0)
    order = [lo, hi, lo, hi, hi]
    for j, i in enumerate(order):
        o = pipe.step(torch.as_tensor(cands[i], dtype=torch.float32).contiguous())
        pipe.wait()
        ref, _ = direct(api, ds, dm, grid, cands[i])
        assert np.array_equal(o.numpy(), ref), f"step {j} (batch {i}) differs after recovery"
    # the device status word is clear afterwards
    assert api.wrf_status_read(None) == 0
    pipe.close()
    print(f"pipeline overflow: keys {needs[lo]} then {needs[hi]} (+{needs[hi] - needs[lo]}), "
          f"recomputed and bit-identical")


def test_pipeline_matches_oracle(api):
    from paper_2506_12787_b300.batched import NativePipeline
    Q, N = 3, 2000
    sc = synth.make_scene(N, H, W, seed=35)
    m = synth.make_mlp(seed=35)
    tx = synth.make_tx(Q, seed=35)
    ds = api.DeviceScene.from_host(sc, dev())
    dm = api.DeviceMLP.from_host(m, dev(), precision=api.WRF_FP32)
    pipe = NativePipeline(ds, dm, api.make_grid(H, W, 16, 16, 9.0), Q)
    out = pipe.step(torch.as_tensor(tx, dtype=torch.float32).contiguous())
    pipe.wait()
    A, slack, _, _ = oracle.forward(sc, m, tx, H, W, 9.0)
    ok, worst, _ = spectrum_error(out.numpy(), A, slack, 1e-4)
    print(f"pipeline vs FP64 oracle: err/peak {worst:.2e}")
    assert ok
    pipe.close()
