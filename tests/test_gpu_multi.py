"""Multi-scene batches: one launch sequence over queries of several resident
scenes (each its own Gaussians and deformation network, Sec. 4.2), replayed
from one CUDA graph.  Each query's spectrum must equal, bit for bit, the
spectrum of the same query run alone through its own scene's single-scene
path, and match the FP64 oracle within 2e-3 x peak (BF16 MLP)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import spectrum_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2506_12787_b300 import api, build
    build.build()
    assert torch.cuda.is_available()
    return api


def dev():
    return torch.device("cuda:0")


def _scenes(H, W):
    ns = [3000, 7000, 12001]
    return ([synth.make_scene(n, H, W, seed=70 + i) for i, n in enumerate(ns)],
            [synth.make_mlp(gain=0.2, bias_std=0.02, seed=80 + i) for i in range(3)])


@pytest.mark.parametrize("tile", [(32, 8, 2, 1, 0), (16, 16, 2, 1, 0), (32, 16, 4, 1, 1)],
                         ids=["32x8", "16x16", "32x16p4b1-tma"])
def test_mixed_batch_equals_each_scene_alone(api, tile):
    """(The third case stages the records with TMA gathers, whose tensor map
    spans the int32 row range: rows come from the device-side query bases.)"""
    from paper_2506_12787_b300.batched import BatchedForward, MultiSceneForward
    H, W = 90, 360
    scs, mls = _scenes(H, W)
    ds = [api.DeviceScene.from_host(s, dev()) for s in scs]
    dm = [api.DeviceMLP.from_host(m, dev(), precision=api.WRF_BF16) for m in mls]
    grid = api.make_grid(H, W, tile[0], tile[1], 9.0, px_per_thread=tile[2],
                         batch_factor=tile[3], tma_staging=tile[4])
    Q = 16
    # unsorted scenes, a repeated scene, and two unused slots
    scene_of = [2, 0, 1, 1, 2, 0, 2, 1, 0, 0, 2, 1, 1, 2]
    tx = synth.make_tx(len(scene_of), seed=90)
    mf = MultiSceneForward(ds, dm, grid, Q, dev())
    mf.set_batch(scene_of, tx)
    mf.reserve()
    g = mf.graph()
    mf.out.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    mf.check()
    out = mf.out.cpu().numpy()
    assert np.all(out[len(scene_of):] == 0), "unused slots render zeros"
    worst = 0.0
    for q, sid in enumerate(scene_of):
        fw = BatchedForward(ds[sid], dm[sid], grid, 1, dev())
        txq = torch.as_tensor(tx[q:q + 1], dtype=torch.float32, device=dev())
        fw.reserve(txq)
        alone = fw.run(txq).cpu().numpy()[0]
        assert np.array_equal(alone, out[q]), f"query {q} (scene {sid}) differs from alone"
        A, slack, _, _ = oracle.forward(scs[sid], mls[sid], tx[q:q + 1], H, W, 9.0)
        ok, err, _ = spectrum_error(out[q:q + 1], A, slack, 2e-3)
        worst = max(worst, err)
        assert ok, (q, err)
    print(f"mixed batch of 3 scenes, tile {tile}: every query bit-identical to its scene alone; "
          f"max err/peak vs oracle {worst:.2e}")
    # a second batch through the same graph: another mix
    scene_of2 = [1, 1, 1, 0]
    tx2 = synth.make_tx(4, seed=91)
    mf.set_batch(scene_of2, tx2)
    g.replay()
    torch.cuda.synchronize()
    mf.check()
    out2 = mf.out.cpu().numpy()
    for q, sid in enumerate(scene_of2):
        fw = BatchedForward(ds[sid], dm[sid], grid, 1, dev())
        txq = torch.as_tensor(tx2[q:q + 1], dtype=torch.float32, device=dev())
        fw.reserve(txq)
        assert np.array_equal(fw.run(txq).cpu().numpy()[0], out2[q])
    assert np.all(out2[4:] == 0)


def test_record_capacity_overflow_is_reported(api):
    from paper_2506_12787_b300.batched import MultiSceneForward
    H, W = 90, 360
    scs, mls = _scenes(H, W)
    ds = [api.DeviceScene.from_host(s, dev()) for s in scs]
    dm = [api.DeviceMLP.from_host(m, dev(), precision=api.WRF_BF16) for m in mls]
    mf = MultiSceneForward(ds, dm, api.make_grid(H, W, 16, 16, 9.0), 4, dev(),
                           rec_capacity=15000, key_capacity=1 << 20)
    mf.set_batch([2, 2], synth.make_tx(2, seed=3))  # 24002 records > 15000
    mf.run()
    torch.cuda.synchronize()
    assert api.wrf_status_read() == api._lib.WRF_ENOSPC
    assert float(mf.out.abs().max()) == 0.0
    mf.set_batch([0, 1], synth.make_tx(2, seed=3))  # 10000 records fit
    mf.run()
    torch.cuda.synchronize()
    assert api.wrf_status_read() == 0
    assert float(mf.out[:2].amax()) > 0.0
