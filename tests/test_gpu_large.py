"""The large batched workload at full size: 200,000 Gaussians (log-scales
N(ln 2 px, 0.5^2)), a 720 x 180 (0.5 degree) FP32 spectrum, 1,024 TX
positions in one launch sequence with the BF16 tensor-core MLP, replayed from
a CUDA graph as the benchmark runs it.  Sampled queries are checked against
the FP64 oracle at 2e-3 x peak; every spectrum must be finite and non-empty,
and the key count must fit the 32-bit key index."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import spectrum_error

pytestmark = pytest.mark.gpu


def test_large_workload_sampled():
    from paper_2506_12787_b300 import api, build
    from paper_2506_12787_b300.batched import BatchedForward
    build.build()
    dev = torch.device("cuda:0")
    N, H, W, Q = 200000, 180, 720, 1024
    sc = synth.make_scene(N, H, W, ls_mean=math.log(2.0), ls_std=0.5, seed=0)
    mh = synth.make_mlp(seed=0)
    tx_np = synth.make_tx(Q, seed=1)
    fw = BatchedForward(api.DeviceScene.from_host(sc, dev),
                        api.DeviceMLP.from_host(mh, dev, precision=api.WRF_BF16),
                        api.make_grid(H, W, 16, 16, 9.0), Q, dev)
    tx = torch.as_tensor(tx_np, device=dev)
    nk = fw.reserve(tx)
    g = fw.graph(tx)
    g.replay()
    torch.cuda.synchronize()
    fw.check()
    print(f"large: {nk} keys ({nk / (N * Q):.2f} tiles per Gaussian)")
    assert 0 < nk < 2 ** 32
    peaks = fw.out.reshape(Q, -1).amax(1)
    assert bool(torch.all(torch.isfinite(fw.out))) and bool(torch.all(peaks > 0))
    idx = [3, 1000]
    out = fw.out[idx].cpu().numpy()
    A, slack, _, _ = oracle.forward(sc, mh, tx_np[idx], H, W, 9.0)
    ok, worst, used = spectrum_error(out, A, slack, 2e-3)
    print(f"large 200k x 1024 (sampled {idx}): max err/peak {worst:.2e}, slack px {used}")
    assert ok
