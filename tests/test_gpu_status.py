"""Device-side failure reporting without a GPU fault: every wait in the
kernels is bounded and, when it runs out, records WRF_ETIMEOUT in the
library's status word and returns.  A diagnostic entry point waits on an
mbarrier phase that nothing completes; the host must read WRF_ETIMEOUT, the
word must clear, and the context must stay usable."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_reports():
    from paper_2506_12787_b300 import _lib, api, build
    build.build()
    L = _lib.load()
    dev = torch.device("cuda:0")
    assert api.wrf_status_read() == 0
    done = torch.full((1,), -1, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    _lib.check(L.wrf_selftest_wait(50_000_000, C.c_void_p(done.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    st = api.wrf_status_read()
    dt = time.perf_counter() - t0
    print(f"bounded wait gave up after {dt * 1e3:.1f} ms, status {st}")
    assert st == _lib.WRF_ETIMEOUT
    assert int(done.item()) == 0
    assert dt < 5.0
    assert api.wrf_status_read() == 0  # cleared by the read
    # the context still works: a normal forward afterwards
    H, W = 32, 64
    sc = synth.make_scene(50, H, W, seed=3)
    out = api.Renderer(api.make_grid(H, W, 16, 16, 9.0), dev).forward(
        api.DeviceScene.from_host(sc, dev), None, torch.zeros((1, 3), device=dev))
    torch.cuda.synchronize()
    assert float(out.max()) > 0 and api.wrf_status_read() == 0


def test_selftest_rejects_bad_limits():
    from paper_2506_12787_b300 import _lib, build
    build.build()
    L = _lib.load()
    assert L.wrf_selftest_wait(0, None, None) == _lib.WRF_EINVAL
    assert L.wrf_selftest_wait(3_000_000_000, None, None) == _lib.WRF_EINVAL
