"""wrf_bin_noalloc: tile binning for callers that cannot allocate device
memory (a host application that owns the device's memory pool, or a
latency-critical loop where a cudaMalloc is not allowed).  The entry point
takes its scratch space from a fixed array inside the library instead of a
caller workspace; its results must be those of wrf_bin.

Kept in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    from paper_2506_12787_b300 import _lib, build
    build.build()
    return _lib.load()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    """Too large a request fails on the host, before any CUDA call."""
    from paper_2506_12787_b300 import _lib, api
    g = api.make_grid(90, 360, 16, 16, 9.0)
    assert lib.wrf_bin_workspace_size(200000, 1024, C.byref(g)) > (4 << 20)
    st = lib.wrf_bin_noalloc(None, 200000, 1024, C.byref(g), None, 0, None, None, None)
    assert st == _lib.WRF_EINVAL
    assert b"scratch" in lib.wrf_last_error()


@pytest.mark.gpu
def test_noalloc_matches_wrf_bin_twice(lib):
    """Two calls in a row through the C ABI give exactly wrf_bin's key lists
    (integer work: bit-exact), including the key count and tile offsets."""
    import torch
    from paper_2506_12787_b300 import _lib, api
    H, W, tw, th = 90, 360, 16, 16
    Q, N = 8, 5000
    dev = torch.device("cuda:0")
    rec = torch.as_tensor(synth.random_rects_records(Q, N, H, W, r_max=30, seed=31), device=dev)
    g = api.make_grid(H, W, tw, th, 9.0)
    T = api.tiles_of(g)
    ws_need = lib.wrf_bin_workspace_size(N, Q, C.byref(g))
    assert 0 < ws_need <= (4 << 20)
    cap = Q * N * 40
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def outputs():
        return (torch.zeros(cap, dtype=torch.int32, device=dev),
                torch.zeros(1, dtype=torch.int64, device=dev),
                torch.zeros(Q * T + 1, dtype=torch.int32, device=dev))

    gids0, nk0, off0 = outputs()
    ws = torch.empty(ws_need, dtype=torch.uint8, device=dev)
    _lib.check(lib.wrf_bin(C.c_void_p(rec.data_ptr()), N, Q, C.byref(g),
                           C.c_void_p(gids0.data_ptr()), cap, C.c_void_p(nk0.data_ptr()),
                           C.c_void_p(off0.data_ptr()), C.c_void_p(ws.data_ptr()), ws_need,
                           stream))
    for call in range(2):
        gids, nk, off = outputs()
        _lib.check(lib.wrf_bin_noalloc(C.c_void_p(rec.data_ptr()), N, Q, C.byref(g),
                                       C.c_void_p(gids.data_ptr()), cap,
                                       C.c_void_p(nk.data_ptr()), C.c_void_p(off.data_ptr()),
                                       stream))
        torch.cuda.synchronize()
        k = int(nk0.item())
        assert k > 0 and int(nk.item()) == k, call
        assert torch.equal(off, off0), call
        assert torch.equal(gids[:k], gids0[:k]), call
    assert api.wrf_status_read() == 0


@pytest.mark.gpu
def test_noalloc_allocates_nothing(lib):
    """After a first (warm-up) call, further calls change neither torch's
    allocator statistics nor the device's free memory."""
    import torch
    from paper_2506_12787_b300 import _lib, api
    H, W, Q, N = 90, 360, 4, 3000
    dev = torch.device("cuda:0")
    rec = torch.as_tensor(synth.random_rects_records(Q, N, H, W, r_max=30, seed=32), device=dev)
    g = api.make_grid(H, W, 16, 16, 9.0)
    T = api.tiles_of(g)
    cap = Q * N * 40
    gids = torch.zeros(cap, dtype=torch.int32, device=dev)
    nk = torch.zeros(1, dtype=torch.int64, device=dev)
    off = torch.zeros(Q * T + 1, dtype=torch.int32, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        _lib.check(lib.wrf_bin_noalloc(C.c_void_p(rec.data_ptr()), N, Q, C.byref(g),
                                       C.c_void_p(gids.data_ptr()), cap,
                                       C.c_void_p(nk.data_ptr()), C.c_void_p(off.data_ptr()),
                                       stream))
        torch.cuda.synchronize()

    call()  # warm-up: the first call in a context looks up the scratch address
    alloc0 = torch.cuda.memory_allocated(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert free1 == free0, (free0, free1)
    assert int(nk.item()) > 0
