"""Batched spectrum synthesis with preallocated device buffers.

One ``BatchedForward`` holds everything a batch of Q queries over one
resident scene needs (records, tile lists, workspaces, output) so that a
forward is a fixed sequence of library calls on one stream with no host
synchronisation: deform+project (Eq. 12-15) -> bin -> render (Eq. 9/13).
Because nothing is allocated or read back inside ``run``, the sequence can be
captured once into a CUDA graph and replayed.

Key capacity: the number of (query, tile, Gaussian) keys depends on the
queries.  ``reserve`` sizes the capacity from one measured forward plus a
margin; if a later batch needs more, the library records WRF_ENOSPC in its
status word and renders zeros, and ``check`` raises so the caller can
``reserve`` again and rerun (the capacity never shrinks).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from .api import (DeviceMLP, DevicePaperScene, DeviceScene, _p, _stream, tiles_of, wrf_bin,
                  wrf_deform_project, wrf_paper_deform_project, wrf_render, wrf_render_complex,
                  wrf_status_read, alloc_records)


class BatchedForward:
    def __init__(self, scene: DeviceScene, mlp: DeviceMLP, grid, Q: int, device="cuda",
                 key_capacity: int = 0, margin: float = 1.25):
        self.scene, self.mlp, self.grid, self.Q = scene, mlp, grid, int(Q)
        self.device = torch.device(device)
        self.margin = margin
        L = _lib.load()
        n = scene.n
        self.T = tiles_of(grid)
        self._mc = mlp.c()
        self.channels = scene.channels
        self.rec = alloc_records(self.Q, n, self.channels, self.device)
        self.dws = torch.empty(max(256, L.wrf_deform_workspace_size(n, self.Q, C.byref(self._mc))),
                               dtype=torch.uint8, device=self.device)
        self.bws = torch.empty(max(256, L.wrf_bin_workspace_size(n, self.Q, C.byref(grid))),
                               dtype=torch.uint8, device=self.device)
        self.n_keys = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.offs = torch.empty(self.Q * self.T + 1, dtype=torch.int32, device=self.device)
        # one channel: spectra [Q,H,W]; two: [Q,2,H,W] = magnitude, phase
        shape = (self.Q, grid.H, grid.W) if self.channels == 1 else (self.Q, 2, grid.H, grid.W)
        self.out = torch.empty(shape, dtype=torch.float32, device=self.device)
        self.cap = 0
        self.gids = None
        self._alloc_keys(int(key_capacity))

    # kernels one run() launches: prep (encodings, per-query terms and
    # weight images in one launch), MLP; bin count, scan reduce, scan top,
    # scan down-sweep, scatter; render
    launches_per_run = 8

    def _alloc_keys(self, cap: int):
        cap = max(int(cap), 1024)
        if cap > self.cap:
            self.gids = torch.empty(cap, dtype=torch.int32, device=self.device)
            self.cap = cap

    def deform_project(self, tx, stream=None):
        wrf_deform_project(self.scene, self.mlp, self.grid, tx, rec=self.rec, ws=self.dws,
                           stream=stream)

    def bin(self, stream=None):
        wrf_bin(self.rec, self.scene.n, self.Q, self.grid, self.cap, gids=self.gids,
                n_keys=self.n_keys, offsets=self.offs, ws=self.bws, stream=stream)

    def render(self, stream=None, out=None):
        render = wrf_render_complex if self.channels == 2 else wrf_render
        return render(self.rec, self.gids, self.offs, self.n_keys, self.cap, self.scene.n,
                          self.Q, self.grid, out=self.out if out is None else out, stream=stream)

    def run(self, tx, stream=None, out=None):
        """Enqueue one forward for tx [Q,3] (device) on `stream`; no sync."""
        assert tx.shape[0] == self.Q
        self.deform_project(tx, stream)
        self.bin(stream)
        return self.render(stream, out)

    def reserve(self, tx, stream=None) -> int:
        """Run once, read the key count and grow the capacity to count*margin."""
        self.run(tx, stream)
        st = stream or torch.cuda.current_stream()
        st.synchronize()
        need = int(self.n_keys.item())
        wrf_status_read(stream)  # clear an overflow recorded by this sizing run
        if need > self.cap:
            self._alloc_keys(int(need * self.margin) + 1024)
            self.run(tx, stream)
            st.synchronize()
        return need

    def check(self, stream=None):
        """Raise WrfError if the device recorded an error (e.g. key overflow)."""
        s = wrf_status_read(stream)
        if s != 0:
            raise _lib.WrfError(s, f"device status (n_keys={int(self.n_keys.item())}, "
                                   f"capacity={self.cap})")

    def graph(self, tx, stream=None, out=None):
        """Capture run(tx) into a CUDA graph (tx, and out if given, must stay
        at the same addresses)."""
        g = torch.cuda.CUDAGraph()
        s = stream or torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(tx, s, out)  # warm the path on the capture stream
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g, stream=s):
            self.run(tx, s, out)
        return g


class PaperForward(BatchedForward):
    """BatchedForward for the paper's own head (Sec. 4.1-4.2, 6.1): the
    tanh-mapped, Cholesky-parameterised scene (DevicePaperScene) through the
    skip network (DevicePaperMLP, or None for no deformation) into
    two-channel records, then the same binning and the two-channel render;
    out [Q,2,H,W] = magnitude, phase.  Same buffers, key-capacity protocol
    and graph capture as BatchedForward, so HostPipeline drives it too."""

    def __init__(self, scene: DevicePaperScene, mlp, grid, Q: int, device="cuda",
                 key_capacity: int = 0, margin: float = 1.25):
        self.scene, self.mlp, self.grid, self.Q = scene, mlp, grid, int(Q)
        self.device = torch.device(device)
        self.margin = margin
        L = _lib.load()
        n = scene.n
        self.T = tiles_of(grid)
        self.channels = 2
        self.rec = alloc_records(self.Q, n, 2, self.device)
        self.dws = None if mlp is None else torch.empty(
            max(256, L.wrf_paper_workspace_size(n, self.Q)), dtype=torch.uint8, device=self.device)
        self.bws = torch.empty(max(256, L.wrf_bin_workspace_size(n, self.Q, C.byref(grid))),
                               dtype=torch.uint8, device=self.device)
        self.n_keys = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.offs = torch.empty(self.Q * self.T + 1, dtype=torch.int32, device=self.device)
        self.out = torch.empty((self.Q, 2, grid.H, grid.W), dtype=torch.float32,
                               device=self.device)
        self.cap = 0
        self.gids = None
        self._alloc_keys(int(key_capacity))
        net = 1 if mlp is None else (2 if mlp.precision in (_lib.WRF_BF16, _lib.WRF_BF16X3)
                                     else 4)
        self.launches_per_run = net + 6

    # kernels one run() launches, set in __init__: the network's (tensor
    # cores: one prep launch and the network; FP32: encodings, per-query
    # terms, weights and the network; no network: the projection alone),
    # binning's five, render
    launches_per_run = 8

    def deform_project(self, tx, stream=None):
        wrf_paper_deform_project(self.scene, self.mlp, self.grid, tx, rec=self.rec, ws=self.dws,
                                 stream=stream)


class MultiSceneForward:
    """One launch sequence over a batch of up to Q queries of several
    resident scenes (each its own Gaussians and BF16 deformation network).

    The scene set is prepared once (per-scene gamma(mean) rows and weight
    images on the device); a batch is the device buffers scene_of [Q]
    (int32; -1 for an unused slot, which renders zeros) and tx [Q,3].  The
    record offsets of the queries are computed on the device, so one captured
    graph serves every mix of scenes.  A query's spectrum equals the spectrum
    of the same query run alone through BatchedForward of its scene."""

    # kernels one run() launches: setup, per-query term, MLP; binning's five;
    # render
    launches_per_run = 9

    def __init__(self, scenes, mlps, grid, Q: int, device="cuda", key_capacity: int = 0,
                 margin: float = 1.25, rec_capacity: int | None = None):
        assert len(scenes) == len(mlps) and 1 <= len(scenes) <= 16
        self.scenes, self.mlps, self.grid, self.Q = list(scenes), list(mlps), grid, int(Q)
        self.device = torch.device(device)
        self.margin = margin
        L = _lib.load()
        S = len(scenes)
        self.S = S
        self._sc = (_lib.Scene * S)(*[sc.c() for sc in scenes])
        self._mc = (_lib.Mlp * S)(*[m.c() for m in mlps])
        nset = L.wrf_multi_set_size(self._sc, self._mc, S)
        if nset == 0:
            raise _lib.WrfError(_lib.WRF_EINVAL, L.wrf_last_error().decode())
        self.set = torch.empty(nset, dtype=torch.uint8, device=self.device)
        _lib.check(L.wrf_multi_set_prepare(self._sc, self._mc, S, C.byref(grid),
                                           _p(self.set), nset, _stream(None)))
        self.n_max = max(sc.n for sc in scenes)
        self.rec_cap = int(rec_capacity) if rec_capacity is not None else self.Q * self.n_max
        self.rec = torch.empty((max(self.rec_cap, 1), 8), dtype=torch.float32, device=self.device)
        self.qbase = torch.zeros(self.Q + 1, dtype=torch.int64, device=self.device)
        self.scene_of = torch.full((self.Q,), -1, dtype=torch.int32, device=self.device)
        self.tx = torch.zeros((self.Q, 3), dtype=torch.float32, device=self.device)
        self.mws = torch.empty(max(256, L.wrf_multi_workspace_size(self.Q)), dtype=torch.uint8,
                               device=self.device)
        self.bws = torch.empty(max(256, L.wrf_bin_workspace_size(self.n_max, self.Q,
                                                                 C.byref(grid))),
                               dtype=torch.uint8, device=self.device)
        self.T = tiles_of(grid)
        self.n_keys = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.offs = torch.empty(self.Q * self.T + 1, dtype=torch.int32, device=self.device)
        self.out = torch.empty((self.Q, grid.H, grid.W), dtype=torch.float32, device=self.device)
        self.cap = 0
        self.gids = None
        self._alloc_keys(int(key_capacity))

    def _alloc_keys(self, cap: int):
        cap = max(int(cap), 1024)
        if cap > self.cap:
            self.gids = torch.empty(cap, dtype=torch.int32, device=self.device)
            self.cap = cap

    def set_batch(self, scene_of, tx):
        """Copy a batch (scene indices [<=Q], TX [<=Q,3]) into the device
        buffers; slots past it are unused (-1)."""
        k = int(len(scene_of))
        self.scene_of.fill_(-1)
        self.scene_of[:k].copy_(torch.as_tensor(scene_of, dtype=torch.int32), non_blocking=True)
        self.tx[:k].copy_(torch.as_tensor(tx, dtype=torch.float32), non_blocking=True)

    def run(self, stream=None, out=None):
        """Enqueue one forward of the batch in scene_of / tx on `stream`."""
        L = _lib.load()
        st = _stream(stream)
        _lib.check(L.wrf_deform_project_multi(
            self._sc, self._mc, self.S, _p(self.set), _p(self.scene_of), _p(self.tx), self.Q,
            C.byref(self.grid), _p(self.rec), self.rec_cap, _p(self.qbase), _p(self.mws),
            self.mws.numel(), st))
        _lib.check(L.wrf_bin_multi(_p(self.rec), _p(self.qbase), self.n_max, self.Q,
                                   C.byref(self.grid), _p(self.gids), self.cap, _p(self.n_keys),
                                   _p(self.offs), _p(self.bws), self.bws.numel(), st))
        out = self.out if out is None else out
        _lib.check(L.wrf_render_multi(_p(self.rec), _p(self.qbase), _p(self.gids), _p(self.offs),
                                      _p(self.n_keys), self.cap, self.Q, C.byref(self.grid),
                                      _p(out), st))
        return out

    def reserve(self, stream=None) -> int:
        """Run the current batch once and grow the key capacity to the
        count it needs times the margin."""
        self.run(stream)
        st = stream or torch.cuda.current_stream()
        st.synchronize()
        need = int(self.n_keys.item())
        wrf_status_read(stream)
        if need > self.cap:
            self._alloc_keys(int(need * self.margin) + 1024)
            self.run(stream)
            st.synchronize()
        return need

    def check(self, stream=None):
        s = wrf_status_read(stream)
        if s != 0:
            raise _lib.WrfError(s, f"device status (n_keys={int(self.n_keys.item())}, "
                                   f"capacity={self.cap})")

    def graph(self, stream=None, out=None):
        """Capture run() into a CUDA graph: it reads whatever batch scene_of /
        tx hold at replay."""
        g = torch.cuda.CUDAGraph()
        s = stream or torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(s, out)
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g, stream=s):
            self.run(s, out)
        return g


class HostPipeline:
    """Spectra for TX batches held in host memory, with the copies overlapped
    with compute: step i's TX upload and forward run on the compute stream
    into device buffer i % 2 while step i-1's spectra are read back to pinned
    host memory on a copy stream.  Each of the two buffer sets has its own
    captured graph.  Results land in a ring of two pinned host buffers: a
    step's spectra are valid until the step two later completes."""

    def __init__(self, fw: BatchedForward):
        self.fw = fw
        dev = fw.device
        self.compute = torch.cuda.Stream(device=dev)
        self.copy = torch.cuda.Stream(device=dev)
        self.tx_dev = [torch.zeros((fw.Q, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        self.out_dev = [fw.out, torch.empty_like(fw.out)]
        self.out_host = [torch.empty(tuple(fw.out.shape), dtype=torch.float32).pin_memory()
                         for _ in range(2)]
        self.graphs = [fw.graph(self.tx_dev[k], self.compute, self.out_dev[k]) for k in range(2)]
        self.done = [torch.cuda.Event() for _ in range(2)]   # forward k finished
        self.freed = [torch.cuda.Event() for _ in range(2)]  # read-back of buffer k finished
        self.i = 0

    @property
    def h2d_bytes(self):
        return self.fw.Q * 3 * 4

    @property
    def d2h_bytes(self):
        return int(self.fw.out.numel()) * 4

    def step(self, tx_host):
        """Enqueue one step for tx_host [Q,3] (pinned FP32); returns the
        pinned host tensor its spectra will land in."""
        k = self.i & 1
        with torch.cuda.stream(self.compute):
            if self.i >= 2:
                self.compute.wait_event(self.freed[k])  # buffer k read back
            self.tx_dev[k].copy_(tx_host, non_blocking=True)
            self.graphs[k].replay()
            self.done[k].record(self.compute)
        with torch.cuda.stream(self.copy):
            self.copy.wait_event(self.done[k])
            self.out_host[k].copy_(self.out_dev[k], non_blocking=True)
            self.freed[k].record(self.copy)
        self.i += 1
        return self.out_host[k]

    def sync(self):
        self.copy.synchronize()
        self.compute.synchronize()


class NativePipeline:
    """The library's host-to-host forward pipeline (wrf_pipeline_*): TX
    positions in host memory in, spectra in pinned host memory out, every
    step's upload, graph replay and read-back issued by the library itself
    (two slots, the read-back of one step overlapping the next step's
    compute; a step whose keys do not fit is recomputed with a grown
    capacity).  This class only marshals arguments and keeps the scene and
    network alive while the pipeline uses them.  ``step`` returns the pinned
    host tensor the step's spectra land in: valid after ``wait`` or once the
    step two later has been issued (two buffers alternate)."""

    def __init__(self, scene: DeviceScene, mlp: DeviceMLP, grid, Q: int, key_margin: float = 0.0):
        self._L = _lib.load()
        self.scene, self.mlp, self.grid, self.Q = scene, mlp, grid, int(Q)
        self._sc, self._mc = scene.c(), mlp.c()
        p = C.c_void_p()
        _lib.check(self._L.wrf_pipeline_create(C.byref(self._sc), C.byref(self._mc),
                                               C.byref(grid), self.Q, float(key_margin),
                                               C.byref(p)))
        self._p = p
        shape = (self.Q, grid.H, grid.W) if scene.channels == 1 else (self.Q, 2, grid.H, grid.W)
        self.out_host = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.i = 0

    @property
    def h2d_bytes(self):
        return self.Q * 3 * 4

    @property
    def d2h_bytes(self):
        return int(self.out_host[0].numel()) * 4

    def step(self, tx_host):
        """Issue one step for tx_host [Q,3] (host FP32, contiguous)."""
        assert tx_host.device.type == "cpu" and tx_host.dtype == torch.float32
        assert tuple(tx_host.shape) == (self.Q, 3) and tx_host.is_contiguous()
        out = self.out_host[self.i & 1]
        _lib.check(self._L.wrf_pipeline_step(self._p, C.c_void_p(tx_host.data_ptr()),
                                             C.c_void_p(out.data_ptr())))
        self.i += 1
        return out

    def wait(self):
        _lib.check(self._L.wrf_pipeline_wait(self._p))

    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            self._L.wrf_pipeline_destroy(self._p)
            self._p = None

    def __del__(self):
        self.close()
