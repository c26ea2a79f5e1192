"""Python binding of the C ABI: the same entry points, taking torch tensors.

PyTorch supplies device memory and streams only; every step of the path runs
in the library's CUDA kernels.  Functions return their outputs as tensors
(allocated with torch when not passed in) and raise WrfError on a non-OK
status.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math

import numpy as np
import torch

from . import _lib
from ._lib import WRF_BF16, WRF_BF16X3, WRF_FP32, WrfError

__all__ = ["DeviceScene", "DeviceMLP", "make_grid", "wrf_deform", "wrf_project",
           "wrf_deform_project", "wrf_bin", "wrf_render", "wrf_render_backward",
           "wrf_project_backward", "wrf_deform_backward", "wrf_status_read", "tiles_of",
           "Renderer", "WrfError", "WRF_FP32", "WRF_BF16", "WRF_BF16X3", "wrf_rssi", "wrf_loss", "wrf_adam", "wrf_render_complex", "alloc_records", "record_tail",
           "DevicePaperScene", "DevicePaperMLP", "wrf_paper_deform_project",
           "wrf_measure_alu_peaks", "wrf_deform_acts", "wrf_anneal_tx"]


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream)


def _f32(a, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float32).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)


@dataclasses.dataclass
class DeviceScene:
    """Reference-frame Gaussians resident on the device (FP32, SoA)."""
    mean: torch.Tensor           # [N,2]
    log_scale: torch.Tensor      # [N,2]
    rot: torch.Tensor            # [N]
    opacity_logit: torch.Tensor  # [N]
    amp: torch.Tensor            # [N], or [N,2]: real and imaginary amplitude

    @classmethod
    def from_host(cls, s, device="cuda"):
        return cls(*(_f32(getattr(s, k), device) for k in
                     ("mean", "log_scale", "rot", "opacity_logit", "amp")))

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @property
    def channels(self) -> int:
        return 2 if self.amp.dim() == 2 else 1

    def c(self) -> _lib.Scene:
        return _lib.Scene(self.n, self.channels, self.mean.data_ptr(), self.log_scale.data_ptr(),
                          self.rot.data_ptr(), self.opacity_logit.data_ptr(),
                          self.amp.data_ptr())


def alloc_records(Q: int, n: int, channels: int, device):
    """Record buffer [Q,N,8]; with 2 channels the view of a Q*N*9-float
    buffer whose last Q*N floats hold the imaginary weights."""
    if channels == 1:
        return torch.empty((Q, n, 8), dtype=torch.float32, device=device)
    return torch.empty(Q * n * 9, dtype=torch.float32, device=device)[: Q * n * 8].view(Q, n, 8)


def record_tail(rec, Q: int, n: int):
    """The imaginary weights [Q,N] that follow a 2-channel record buffer."""
    base = rec.reshape(-1)
    return torch.as_strided(base, (Q, n), (n, 1), base.storage_offset() + Q * n * 8)


@dataclasses.dataclass
class DeviceMLP:
    """Deformation MLP weights resident on the device (FP32 masters)."""
    W: list
    b: list
    L_mean: int = 6
    L_tx: int = 10
    room_min: tuple = (0.0, 0.0, 0.0)
    room_size: tuple = (5.0, 5.0, 3.0)
    precision: int = WRF_FP32

    @classmethod
    def from_host(cls, m, device="cuda", precision=WRF_FP32):
        return cls([_f32(w, device) for w in m.W], [_f32(b, device) for b in m.b], m.L_mean,
                   m.L_tx, tuple(m.room_min), tuple(m.room_size), precision)

    @property
    def dims(self):
        return [int(self.W[0].shape[1])] + [int(w.shape[0]) for w in self.W]

    def with_precision(self, precision):
        return dataclasses.replace(self, precision=precision)

    def c(self) -> _lib.Mlp:
        m = _lib.Mlp()
        m.n_layers = len(self.W)
        for i, d in enumerate(self.dims):
            m.dims[i] = d
        for i, (w, b) in enumerate(zip(self.W, self.b)):
            m.W[i] = w.data_ptr()
            m.b[i] = b.data_ptr()
        m.L_mean, m.L_tx = self.L_mean, self.L_tx
        for i in range(3):
            m.room_min[i] = self.room_min[i]
            m.room_size[i] = self.room_size[i]
        m.precision = self.precision
        return m


def make_grid(H=90, W=360, tile_w=16, tile_h=16, q_cut=9.0, wrap=False, px_per_thread=0,
              batch_factor=0, tma_staging=0) -> _lib.Grid:
    """Spectrum grid; wrap=True makes the azimuth axis periodic (0 = 360 degrees).
    px_per_thread (2 or 4), batch_factor (1 or 2) and tma_staging (0: per-thread
    cp.async, 1: TMA gathers) are the rasteriser's launch knobs (0 = defaults)."""
    return _lib.Grid(H, W, tile_w, tile_h, float(q_cut), int(bool(wrap)), int(px_per_thread),
                     int(batch_factor), int(tma_staging))


def tiles_of(grid) -> int:
    return ((grid.W + grid.tile_w - 1) // grid.tile_w) * ((grid.H + grid.tile_h - 1) // grid.tile_h)


def _ws(nbytes, device):
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def wrf_deform(scene: DeviceScene, mlp: DeviceMLP, grid, tx, resid=None, ws=None, stream=None):
    """Residuals [Q,N,5] (Eq. 14)."""
    L = _lib.load()
    Q, dev = int(tx.shape[0]), tx.device
    mc = mlp.c()
    if resid is None:
        resid = torch.empty((Q, scene.n, 5), dtype=torch.float32, device=dev)
    need = L.wrf_deform_workspace_size(scene.n, Q, C.byref(mc))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_deform(C.byref(scene.c()), C.byref(mc), C.byref(grid), _p(tx), Q, _p(resid),
                            _p(ws), ws.numel(), _stream(stream)))
    return resid


def wrf_deform_acts(scene: DeviceScene, mlp: DeviceMLP, grid, tx, resid=None, acts=None, ws=None,
                    stream=None):
    """Residuals [Q,N,5] and the hidden activations [n_layers-1, Q*N, 128]
    (FP32 MLP) saved for wrf_deform_backward."""
    L = _lib.load()
    Q, dev = int(tx.shape[0]), tx.device
    mc = mlp.c()
    if resid is None:
        resid = torch.empty((Q, scene.n, 5), dtype=torch.float32, device=dev)
    if acts is None:
        acts = torch.empty((len(mlp.W) - 1, Q * scene.n, 128), dtype=torch.float32, device=dev)
    need = L.wrf_deform_workspace_size(scene.n, Q, C.byref(mc))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_deform_acts(C.byref(scene.c()), C.byref(mc), C.byref(grid), _p(tx), Q,
                                 _p(resid), _p(acts), _p(ws), ws.numel(), _stream(stream)))
    return resid, acts


def wrf_project(scene: DeviceScene, resid, Q: int, grid, rec=None, tile_count=None, stream=None):
    """Records [Q,N,8] and tile counts [Q,N] (Eq. 12-13)."""
    L = _lib.load()
    dev = scene.mean.device
    if rec is None:
        rec = alloc_records(Q, scene.n, scene.channels, dev)
    if tile_count is None:
        tile_count = torch.empty((Q, scene.n), dtype=torch.int32, device=dev)
    _lib.check(L.wrf_project(C.byref(scene.c()), _p(resid), Q, C.byref(grid), _p(rec),
                             _p(tile_count), _stream(stream)))
    return rec, tile_count


def wrf_deform_project(scene: DeviceScene, mlp: DeviceMLP, grid, tx, rec=None, tile_count=None,
                       ws=None, stream=None):
    L = _lib.load()
    Q, dev = int(tx.shape[0]), tx.device
    mc = mlp.c()
    if rec is None:
        rec = alloc_records(Q, scene.n, scene.channels, dev)
    need = L.wrf_deform_workspace_size(scene.n, Q, C.byref(mc))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_deform_project(C.byref(scene.c()), C.byref(mc), C.byref(grid), _p(tx), Q,
                                    _p(rec), _p(tile_count), _p(ws), ws.numel(), _stream(stream)))
    return rec, tile_count


@dataclasses.dataclass
class DevicePaperScene:
    """The paper's primitives on the device (Sec. 4.1): raw angular centres,
    Cholesky entries, attenuation logits, complex responses (FP32, SoA)."""
    mu: torch.Tensor          # [N,2]
    chol: torch.Tensor        # [N,3]
    attn_logit: torch.Tensor  # [N]
    psi: torch.Tensor         # [N,2]

    @classmethod
    def from_host(cls, s, device="cuda"):
        return cls(*(_f32(getattr(s, k), device) for k in ("mu", "chol", "attn_logit", "psi")))

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    channels = 2

    def c(self) -> _lib.PaperScene:
        return _lib.PaperScene(self.n, self.mu.data_ptr(), self.chol.data_ptr(),
                               self.attn_logit.data_ptr(), self.psi.data_ptr())


@dataclasses.dataclass
class DevicePaperMLP:
    """The paper's deformation network (Sec. 6.1: hidden layers with a skip
    every two layers, outputs dmu, dpsi, ddelta), FP32 on the device."""
    W: list
    b: list
    L_mean: int = 10
    L_tx: int = 6
    room_min: tuple = (0.0, 0.0, 0.0)
    room_size: tuple = (5.0, 5.0, 3.0)
    precision: int = WRF_FP32

    @classmethod
    def from_host(cls, m, device="cuda", precision=WRF_FP32):
        return cls([_f32(w, device) for w in m.W], [_f32(b, device) for b in m.b], m.L_mean,
                   m.L_tx, tuple(m.room_min), tuple(m.room_size), precision)

    def c(self) -> _lib.PaperMlp:
        m = _lib.PaperMlp()
        m.n_hidden = len(self.W) - 1
        m.width = int(self.W[0].shape[0])
        for i, (w, b) in enumerate(zip(self.W, self.b)):
            m.W[i] = w.data_ptr()
            m.b[i] = b.data_ptr()
        m.L_mean, m.L_tx = self.L_mean, self.L_tx
        for i in range(3):
            m.room_min[i] = self.room_min[i]
            m.room_size[i] = self.room_size[i]
        m.precision = self.precision
        return m


def wrf_paper_deform_project(scene: DevicePaperScene, mlp, grid, tx, rec=None, ws=None,
                             stream=None):
    """Two-channel records [Q,N,8] (+ imaginary tail) of the paper's head;
    mlp None: no deformation."""
    L = _lib.load()
    Q, dev = int(tx.shape[0]), scene.mu.device
    if rec is None:
        rec = alloc_records(Q, scene.n, 2, dev)
    if mlp is not None and ws is None:
        ws = _ws(L.wrf_paper_workspace_size(scene.n, Q), dev)
    mc = None if mlp is None else mlp.c()
    _lib.check(L.wrf_paper_deform_project(C.byref(scene.c()), None if mc is None else C.byref(mc),
                                          C.byref(grid), _p(tx), Q, _p(rec), _p(ws),
                                          0 if ws is None else ws.numel(), _stream(stream)))
    return rec


def wrf_measure_alu_peaks(stream=None):
    """(FP32 FLOP/s with fma, FP32 FLOP/s with fma.rn.f32x2, MUFU ex2 per second)
    of the current device, measured by the library's probe kernels."""
    L = _lib.load()
    out = [C.c_double(0.0) for _ in range(3)]
    _lib.check(L.wrf_measure_alu_peaks(*(C.byref(o) for o in out), _stream(stream)))
    return tuple(o.value for o in out)


def wrf_loss(pred, target, lambda1: float = 0.7, want_grad: bool = True, out=None, d_pred=None,
             ws=None, stream=None):
    """Eq. 16 loss over a batch of maps [Q,H,W]: out [1+Q] = (L, SSIM_q...) and,
    if want_grad, d_pred = dL/dpred [Q,H,W]."""
    L = _lib.load()
    Q, H, W = (int(v) for v in pred.shape)
    dev = pred.device
    if out is None:
        out = torch.empty(1 + Q, dtype=torch.float32, device=dev)
    if want_grad and d_pred is None:
        d_pred = torch.empty_like(pred)
    ws = _ws(L.wrf_loss_workspace_size(Q, H, W), dev) if ws is None else ws
    _lib.check(L.wrf_loss(_p(pred), _p(target), Q, H, W, float(lambda1), _p(out),
                          _p(d_pred) if want_grad else None, _p(ws), ws.numel(), _stream(stream)))
    return out, (d_pred if want_grad else None)


def wrf_adam(groups, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None):
    """One Adam step; groups = [(param, grad, m, v, lr), ...] of contiguous FP32
    device tensors (m, v: optimizer state, zero before step 1)."""
    L = _lib.load()
    arr = (_lib.AdamGroup * len(groups))()
    for i, (p, g, m, v, lr) in enumerate(groups):
        for t in (p, g, m, v):
            assert t.is_contiguous() and t.dtype == torch.float32 and t.numel() == p.numel()
        arr[i] = _lib.AdamGroup(_p(p), _p(g), _p(m), _p(v), p.numel(), float(lr))
    _lib.check(L.wrf_adam(arr, len(groups), int(step), float(beta1), float(beta2), float(eps),
                          _stream(stream)))


def wrf_anneal_tx(tx, normals, iteration: int, gamma: float, tau: int, room_size, idx=None,
                  n_positions=None, out=None, stream=None):
    """Eq. 17-18: TX positions (tx[idx] or tx) plus the anneal-smoothing noise
    of fine-stage iteration `iteration`, in metres ([Q,3] FP32 device)."""
    L = _lib.load()
    Q = int(normals.shape[0])
    if out is None:
        out = torch.empty((Q, 3), dtype=torch.float32, device=normals.device)
    if idx is not None:
        idx = idx.to(device=normals.device, dtype=torch.int32).contiguous()
    ns = int(tx.shape[0]) if n_positions is None else int(n_positions)
    room = (C.c_float * 3)(*[float(v) for v in room_size])
    _lib.check(L.wrf_anneal_tx(_p(tx), _p(idx), ns, _p(normals), Q, int(iteration), float(gamma),
                               int(tau), room, _p(out), _stream(stream)))
    return out


def wrf_rssi(scene: DeviceScene, mlp: DeviceMLP, grid, tx, rssi=None, map_out=None, ws=None,
             stream=None):
    """RSSI head (Sec. 7.2): pooled map magnitude per query, rssi [Q]; the
    un-pooled maps go to map_out [Q,H,W] when it is given."""
    L = _lib.load()
    Q, dev = int(tx.shape[0]), tx.device
    mc = mlp.c()
    if rssi is None:
        rssi = torch.empty(Q, dtype=torch.float32, device=dev)
    need = L.wrf_deform_workspace_size(scene.n, Q, C.byref(mc))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_rssi(C.byref(scene.c()), C.byref(mc), C.byref(grid), _p(tx), Q, _p(rssi),
                          _p(map_out), _p(ws), ws.numel(), _stream(stream)))
    return rssi


def wrf_bin(rec, n: int, Q: int, grid, key_capacity: int, gids=None, n_keys=None, offsets=None,
            ws=None, stream=None):
    """Tile lists: gids [cap] (uint32 stored as int32), n_keys [1] int64, offsets [Q*T+1]."""
    L = _lib.load()
    dev = rec.device
    T = tiles_of(grid)
    if gids is None:
        gids = torch.empty(max(int(key_capacity), 1), dtype=torch.int32, device=dev)
    if n_keys is None:
        n_keys = torch.empty(1, dtype=torch.int64, device=dev)
    if offsets is None:
        offsets = torch.empty(Q * T + 1, dtype=torch.int32, device=dev)
    need = L.wrf_bin_workspace_size(n, Q, C.byref(grid))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_bin(_p(rec), n, Q, C.byref(grid), _p(gids), int(key_capacity), _p(n_keys),
                         _p(offsets), _p(ws), ws.numel(), _stream(stream)))
    return gids, n_keys, offsets


def wrf_render(rec, gids, offsets, n_keys, key_capacity: int, n: int, Q: int, grid, out=None,
               stream=None):
    L = _lib.load()
    if out is None:
        out = torch.empty((Q, grid.H, grid.W), dtype=torch.float32, device=offsets.device)
    _lib.check(L.wrf_render(_p(rec), _p(gids), _p(offsets), _p(n_keys), int(key_capacity), n, Q,
                            C.byref(grid), _p(out), _stream(stream)))
    return out


def wrf_render_complex(rec, gids, offsets, n_keys, key_capacity: int, n: int, Q: int, grid,
                       out=None, stream=None):
    """Two channels: out [Q,2,H,W] = magnitude, phase (records with their tail)."""
    L = _lib.load()
    if out is None:
        out = torch.empty((Q, 2, grid.H, grid.W), dtype=torch.float32, device=offsets.device)
    _lib.check(L.wrf_render_complex(_p(rec), _p(gids), _p(offsets), _p(n_keys), int(key_capacity),
                                    n, Q, C.byref(grid), _p(out), _stream(stream)))
    return out


def wrf_render_backward(rec, gids, offsets, n_keys, key_capacity: int, n: int, Q: int, grid,
                        dA, d_rec=None, stream=None):
    L = _lib.load()
    if d_rec is None:
        d_rec = torch.zeros((Q, n, 6), dtype=torch.float32, device=dA.device)
    _lib.check(L.wrf_render_backward(_p(rec), _p(gids), _p(offsets), _p(n_keys),
                                     int(key_capacity), n, Q, C.byref(grid), _p(dA.contiguous()),
                                     _p(d_rec), _stream(stream)))
    return d_rec


def wrf_project_backward(scene: DeviceScene, resid, Q: int, d_rec, d_resid=None, stream=None):
    L = _lib.load()
    dev, N = scene.mean.device, scene.n
    if d_resid is None and resid is not None:
        d_resid = torch.empty((Q, N, 5), dtype=torch.float32, device=dev)
    g = dict(d_mean=torch.empty((N, 2), device=dev), d_log_scale=torch.empty((N, 2), device=dev),
             d_rot=torch.empty(N, device=dev), d_opacity=torch.empty(N, device=dev),
             d_amp=torch.empty(N, device=dev))
    _lib.check(L.wrf_project_backward(C.byref(scene.c()), _p(resid), Q, _p(d_rec), _p(d_resid),
                                      _p(g["d_mean"]), _p(g["d_log_scale"]), _p(g["d_rot"]),
                                      _p(g["d_opacity"]), _p(g["d_amp"]), _stream(stream)))
    g["d_resid"] = d_resid
    return g


def wrf_deform_backward(scene: DeviceScene, mlp: DeviceMLP, grid, tx, d_resid, d_mean=None,
                        stop_grad_mean=False, ws=None, stream=None, acts=None):
    """dW, db (lists) and d_mean accumulated through gamma(mean) (unless stopped);
    acts: the activations saved by wrf_deform_acts (else recomputed)."""
    L = _lib.load()
    dev, Q = tx.device, int(tx.shape[0])
    mc = mlp.c()
    dW = [torch.empty_like(w) for w in mlp.W]
    db = [torch.empty_like(b) for b in mlp.b]
    if d_mean is None:
        d_mean = torch.zeros((scene.n, 2), dtype=torch.float32, device=dev)
    arr = C.c_void_p * len(dW)
    pW = arr(*[w.data_ptr() for w in dW])
    pb = arr(*[b.data_ptr() for b in db])
    need = L.wrf_deform_backward_workspace_size(scene.n, Q, C.byref(mc))
    ws = _ws(need, dev) if ws is None else ws
    _lib.check(L.wrf_deform_backward(C.byref(scene.c()), C.byref(mc), C.byref(grid), _p(tx), Q,
                                     _p(d_resid), _p(acts), pW, pb, _p(d_mean),
                                     int(bool(stop_grad_mean)),
                                     _p(ws), ws.numel(), _stream(stream)))
    return dW, db, d_mean


def wrf_status_read(stream=None) -> int:
    """First device-side status recorded since the last read (synchronises)."""
    return int(_lib.load().wrf_status_read(_stream(stream)))


class Renderer:
    """The forward path (deform+project -> bin -> render) with reusable
    workspaces and a key capacity that grows when binning reports overflow.

    The tile lists and records of the last call are kept for the backward.
    """

    def __init__(self, grid, device="cuda", key_capacity: int = 0, fused: bool = True):
        self.grid = grid
        self.device = torch.device(device)
        self.cap = int(key_capacity)
        self.fused = fused
        self._ws = {}
        self._nk_host = None   # pinned key count of a deferred binning
        self._pending = None   # (event, capacity, stream) of a deferred binning

    def _buf(self, name, nbytes):
        b = self._ws.get(name)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
            self._ws[name] = b
        return b

    def _tensor(self, name, shape, dtype):
        numel = int(np.prod(shape))
        nbytes = numel * torch.empty((), dtype=dtype).element_size()
        return self._buf(name, nbytes)[:nbytes].view(dtype)[:numel].view(shape)

    def project(self, scene: DeviceScene, mlp, tx, stream=None, acts=None):
        """Records (and residuals on the unfused path); acts, a tensor
        [n_layers-1, Q*N, 128], receives the hidden activations (unfused,
        FP32 MLP) for the backward."""
        L = _lib.load()
        Q = int(tx.shape[0])
        # 2 channels: the imaginary weights follow the Q x N records
        buf = self._buf("rec", Q * scene.n * (8 + (scene.channels == 2)) * 4)
        rec = buf[: Q * scene.n * 32].view(torch.float32).view(Q, scene.n, 8)
        if mlp is None:
            wrf_project(scene, None, Q, self.grid, rec=rec, tile_count=None, stream=stream)
            return rec, None
        mc = mlp.c()
        ws = self._buf("dws", L.wrf_deform_workspace_size(scene.n, Q, C.byref(mc)))
        if self.fused:
            wrf_deform_project(scene, mlp, self.grid, tx, rec=rec, ws=ws, stream=stream)
            return rec, None
        resid = self._tensor("resid", (Q, scene.n, 5), torch.float32)
        if acts is not None:
            wrf_deform_acts(scene, mlp, self.grid, tx, resid=resid, acts=acts, ws=ws, stream=stream)
        else:
            wrf_deform(scene, mlp, self.grid, tx, resid=resid, ws=ws, stream=stream)
        wrf_project(scene, resid, Q, self.grid, rec=rec, tile_count=None, stream=stream)
        return rec, resid

    def bin_and_render(self, rec, n, Q, stream=None, out=None, channels=1, deferred=False):
        """Bins and renders.  The key count is read back (a host sync) and the
        binning repeated with a larger key capacity until the keys fit --
        unless deferred is set and a capacity is known: then one pass runs with
        the current capacity, the key count is copied back asynchronously, and
        the caller must call key_overflow() before using the results (a
        result with too many keys is all zeros and must be recomputed)."""
        L = _lib.load()
        T = tiles_of(self.grid)
        if deferred and self.cap > 0:
            gids = self._tensor("gids", (self.cap,), torch.int32)
            n_keys = self._tensor("nk", (1,), torch.int64)
            offs = self._tensor("offs", (Q * T + 1,), torch.int32)
            bws = self._buf("bws", L.wrf_bin_workspace_size(n, Q, C.byref(self.grid)))
            wrf_bin(rec, n, Q, self.grid, self.cap, gids=gids, n_keys=n_keys, offsets=offs,
                    ws=bws, stream=stream)
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            if self._nk_host is None:
                self._nk_host = torch.zeros(1, dtype=torch.int64, pin_memory=True)
            with torch.cuda.stream(s):
                self._nk_host.copy_(n_keys, non_blocking=True)
                ev = None
                if not torch.cuda.is_current_stream_capturing():
                    # (inside a CUDA-graph capture the caller synchronises
                    # after the replay instead)
                    ev = torch.cuda.Event()
                    ev.record(s)
            self._pending = (ev, self.cap, s)
        else:
            gids, n_keys, offs = self._bin_checked(rec, n, Q, T, stream)
        render = wrf_render_complex if channels == 2 else wrf_render
        out = render(rec, gids, offs, n_keys, self.cap, n, Q, self.grid, out=out, stream=stream)
        self.last = dict(rec=rec, gids=gids, offs=offs, n_keys=n_keys, n=n, Q=Q)
        return out

    def key_overflow(self) -> bool:
        """After a deferred bin_and_render: waits for its key count (the
        binning only, not the rest of the stream) and returns True if the keys
        did not fit -- the capacity has then been raised and the results of
        that call are void.  (A call captured in a CUDA graph is checked with
        replayed_key_overflow after each replay.)"""
        if self._pending is None:
            return False
        ev, cap, s = self._pending
        self._pending = None
        if ev is None:
            return False
        ev.synchronize()
        need = int(self._nk_host[0])
        if need <= cap:
            return False
        wrf_status_read(s)  # clear the recorded overflow
        self.cap = max(self.cap, int(need * 1.25) + 1024)
        return True

    def replayed_key_overflow(self, cap, stream=None) -> bool:
        """key_overflow for a deferred binning captured in a CUDA graph with
        key capacity cap, after the caller has synchronised with the replay."""
        need = int(self._nk_host[0])
        if need <= cap:
            return False
        wrf_status_read(stream)  # clear the recorded overflow
        self.cap = max(self.cap, int(need * 1.25) + 1024)
        return True

    def _bin_checked(self, rec, n, Q, T, stream):
        L = _lib.load()
        if self.cap <= 0:
            self.cap = max(1 << 16, Q * n * 6)
        while True:
            gids = self._tensor("gids", (self.cap,), torch.int32)
            n_keys = self._tensor("nk", (1,), torch.int64)
            offs = self._tensor("offs", (Q * T + 1,), torch.int32)
            bws = self._buf("bws", L.wrf_bin_workspace_size(n, Q, C.byref(self.grid)))
            wrf_bin(rec, n, Q, self.grid, self.cap, gids=gids, n_keys=n_keys, offsets=offs,
                    ws=bws, stream=stream)
            need = int(n_keys.item())
            if need <= self.cap:
                return gids, n_keys, offs
            wrf_status_read(stream)  # clear the recorded overflow
            self.cap = int(need * 1.25) + 1024

    def forward_paper(self, scene: DevicePaperScene, mlp, tx, stream=None, out=None):
        """Magnitude and phase [Q,2,H,W] with the paper's head (Sec. 6.1)."""
        L = _lib.load()
        Q = int(tx.shape[0])
        buf = self._buf("rec", Q * scene.n * 9 * 4)
        rec = buf[: Q * scene.n * 32].view(torch.float32).view(Q, scene.n, 8)
        ws = None if mlp is None else self._buf("pws", L.wrf_paper_workspace_size(scene.n, Q))
        wrf_paper_deform_project(scene, mlp, self.grid, tx, rec=rec, ws=ws, stream=stream)
        out = self.bin_and_render(rec, scene.n, Q, stream=stream, out=out, channels=2)
        self.last["resid"] = None
        return out

    def forward(self, scene: DeviceScene, mlp, tx, stream=None, out=None, acts=None,
                deferred=False):
        """Spectra [Q,H,W] (deferred: see bin_and_render)."""
        Q = int(tx.shape[0])
        rec, resid = self.project(scene, mlp, tx, stream=stream, acts=acts)
        out = self.bin_and_render(rec, scene.n, Q, stream=stream, out=out, channels=scene.channels,
                                  deferred=deferred)
        self.last["resid"] = resid
        return out
