"""FP64 CPU oracle for SwiftWRF spectrum synthesis (arXiv 2506.12787).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or runs
anything in this package.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg use it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
rows); this module loads it with ctypes and converts numpy arrays.  A second,
independent implementation of the rendering sum, ``brute.py``, evaluates every
pixel against every Gaussian with numpy broadcasting; the tests pin the C
oracle to it.

Function -> paper:
  pe            Sec. 4.2 Eq. 15
  deform        Sec. 4.2 Eq. 14 (MLP over [gamma(mean), gamma(tx)])
  project       Sec. 4.1 Eq. 8, Sec. 4.2 Eq. 12-13 (deformed centre/covariance/weight)
  render        Sec. 4.1 Eq. 9, Sec. 4.2 Eq. 13 (order-free truncated sum)
  bin_f32       tile lists, Sec. 4.1 ("spectrum domain partitioned into tiles")
  grad          derivatives of the above (Sec. 4.4 training by back-propagation)
  mlp_grad      the MLP part of grad, with the slack of ReLU decisions that an FP32
                forward may take either way
  wrap          optional azimuth periodicity (0 and W columns the same direction:
                every sum runs over the images mx + m W of each Gaussian, the tile
                lists cover columns modulo W)
  forward_complex  two channels (real and imaginary amplitude): Sec. 6.1 renders
                them as separate channels and decomposes the result into
                magnitude and phase
  rssi          Sec. 7.2 (RSSI head: global average pool of the rendered map) with
                RSSI as the spectrum magnitude averaged over azimuth and elevation
                (Sec. 6.6)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

D = C.POINTER(C.c_double)
F = C.POINTER(C.c_float)
I = C.POINTER(C.c_int)
U32 = C.POINTER(C.c_uint32)
I64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_pe.argtypes = [D, C.c_int, C.c_int, D]
        L.or_deform.argtypes = [C.c_int, D, C.c_int, C.c_int, C.c_int, D, C.c_int, C.c_int, D, D,
                                C.c_int, I, D, D]
        L.or_project.argtypes = [C.c_int, D, D, D, D, D, C.c_int, D, C.c_double, D]
        L.or_project.restype = None
        L.or_render.argtypes = [C.c_int, C.c_int, D, C.c_int, C.c_int, C.c_double, C.c_double,
                                D, D]
        L.or_bin_f32.argtypes = [C.c_int, C.c_int, F, C.c_int, C.c_int, C.c_int, C.c_int, U32,
                                 U32, C.c_int64, I64, U32]
        L.or_render_grad.argtypes = [C.c_int, C.c_int, D, C.c_int, C.c_int, C.c_double, D, D]
        L.or_render_w.argtypes = [C.c_int, C.c_int, D, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.c_int, D, D]
        L.or_bin_f32_w.argtypes = [C.c_int, C.c_int, F, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_int, U32, U32, C.c_int64, I64, U32]
        L.or_render_grad_w.argtypes = [C.c_int, C.c_int, D, C.c_int, C.c_int, C.c_double,
                                       C.c_int, D, D]
        L.or_project_grad.argtypes = [C.c_int, D, D, D, D, C.c_int, D, D, D, D, D, D, D, D]
        L.or_project_grad.restype = None
        L.or_mlp_grad.argtypes = [C.c_int, D, C.c_int, C.c_int, C.c_int, D, C.c_int, C.c_int, D,
                                  D, C.c_int, I, D, D, C.c_int, D, D]
        L.or_mlp_grad_slack.argtypes = [C.c_int, D, C.c_int, C.c_int, C.c_int, D, C.c_int,
                                        C.c_int, D, D, C.c_int, I, D, D, C.c_int, C.c_double, D,
                                        D, D, D]
        L.or_num_threads.argtypes = []
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(D)


def _null(t):
    return C.cast(None, t)


def num_threads() -> int:
    return int(lib().or_num_threads())


def pe(x, L: int) -> np.ndarray:
    """gamma(x) for one vector x (Eq. 15)."""
    x, px = _d(np.atleast_1d(x))
    out = np.zeros(x.shape[0] * (2 * L + 1))
    lib().or_pe(px, x.shape[0], L, out.ctypes.data_as(D))
    return out


def flat_params(mlp) -> tuple:
    """MLP weights -> (dims int array, flat FP64 params [W0, b0, W1, b1, ...])."""
    dims = np.asarray(mlp.dims, dtype=np.int32)
    parts = []
    for W, b in zip(mlp.W, mlp.b):
        parts.append(np.asarray(W, np.float64).ravel())
        parts.append(np.asarray(b, np.float64).ravel())
    return dims, np.concatenate(parts)


def unflat_params(mlp, flat):
    Ws, bs, o = [], [], 0
    for W, b in zip(mlp.W, mlp.b):
        Ws.append(flat[o:o + W.size].reshape(W.shape)); o += W.size
        bs.append(flat[o:o + b.size].reshape(b.shape)); o += b.size
    return Ws, bs


def deform(scene, mlp, tx, H: int, W: int) -> np.ndarray:
    """Residuals [Q,N,out] (Eq. 14), row by row in FP64."""
    mean, pm = _d(scene.mean)
    tx, pt = _d(np.atleast_2d(tx))
    dims, params = flat_params(mlp)
    params, pp = _d(params)
    rmin, prm = _d(mlp.room_min)
    rsz, prs = _d(mlp.room_size)
    N, Q = mean.shape[0], tx.shape[0]
    out = np.zeros((Q, N, int(dims[-1])))
    rc = lib().or_deform(N, pm, H, W, Q, pt, mlp.L_mean, mlp.L_tx, prm, prs, len(mlp.W),
                         dims.ctypes.data_as(I), pp, out.ctypes.data_as(D))
    if rc != 0:
        raise ValueError(f"or_deform failed ({rc})")
    return out


def project(scene, resid, q_cut: float, Q: int | None = None) -> np.ndarray:
    """Deformed Gaussians [Q,N,8] = (mx, my, A, B, C, w, rx, ry) (Eq. 12/13)."""
    arrs = [_d(a) for a in scene.arrays()]
    N = arrs[0][0].shape[0]
    if resid is None:
        Q = 1 if Q is None else Q
        pr = _null(D)
    else:
        resid, pr = _d(resid)
        Q = resid.shape[0]
    out = np.zeros((Q, N, 8))
    lib().or_project(N, arrs[0][1], arrs[1][1], arrs[2][1], arrs[3][1], arrs[4][1], Q, pr,
                     float(q_cut), out.ctypes.data_as(D))
    return out


def render(proj, H: int, W: int, q_cut: float, band: float = 1e-4, with_slack: bool = True,
           wrap: bool = False):
    """Spectra [Q,H,W] (Eq. 9/13) and the per-pixel cutoff-band slack."""
    proj, pp = _d(proj)
    Q, N = proj.shape[0], proj.shape[1]
    out = np.zeros((Q, H, W))
    slack = np.zeros((Q, H, W)) if with_slack else None
    rc = lib().or_render_w(Q, N, pp, H, W, float(q_cut), float(band), int(wrap),
                           out.ctypes.data_as(D), slack.ctypes.data_as(D) if with_slack else _null(D))
    if rc != 0:
        raise ValueError(f"or_render failed ({rc})")
    return out, slack


def forward(scene, mlp, tx, H: int, W: int, q_cut: float, band: float = 1e-4,
            wrap: bool = False):
    """Full path: deform -> project -> render. mlp=None skips the MLP."""
    tx = np.atleast_2d(tx)
    resid = deform(scene, mlp, tx, H, W) if mlp is not None else None
    proj = project(scene, resid, q_cut, Q=tx.shape[0])
    A, slack = render(proj, H, W, q_cut, band, wrap=wrap)
    return A, slack, proj, resid


def forward_complex(scene, mlp, tx, H: int, W: int, q_cut: float, band: float = 1e-4,
                    wrap: bool = False):
    """Two channels: scene.amp [N, 2] holds the real and imaginary amplitude.
    The geometry (deformation, projection, footprint) is shared; each channel
    is the order-free sum with its own weight sigmoid(opacity) * amp_c (Eq.
    9/13), and the result is decomposed into magnitude |A| and phase arg A
    (Sec. 6.1; arg 0 = 0).  Returns (re, im, magnitude, phase, slack), slack
    the larger of the two channels' cutoff-band slacks."""
    amp = np.asarray(scene.amp, np.float64)
    parts = []
    for c in range(2):
        sc = type(scene)(scene.mean, scene.log_scale, scene.rot, scene.opacity_logit,
                         np.ascontiguousarray(amp[:, c]))
        parts.append(forward(sc, mlp, tx, H, W, q_cut, band, wrap=wrap))
    re, im = parts[0][0], parts[1][0]
    return re, im, np.hypot(re, im), np.arctan2(im, re), np.maximum(parts[0][1], parts[1][1])


def rssi(scene, mlp, tx, H: int, W: int, q_cut: float, band: float = 1e-4, wrap: bool = False):
    """RSSI head of Sec. 7.2: each query's H x W map (Eq. 9/13) reduced by a
    global average pool of its magnitude (Sec. 6.6 averages the spectrum
    magnitude over azimuth and elevation; one real channel, so the magnitude is
    |A|).  Returns the pooled values [Q] and the pooled cutoff-band slack [Q]:
    a pooled GPU value is correct within tol + slack."""
    if np.asarray(scene.amp).ndim == 2:  # two channels: the complex map's magnitude
        _, _, mag, _, slack = forward_complex(scene, mlp, tx, H, W, q_cut, band, wrap=wrap)
        return mag.mean(axis=(1, 2)), slack.mean(axis=(1, 2))
    A, slack, _, _ = forward(scene, mlp, tx, H, W, q_cut, band, wrap=wrap)
    return np.abs(A).mean(axis=(1, 2)), slack.mean(axis=(1, 2))


def tiles(H: int, W: int, tw: int, th: int):
    return (W + tw - 1) // tw, (H + th - 1) // th


def bin_f32(rec32, H: int, W: int, tw: int, th: int, cap: int | None = None, wrap: bool = False):
    """Tile lists from FP32 records [Q,N,8]: (counts [Q,N], gids [K], offsets [Q*T+1])."""
    rec32 = np.ascontiguousarray(rec32, dtype=np.float32)
    Q, N = rec32.shape[0], rec32.shape[1]
    ntx, nty = tiles(H, W, tw, th)
    T = ntx * nty
    counts = np.zeros((Q, N), np.uint32)
    offsets = np.zeros(Q * T + 1, np.uint32)
    nk = C.c_int64(0)
    if cap is None:
        cap = 0
        lib().or_bin_f32_w(Q, N, rec32.ctypes.data_as(F), H, W, tw, th, int(wrap),
                           counts.ctypes.data_as(U32), _null(U32), 0, C.byref(nk),
                           offsets.ctypes.data_as(U32))
        cap = int(nk.value)
    gids = np.zeros(max(cap, 1), np.uint32)
    rc = lib().or_bin_f32_w(Q, N, rec32.ctypes.data_as(F), H, W, tw, th, int(wrap),
                            counts.ctypes.data_as(U32), gids.ctypes.data_as(U32), int(cap),
                            C.byref(nk), offsets.ctypes.data_as(U32))
    if rc == -2:
        return counts, None, offsets, int(nk.value)
    if rc != 0:
        raise ValueError(f"or_bin_f32 failed ({rc})")
    return counts, gids[: int(nk.value)], offsets, int(nk.value)


# ReLU decisions whose pre-activation lies within this fraction of the
# magnitude of its terms (|b| + sum |W a|) of zero: an FP32 evaluation of the
# same row may take them either way (its rounding error is ~1e-6 of that
# magnitude), so both gradients are correct; mlp_grad reports the slack.
RELU_BAND = 4e-6


def mlp_grad(scene, mlp, tx, H: int, W: int, d_resid, stop_grad_mean: bool = False,
             band: float = RELU_BAND):
    """FP64 back-propagation through F_theta (Eq. 14-15) of dL/d(resid)
    [Q,N,5]: returns (dW list, db list, d_mean [N,2] through gamma(mean),
    slack dict).  slack holds, per gradient element, the summed absolute
    change when one ambiguous ReLU decision (|z| <= band * magnitude) is
    taken the other way: d_W, d_b (lists) and d_mean; "decisions" counts
    them (0 with band = 0)."""
    tx = np.atleast_2d(tx)
    Q = tx.shape[0]
    dims, params = flat_params(mlp)
    params, ppar = _d(params)
    N = int(np.asarray(scene.mean).shape[0])
    dparams = np.zeros_like(params)
    sl = np.zeros_like(params)
    dmean = np.zeros((N, 2))
    dmean_sl = np.zeros((N, 2))
    mean, pm = _d(scene.mean)
    txd, pt = _d(tx)
    rmin, prm = _d(mlp.room_min)
    rsz, prs = _d(mlp.room_size)
    dr, pdr = _d(d_resid)
    rc = lib().or_mlp_grad_slack(N, pm, H, W, Q, pt, mlp.L_mean, mlp.L_tx, prm, prs, len(mlp.W),
                                 dims.ctypes.data_as(I), ppar, pdr, int(stop_grad_mean),
                                 float(band), dparams.ctypes.data_as(D), dmean.ctypes.data_as(D),
                                 sl.ctypes.data_as(D), dmean_sl.ctypes.data_as(D))
    if rc != 0:
        raise ValueError(f"or_mlp_grad_slack failed ({rc})")
    dW, db = unflat_params(mlp, dparams)
    sW, sb = unflat_params(mlp, sl)
    return dW, db, dmean, dict(d_W=sW, d_b=sb, d_mean=dmean_sl)


def grad(scene, mlp, tx, H: int, W: int, q_cut: float, dA, stop_grad_mean: bool = False,
         wrap: bool = False, band: float = RELU_BAND):
    """Analytic FP64 gradient of L given dL/dA [Q,H,W].

    Returns a dict with d_mean [N,2], d_log_scale [N,2], d_rot [N],
    d_opacity [N], d_amp [N], d_W (list), d_b (list), d_resid [Q,N,5] and
    d_proj [Q,N,6]; with an MLP also "slack": the ambiguous-ReLU slack of
    d_W, d_b and d_mean (see mlp_grad; band = the width of the ambiguous
    zone, as a fraction of a pre-activation's magnitude)."""
    tx = np.atleast_2d(tx)
    Q = tx.shape[0]
    resid = deform(scene, mlp, tx, H, W) if mlp is not None else None
    proj = project(scene, resid, q_cut, Q=Q)
    proj, pp = _d(proj)
    dA, pdA = _d(dA)
    N = proj.shape[1]
    dproj = np.zeros((Q, N, 6))
    lib().or_render_grad_w(Q, N, pp, H, W, float(q_cut), int(wrap), pdA, dproj.ctypes.data_as(D))
    arrs = [_d(a) for a in scene.arrays()]
    dresid = np.zeros((Q, N, 5))
    d_mean = np.zeros((N, 2)); d_ls = np.zeros((N, 2)); d_rot = np.zeros(N)
    d_op = np.zeros(N); d_amp = np.zeros(N)
    presid = _d(resid)[1] if resid is not None else _null(D)
    lib().or_project_grad(N, arrs[1][1], arrs[2][1], arrs[3][1], arrs[4][1], Q, presid,
                          dproj.ctypes.data_as(D), dresid.ctypes.data_as(D),
                          d_mean.ctypes.data_as(D), d_ls.ctypes.data_as(D),
                          d_rot.ctypes.data_as(D), d_op.ctypes.data_as(D),
                          d_amp.ctypes.data_as(D))
    out = dict(d_mean=d_mean, d_log_scale=d_ls, d_rot=d_rot, d_opacity=d_op, d_amp=d_amp,
               d_resid=dresid, d_proj=dproj)
    if mlp is not None:
        dW, db, dmean_mlp, slack = mlp_grad(scene, mlp, tx, H, W, dresid, stop_grad_mean,
                                            band)
        out["d_mean"] = d_mean + dmean_mlp
        out["d_mean_direct"] = d_mean
        out["d_W"], out["d_b"] = dW, db
        out["slack"] = slack
    return out
