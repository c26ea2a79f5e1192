"""Seeded synthetic inputs for the spectrum-synthesis path.

This module holds only random-number draws and shape bookkeeping: no step of
the method (positional encoding, MLP, deformation, projection, binning,
rasterisation) is computed here.  Both the FP64 oracle and the CUDA library
take their inputs from these generators, so neither depends on the other.

Every generator uses numpy's counter-based Philox bit generator with an
explicit seed, and draws its arrays in a fixed order, so a (function, seed)
pair always yields the same bytes.

Scene shapes follow the paper's indoor workloads: a 360 x 90 (1 degree)
azimuth x elevation spectrum (Sec. 3.1, Eq. 5), about 10k Gaussians scattered
over the spectrum plane (Sec. 6.1), and a transmitter moving inside a room.
The datasets the paper trains on (NeRF2-s23 and the ray-traced rooms) are not
used; these synthetic scenes stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ROOM_MIN = (0.0, 0.0, 0.0)
ROOM_SIZE = (5.0, 5.0, 3.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclasses.dataclass
class Scene:
    """Reference-frame Gaussians, structure of arrays, FP32.

    mean:          [N,2] pixels; x = azimuth column, y = elevation row
    log_scale:     [N,2] natural log of the two principal std-devs (pixels)
    rot:           [N]   rotation of the first principal axis (radians)
    opacity_logit: [N]   pre-sigmoid attenuation
    amp:           [N]   scalar signal response (one channel)
    """
    mean: np.ndarray
    log_scale: np.ndarray
    rot: np.ndarray
    opacity_logit: np.ndarray
    amp: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def arrays(self):
        return (self.mean, self.log_scale, self.rot, self.opacity_logit, self.amp)


@dataclasses.dataclass
class MLP:
    """Deformation MLP weights: W[l] is [out, in] row-major, b[l] is [out]."""
    W: list
    b: list
    L_mean: int = 6
    L_tx: int = 10
    room_min: tuple = ROOM_MIN
    room_size: tuple = ROOM_SIZE

    @property
    def dims(self):
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]


def make_scene(n: int, H: int, W: int, *, ls_mean: float = math.log(3.0),
               ls_std: float = 0.3, seed: int = 0) -> Scene:
    """Means U[0,W) x U[0,H); log-scales N(ls_mean, ls_std^2); rotation
    U[0,pi); opacity logit N(0,1); amplitude U(0,1)."""
    g = rng(seed)
    mx = g.uniform(0.0, W, size=n)
    my = g.uniform(0.0, H, size=n)
    ls = g.normal(ls_mean, ls_std, size=(n, 2))
    rot = g.uniform(0.0, math.pi, size=n)
    op = g.normal(0.0, 1.0, size=n)
    amp = g.uniform(0.0, 1.0, size=n)
    f = np.float32
    return Scene(np.stack([mx, my], 1).astype(f), ls.astype(f), rot.astype(f),
                 op.astype(f), amp.astype(f))


def mlp_dims(L_mean: int = 6, L_tx: int = 10, hidden: int = 128,
             n_hidden: int = 4, out: int = 5):
    d_in = 2 * (2 * L_mean + 1) + 3 * (2 * L_tx + 1)
    return [d_in] + [hidden] * n_hidden + [out]


def make_mlp(*, L_mean: int = 6, L_tx: int = 10, hidden: int = 128,
             n_hidden: int = 4, out: int = 5, gain: float = 0.1,
             bias_std: float = 0.0, seed: int = 0) -> MLP:
    """Xavier-uniform weights U(+-gain*sqrt(6/(in+out))); biases 0 unless
    bias_std > 0 (then N(0, bias_std^2), used by tests that want non-zero
    biases to be exercised)."""
    g = rng(seed + 1000)
    dims = mlp_dims(L_mean, L_tx, hidden, n_hidden, out)
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = gain * math.sqrt(6.0 / (fan_in + fan_out))
        Ws.append(g.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32))
        if bias_std > 0:
            bs.append(g.normal(0.0, bias_std, size=fan_out).astype(np.float32))
        else:
            bs.append(np.zeros(fan_out, np.float32))
    return MLP(Ws, bs, L_mean, L_tx)


def complex_amplitudes(scene: Scene, *, seed: int = 0) -> Scene:
    """Copy of a scene with two-channel amplitudes amp * (cos phi, sin phi),
    phi ~ U[-pi, pi) (real and imaginary response)."""
    g = rng(seed + 5000)
    ph = g.uniform(-math.pi, math.pi, size=scene.amp.shape[0])
    a = scene.amp.astype(np.float64)
    amp = np.stack([a * np.cos(ph), a * np.sin(ph)], 1).astype(np.float32)
    return Scene(scene.mean, scene.log_scale, scene.rot, scene.opacity_logit, amp)


@dataclasses.dataclass
class PaperScene:
    """Primitives of the paper's head, structure of arrays, FP32.

    mu:         [N,2] raw angular centre (u, v) before the tanh map
    chol:       [N,3] Cholesky entries (l1, l2, l3) of Sigma (pixels)
    attn_logit: [N]   pre-sigmoid attenuation a
    psi:        [N,2] complex response (re, im)
    """
    mu: np.ndarray
    chol: np.ndarray
    attn_logit: np.ndarray
    psi: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])


def make_paper_scene(n: int, H: int, W: int, *, ls_mean: float = math.log(3.0),
                     ls_std: float = 0.3, seed: int = 0) -> PaperScene:
    """Centres uniform over the map (u = atanh(2x/W - 1)), diagonal Cholesky
    entries exp(N(ls_mean, ls_std^2)) pixels, off-diagonal N(0, 0.5^2) pixels,
    attenuation logit N(0,1), response |psi| ~ U(0,1) with a uniform phase."""
    g = rng(seed + 7000)
    x = g.uniform(0.0, W, size=n)
    y = g.uniform(0.0, H, size=n)
    u = np.arctanh(np.clip(2.0 * x / W - 1.0, -0.999999, 0.999999))
    v = np.arctanh(np.clip(2.0 * y / H - 1.0, -0.999999, 0.999999))
    l1 = np.exp(g.normal(ls_mean, ls_std, size=n))
    l3 = np.exp(g.normal(ls_mean, ls_std, size=n))
    l2 = g.normal(0.0, 0.5, size=n)
    a = g.normal(0.0, 1.0, size=n)
    r = g.uniform(0.0, 1.0, size=n)
    ph = g.uniform(-math.pi, math.pi, size=n)
    f = np.float32
    return PaperScene(np.stack([u, v], 1).astype(f), np.stack([l1, l2, l3], 1).astype(f),
                      a.astype(f), np.stack([r * np.cos(ph), r * np.sin(ph)], 1).astype(f))


def make_paper_mlp(*, L_mean: int = 10, L_tx: int = 6, width: int = 156, n_hidden: int = 8,
                   skips=(2, 4, 6), gain: float = 0.1, bias_std: float = 0.0,
                   seed: int = 0) -> MLP:
    """The paper's deformation network shape: n_hidden layers of `width`, the
    encoded input concatenated to the activations entering the layers in
    `skips` (0-based), output 5; Xavier-uniform weights times `gain`."""
    g = rng(seed + 8000)
    din = 2 * (2 * L_mean + 1) + 3 * (2 * L_tx + 1)
    ins = [din] + [width + (din if l in skips else 0) for l in range(1, n_hidden)] + [width]
    outs = [width] * n_hidden + [5]
    Ws, bs = [], []
    for fan_in, fan_out in zip(ins, outs):
        lim = gain * math.sqrt(6.0 / (fan_in + fan_out))
        Ws.append(g.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32))
        bs.append((g.normal(0.0, bias_std, size=fan_out) if bias_std > 0
                   else np.zeros(fan_out)).astype(np.float32))
    return MLP(Ws, bs, L_mean, L_tx)


def zero_mlp(L_mean: int = 6, L_tx: int = 10, hidden: int = 128,
             n_hidden: int = 4, out: int = 5) -> MLP:
    dims = mlp_dims(L_mean, L_tx, hidden, n_hidden, out)
    Ws = [np.zeros((dims[i + 1], dims[i]), np.float32) for i in range(len(dims) - 1)]
    bs = [np.zeros(dims[i + 1], np.float32) for i in range(len(dims) - 1)]
    return MLP(Ws, bs, L_mean, L_tx)


def make_tx(q: int, *, seed: int = 0, room_min=ROOM_MIN, room_size=ROOM_SIZE) -> np.ndarray:
    """TX positions [Q,3] metres, uniform in the room box."""
    g = rng(seed + 2000)
    lo = np.asarray(room_min, np.float64)
    sz = np.asarray(room_size, np.float64)
    return (lo + g.uniform(0.0, 1.0, size=(q, 3)) * sz).astype(np.float32)


def jitter_means(scene: Scene, std_px: float, *, seed: int = 0) -> Scene:
    """Copy of a scene with means jittered by N(0, std_px^2) (training targets)."""
    g = rng(seed + 3000)
    m = scene.mean.astype(np.float64) + g.normal(0.0, std_px, size=scene.mean.shape)
    return Scene(m.astype(np.float32), scene.log_scale.copy(), scene.rot.copy(),
                 scene.opacity_logit.copy(), scene.amp.copy())


def random_rects_records(q: int, n: int, H: int, W: int, *, r_max: float = 20.0,
                         off_grid: float = 0.1, seed: int = 0) -> np.ndarray:
    """FP32 records [Q,N,8] for binning tests.  Only the fields binning reads
    are meaningful: [0]=centre x, [1]=centre y, [6]=half-width x, [7]=half-width y.
    A fraction `off_grid` of the centres are placed outside the grid; a few
    half-widths are zero (degenerate footprints)."""
    g = rng(seed + 4000)
    rec = np.zeros((q, n, 8), np.float64)
    rec[..., 0] = g.uniform(-0.1 * W, 1.1 * W, size=(q, n))
    rec[..., 1] = g.uniform(-0.1 * H, 1.1 * H, size=(q, n))
    far = g.uniform(0, 1, size=(q, n)) < off_grid
    rec[..., 0][far] += W * 3.0
    rec[..., 6] = g.uniform(0.0, r_max, size=(q, n))
    rec[..., 7] = g.uniform(0.0, r_max, size=(q, n))
    zero = g.uniform(0, 1, size=(q, n)) < 0.02
    rec[..., 6][zero] = 0.0
    # remaining fields: plausible positive-definite conic and weights
    rec[..., 2] = g.uniform(0.01, 0.5, size=(q, n))
    rec[..., 4] = g.uniform(0.01, 0.5, size=(q, n))
    rec[..., 3] = 0.0
    rec[..., 5] = g.uniform(0.0, 1.0, size=(q, n))
    return rec.astype(np.float32)


def poisson_arrivals(rate_per_s: float, duration_s: float, n_scenes: int, *,
                     seed: int = 0):
    """Arrival times (s) of a Poisson stream and a uniformly drawn scene index
    per arrival."""
    g = rng(seed + 5000)
    n_exp = int(rate_per_s * duration_s * 1.2) + 16
    gaps = g.exponential(1.0 / rate_per_s, size=n_exp)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    scenes = g.integers(0, n_scenes, size=t.shape[0])
    return t, scenes


# Workloads (sizes and distributions stated once, used by tests and bench).
CONFIGS = {
    "plain_1q_n1024": dict(n=1024, H=90, W=360, Q=1, ls_mean=math.log(3.0), ls_std=0.3,
                           precision="fp32"),
    "batched_q256_n20k": dict(n=20000, H=90, W=360, Q=256, ls_mean=math.log(3.0), ls_std=0.3,
                              precision="bf16"),
    "train_q64_n20k": dict(n=20000, H=90, W=360, Q=64, ls_mean=math.log(3.0), ls_std=0.3,
                           precision="bf16"),
    "serving_8scenes": dict(scene_sizes=(5000, 10000, 20000, 20000, 40000, 40000, 80000, 120000),
                            H=90, W=360, rate=50000.0, ls_mean=math.log(3.0), ls_std=0.3),
    "large_q1024_n200k": dict(n=200000, H=180, W=720, Q=1024, ls_mean=math.log(2.0), ls_std=0.5,
                              precision="bf16"),
}
