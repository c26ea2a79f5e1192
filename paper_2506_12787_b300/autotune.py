"""Launch-configuration autotuner for the batched forward.

The rasteriser has three independent knobs:
  * the tile shape (tile_w x tile_h pixels per CTA: 8x8, 16x8, 16x16, 32x8,
    32x16), which also sets the binning granularity;
  * pixels per thread (2: rows y and y + 4 of an 8 x 8 warp block; 4: also
    column x + 8, a 16 x 8 warp block, tiles at least 16 wide), which sets
    the threads per tile;
  * records per thread per shared-memory batch (1 or 2), so a staged batch
    holds (tile pixels / pixels per thread) x that many Gaussians: 32 to 512
    depending on the other two knobs;
  * how the records are staged: per-thread cp.async, or TMA gathers of four
    records per copy.
For a workload (scene size N and channels, grid H x W, queries per launch
Q, MLP precision, cutoff, wrap) every combination in the search space is tried: a
BatchedForward is built, its key capacity reserved, the step captured as a
CUDA graph and replayed a few times; the combination with the smallest mean
replay time (CUDA events on the launching stream) wins.  Results persist in a
JSON cache whose key names the workload and the search space, so a cache
entry is only reused for the same workload searched over the same knobs.
"""
from __future__ import annotations

import hashlib
import json
import os
import re

import torch

from . import api
from .batched import BatchedForward

TILE_SHAPES = ((8, 8), (16, 8), (16, 16), (32, 8), (32, 16))
PX_PER_THREAD = (2, 4)
BATCH_FACTORS = (1, 2)
STAGINGS = (0, 1)  # 0: per-thread cp.async, 1: TMA gathers
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def space(shapes=TILE_SHAPES, pxs=PX_PER_THREAD, bfs=BATCH_FACTORS, stagings=STAGINGS):
    """Every supported (tile_w, tile_h, px_per_thread, batch_factor, tma)."""
    return [(tw, th, px, bf, tma) for tw, th in shapes for px in pxs for bf in bfs
            for tma in stagings if not (px == 4 and tw < 16)]


def batch_records(tw, th, px, bf, tma=0):
    """Gaussians one staged shared-memory batch holds."""
    return tw * th // px * bf


def config_name(tw, th, px=2, bf=1, tma=0):
    return f"{tw}x{th}p{px}b{bf}" + ("t" if tma else "")


def parse_config(s: str):
    """'32x8' (default knobs), '32x8p4b2' or '32x8p4b2t' (TMA staging) ->
    (tile_w, tile_h, px, bf, tma)."""
    m = re.fullmatch(r"(\d+)x(\d+)(?:p(\d))?(?:b(\d))?(t?)", s.strip())
    if not m:
        raise ValueError(f"bad launch configuration {s!r}: want WxH or WxHpPXbBF[t]")
    tw, th = int(m.group(1)), int(m.group(2))
    return tw, th, int(m.group(3) or 2), int(m.group(4) or 1), 1 if m.group(5) else 0


def make_grid(H, W, cfg, q_cut, wrap=False):
    tw, th, px, bf, tma = (tuple(cfg) + (0,))[:5]
    return api.make_grid(H, W, tw, th, q_cut, wrap, px_per_thread=px, batch_factor=bf,
                         tma_staging=tma)


def workload_key(n, H, W, Q, precision, q_cut, wrap=False, candidates=None, channels=1):
    key = f"n{n}_h{H}_w{W}_q{Q}_p{precision}_c{q_cut:g}_ch{channels}" + ("_wrap" if wrap else "")
    cand = space() if candidates is None else candidates
    sig = hashlib.sha1(",".join(config_name(*c) for c in sorted(cand)).encode()).hexdigest()[:10]
    return f"{key}_s{sig}"


def time_step(fw, tx, stream, reps):
    g = fw.graph(tx, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g.replay()
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _load(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def tune(scene: api.DeviceScene, mlp: api.DeviceMLP, H: int, W: int, tx, q_cut=9.0, reps=5,
         cache_path: str | None = DEFAULT_CACHE, candidates=None, verbose=False, wrap=False):
    """Best (tile_w, tile_h, px_per_thread, batch_factor, tma) for this workload and
    the timings of every candidate (ms per step, keyed by config_name).
    tx: device tensor [Q,3] of representative TX positions."""
    Q = int(tx.shape[0])
    cand = space() if candidates is None else [tuple(c) for c in candidates]
    key = workload_key(scene.n, H, W, Q, mlp.precision, q_cut, wrap, cand, scene.channels)
    cache = _load(cache_path)
    if key in cache:
        e = cache[key]
        return tuple(e["best"]), e["ms"]
    stream = torch.cuda.Stream(device=tx.device)
    times = {}
    for cfg in cand:
        fw = BatchedForward(scene, mlp, make_grid(H, W, cfg, q_cut, wrap), Q, tx.device)
        with torch.cuda.stream(stream):
            fw.reserve(tx, stream)
        name = config_name(*cfg)
        times[name] = time_step(fw, tx, stream, reps)
        if verbose:
            print(f"{name} ({batch_records(*cfg)} Gaussians per batch): "
                  f"{times[name]:.3f} ms/step")
        del fw
    best_name = min(times, key=times.get)
    best = parse_config(best_name)
    if cache_path:
        cache = _load(cache_path)
        cache[key] = {"best": list(best), "ms": times}
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best, times
