"""Tile-shape autotuner for the batched forward.

For a workload (scene size N, grid H x W, queries per launch Q, MLP
precision) every supported tile shape is tried: a BatchedForward is built,
its key capacity reserved, the step captured as a CUDA graph and replayed a
few times; the shape with the smallest mean replay time (CUDA events on the
launching stream) wins.  Results persist in a JSON cache keyed by the
workload so later runs skip the search.
"""
from __future__ import annotations

import json
import os

import torch

from . import api
from .batched import BatchedForward

TILE_SHAPES = ((8, 8), (16, 8), (16, 16), (32, 8), (32, 16))
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def workload_key(n, H, W, Q, precision, q_cut, wrap=False):
    return f"n{n}_h{H}_w{W}_q{Q}_p{precision}_c{q_cut:g}" + ("_wrap" if wrap else "")


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


def tune(scene: api.DeviceScene, mlp: api.DeviceMLP, H: int, W: int, tx, q_cut=9.0, reps=5,
         cache_path: str | None = DEFAULT_CACHE, shapes=TILE_SHAPES, verbose=False, wrap=False):
    """Best (tile_w, tile_h) for this workload and the timings of all shapes
    (ms per step).  tx: device tensor [Q,3] of representative TX positions."""
    Q = int(tx.shape[0])
    key = workload_key(scene.n, H, W, Q, mlp.precision, q_cut, wrap)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        e = cache[key]
        return tuple(e["best"]), e["ms"]
    stream = torch.cuda.Stream(device=tx.device)
    times = {}
    for tw, th in shapes:
        grid = api.make_grid(H, W, tw, th, q_cut, wrap)
        fw = BatchedForward(scene, mlp, grid, Q, tx.device)
        with torch.cuda.stream(stream):
            fw.reserve(tx, stream)
        times[f"{tw}x{th}"] = time_step(fw, tx, stream, reps)
        if verbose:
            print(f"tile {tw}x{th}: {times[f'{tw}x{th}']:.3f} ms/step")
        del fw
    best = min(times, key=times.get)
    best_t = tuple(int(v) for v in best.split("x"))
    if cache_path:
        cache[key] = {"best": list(best_t), "ms": times}
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best_t, times
