"""Autotuner of the compositing launch shape: the tile shape and the number of
Gaussians a block stages per batch.

Neither changes any result: every pixel composites the same depth-ordered
contributors whatever the tiling, and the batch only sets how much of a tile's
list sits in shared memory at a time. Only the speed changes. A tile shape that
follows the typical footprint of the scene's Gaussians wastes fewer evaluations;
a smaller batch stages fewer Gaussians a pixel never reaches before the tile
stops, a larger one pays fewer block barriers. The tuner times the fused batched
step (adp_train_step_batched) under every (shape, batch) pair, each captured as a
CUDA graph, and keeps the fastest. Results are cached per (Gaussian count, SH
degree, camera sizes).
"""
from __future__ import annotations

import itertools

import torch

from . import _abi as A
from .pipeline import BatchedStep

SHAPES = ((16, 16), (8, 32), (32, 8))
BATCHES = (256, 128, 64)
_cache = {}


def _time(step, reps):
    graph = step.capture()
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(g, cams, target, reps=5, shapes=SHAPES, batches=BATCHES, params=None):
    """Returns (params with the fastest tile shape and batch, {(tw, th, batch): ms})."""
    key = (g.n, g.sh_degree, tuple((int(c["width"]), int(c["height"])) for c in cams),
           tuple(shapes), tuple(batches))
    if key in _cache:
        best, times = _cache[key]
    else:
        times = {}
        for (tw, th), b in itertools.product(shapes, batches):
            p = A.default_params(tile_w=tw, tile_h=th, batch=b)
            step = BatchedStep(g, cams, target, params=p)
            ms = _time(step, reps)
            if step.fits():
                times[(tw, th, b)] = ms
            del step
            torch.cuda.empty_cache()
        best = min(times, key=times.get)
        _cache[key] = (best, times)
    out = A.default_params() if params is None else params
    out.tile_w, out.tile_h, out.batch = best
    return out, dict(times)


def tune_tile_shape(g, cams, target, reps=5, shapes=SHAPES, params=None):
    """The tile shape alone (batch 256): (params, {(tw, th): ms})."""
    out, times = tune(g, cams, target, reps, shapes, (256,), params)
    return out, {(k[0], k[1]): v for k, v in times.items()}
