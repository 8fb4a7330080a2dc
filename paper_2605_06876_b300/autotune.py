"""Tile-shape autotuner.

The per-pixel result does not depend on the tile shape (every pixel composites the
same depth-ordered contributors), only the speed does: a shape that follows the
typical footprint of the scene's Gaussians wastes fewer evaluations. The tuner times
the view-dependent stages (projection, binning, compositing, error statistics,
backward) under each 256-pixel tile shape, as a CUDA graph, and keeps the fastest.
Results are cached per (Gaussian count, SH degree, camera sizes).
"""
from __future__ import annotations

import torch

from . import _abi as A
from .pipeline import ViewStages, capture_graph

SHAPES = ((16, 16), (8, 32), (32, 8))
_cache = {}


def tune_tile_shape(g, cams, target, reps=5, shapes=SHAPES, params=None):
    """Returns (params with the fastest tile shape, {shape: ms})."""
    key = (g.n, g.sh_degree, tuple((int(c["width"]), int(c["height"])) for c in cams))
    if key in _cache:
        best, times = _cache[key]
    else:
        times = {}
        for tw, th in shapes:
            p = A.default_params(tile_w=tw, tile_h=th)
            vs = ViewStages(g, cams, target, params=p)
            graph = capture_graph(vs.run)
            graph.replay()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                graph.replay()
            e1.record()
            torch.cuda.synchronize()
            if not vs.fits():
                continue
            times[(tw, th)] = e0.elapsed_time(e1) / reps
            del vs, graph
        best = min(times, key=times.get)
        _cache[key] = (best, times)
    out = A.default_params() if params is None else params
    out.tile_w, out.tile_h = best
    return out, dict(times)
