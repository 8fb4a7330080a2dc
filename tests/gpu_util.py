"""Helpers shared by the GPU parity tests (inputs from `scenes`, references from
the oracle; nothing here computes any step of the method)."""
import numpy as np
import torch

import oracle as O
import scenes
from paper_2605_06876_b300 import ops

DEV = "cuda"


def np_(t):
    return t.detach().cpu().numpy()


def oracle_projected_to_gpu(orps, n):
    """The oracle's projections of V views, rounded to float32 records."""
    recs = []
    for pr in orps:
        xyod = np.stack([pr["mean2d"][:, 0], pr["mean2d"][:, 1], pr["opacity"], pr["depth"]], 1)
        con = np.concatenate([pr["conic"], np.zeros((n, 1))], 1)
        rgb = np.concatenate([pr["rgb"], np.zeros((n, 1))], 1)
        recs.append((xyod, con, rgb, pr["rect"], pr["tiles"]))
    cat = lambda k, dt: torch.as_tensor(np.ascontiguousarray(np.concatenate([r[k] for r in recs]), dt), device=DEV)
    return ops.Projected(cat(0, np.float32), cat(1, np.float32), cat(2, np.float32),
                         cat(3, np.int32), cat(4, np.int32))


def gpu_forward(scene, cams, params=None, bg=(0.0, 0.0, 0.0)):
    g = ops.Gaussians.from_scene(scene, DEV)
    pr = ops.project(g, cams, params)
    bins = ops.bin_sort(g.n, pr, cams, params)
    img = ops.render(g.n, pr, bins, cams, bg, params)
    torch.cuda.synchronize()
    return g, pr, bins, img


def c0_inputs():
    """The tiny plain step: 2,000 Gaussians, 128x128, SH degree 0, target rendered
    by the oracle from a second seed's 4,000-Gaussian scene."""
    sc = scenes.scene_box(0, 2000, 0)
    tg = scenes.scene_box(1, 4000, 0)
    cam = scenes.camera_origin_forward(128, 128)
    pr_t = O.project(O.theta_of(tg), 0, cam)
    target = O.render(pr_t, cam)["rgb"].astype(np.float32).reshape(128, 128, 3)
    return sc, cam, target


def small_cluster_inputs(n=20000, W=320, H=208, views=1, seed=10):
    sc = scenes.scene_clusters(seed, n, 3)
    cams = scenes.ring_cameras(seed + 1, views, 4.0, W, H)
    return sc, cams
