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


COLOUR_TOL = 2e-4


def compare_render(rgb, T, n_contrib, dominant, o, label=""):
    """Per-pixel parity of a GPU render with the oracle's (o = oracle.render with
    its default, absolute 1e-6 tie bands): colour within COLOUR_TOL, T within 1e-4,
    the contributor count and the dominant id exact, except at tie pixels. Every
    disagreement must lie at a tie (a contributor's alpha or stop test within the
    band of its threshold, or, for the dominant id alone, a weight margin within
    the band, where the GPU's id must be the oracle's first or second). The pixels
    excused that way must be at most 1e-4 of the pixels. Returns (tie fraction,
    excused pixels, pixels), also printed."""
    tie = o["tie"] != 0
    P = len(tie)
    err = np.abs(np.asarray(rgb, np.float64) - o["rgb"]).max(1)
    bad = (err > COLOUR_TOL) | (np.abs(T - o["T"]) > 1e-4) | (n_contrib != o["n_contrib"])
    dbad = dominant != o["dominant"]
    dtie = (o["tie"] & 8) != 0
    assert not np.any(bad & ~tie), (label, "colour/T/count outside ties", np.nonzero(bad & ~tie)[0][:10],
                                   err[bad & ~tie][:10])
    ok_dom = ~dbad | (tie & ~dtie) | (dtie & (dominant == o["second"]))
    assert np.all(ok_dom), (label, "dominant outside ties", np.nonzero(~ok_dom)[0][:10])
    excused = int((bad | dbad).sum())
    print(f"[parity] {label}: {P} pixels, tie fraction {tie.mean():.3g}, excused {excused}")
    assert excused <= int(1e-4 * P), (label, "excused pixels", excused, P)
    return float(tie.mean()), excused, P
