"""Seeded synthetic inputs for the AdpSplit hot path.

This module only draws random inputs: Gaussian scenes, pinhole cameras, fallback
noise and stand-in image/dominant maps for stage tests. It holds none of the
method's arithmetic (no projection, compositing, error maps or splitting), so both
the CUDA path and the FP64 oracle can take their inputs from here without sharing
any computation.

Every array it returns is float32 (the storage precision of the CUDA path) or an
integer type; the oracle widens float32 to float64 losslessly.

The shapes and distributions follow the workloads the paper trains on (indoor and
outdoor captures of MipNeRF360, Deep-Blending and Tanks&Temples, Sec. 5.1), which are
not available here: the cluster scenes below stand in for them.

Parameter layout of a scene (a plain dict):
    mean      [n, 3]     world-space centre
    logit     [n]        opacity logit (opacity = sigmoid(logit))
    logscale  [n, 3]     log of the per-axis standard deviation
    quat      [n, 4]     rotation quaternion (w, x, y, z), unit norm
    sh        [n, K, 3]  spherical-harmonic coefficients, K = (degree + 1)^2,
                         coefficient-major with the RGB channel innermost
    sh_degree int
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "camera_look_at",
    "camera_origin_forward",
    "scene_box",
    "scene_clusters",
    "ring_cameras",
    "hemisphere_cameras",
    "uneven_resolutions",
    "fallback_noise",
    "error_stage_inputs",
    "subscene_for_gradients",
    "scene_initial_points",
    "CONFIGS",
]

# The DC coefficient range that maps to colours in [0, 1] under the 3DGS colour
# decode is [-sqrt(pi), sqrt(pi)]: a uniform colour is drawn as a uniform DC value.
_DC_HALF_RANGE = math.sqrt(math.pi)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _attributes(rng, n, sh_degree, mean):
    """Per-Gaussian attribute distributions shared by every workload."""
    K = (sh_degree + 1) ** 2
    logscale = rng.normal(-3.0, 0.5, size=(n, 3))
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    logit = rng.normal(0.0, 1.0, size=n)
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, K - 1, 3))
    return {
        "mean": _f32(mean),
        "logit": _f32(logit),
        "logscale": _f32(logscale),
        "quat": _f32(quat),
        "sh": _f32(sh),
        "sh_degree": int(sh_degree),
    }


def scene_box(seed: int, n: int, sh_degree: int = 0):
    """Means uniform in [-1,1]^2 x [2,6] (the tiny config's scene)."""
    rng = np.random.default_rng(seed)
    mean = np.stack(
        [rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 6, n)], axis=1
    )
    return _attributes(rng, n, sh_degree, mean)


def _random_rotation(rng):
    """A random orthonormal 3x3 matrix with det +1 (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _uniform_ball(rng, n, radius):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * (radius * rng.uniform(0, 1, size=(n, 1)) ** (1.0 / 3.0))


def scene_clusters(seed: int, n: int, sh_degree: int = 3, n_clusters: int = 64,
                   background_frac: float = 0.2):
    """Mixture of anisotropic 3D clusters plus a uniform background.

    Cluster centres are uniform in the radius-8 ball, cluster axis scales are
    U(0.2, 1.5) with a random orientation; the background is uniform in the
    radius-10 ball and holds `background_frac` of the points.
    """
    rng = np.random.default_rng(seed)
    n_bg = int(round(background_frac * n))
    n_cl = n - n_bg
    centres = _uniform_ball(rng, n_clusters, 8.0)
    axes = rng.uniform(0.2, 1.5, size=(n_clusters, 3))
    rots = np.stack([_random_rotation(rng) for _ in range(n_clusters)])
    which = rng.integers(0, n_clusters, size=n_cl)
    local = rng.normal(size=(n_cl, 3)) * axes[which]
    pts = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    bg = _uniform_ball(rng, n_bg, 10.0)
    mean = np.concatenate([pts, bg], axis=0)
    mean = mean[rng.permutation(n)]
    return _attributes(rng, n, sh_degree, mean)


def camera_look_at(position, target, width, height, fov_deg=60.0):
    """OpenCV pinhole camera (x right, y down, z forward) looking at `target`.

    Focal length from the horizontal field of view, principal point at the image
    centre ((W-1)/2, (H-1)/2). World +y is "down". Returns float32 fields:
    width, height, fx, fy, px, py, R (world->camera, row-major 3x3), t.
    """
    position = np.asarray(position, dtype=np.float64)
    forward = np.asarray(target, dtype=np.float64) - position
    forward /= np.linalg.norm(forward)
    down = np.array([0.0, 1.0, 0.0])
    if abs(np.dot(down, forward)) > 0.999:
        down = np.array([0.0, 0.0, 1.0])
    right = np.cross(down, forward)
    right /= np.linalg.norm(right)
    down_c = np.cross(forward, right)
    R = np.stack([right, down_c, forward], axis=0)
    t = -R @ position
    f = width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return {
        "width": int(width),
        "height": int(height),
        "fx": np.float32(f),
        "fy": np.float32(f),
        "px": np.float32((width - 1) / 2.0),
        "py": np.float32((height - 1) / 2.0),
        "R": _f32(R.reshape(9)),
        "t": _f32(t),
    }


def camera_origin_forward(width, height, fov_deg=60.0):
    """Camera at the origin looking along +z with identity rotation."""
    f = width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return {
        "width": int(width),
        "height": int(height),
        "fx": np.float32(f),
        "fy": np.float32(f),
        "px": np.float32((width - 1) / 2.0),
        "py": np.float32((height - 1) / 2.0),
        "R": _f32(np.eye(3).reshape(9)),
        "t": _f32(np.zeros(3)),
    }


def ring_cameras(seed, n_views, radius, width, height, fov_deg=60.0):
    """Cameras on a horizontal ring around the origin, looking at the origin."""
    rng = np.random.default_rng(seed)
    angles = rng.uniform(0, 2 * math.pi, size=n_views)
    return [
        camera_look_at((radius * math.cos(a), 0.0, radius * math.sin(a)), (0, 0, 0),
                       width, height, fov_deg)
        for a in angles
    ]


def uneven_resolutions(seed, n_views):
    """Resolutions between 640x416 and 1600x1056 (landscape, one draw per view)."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(0, 1, size=n_views)
    return [(640 + int(round(960 * x)), 416 + int(round(640 * x))) for x in s]


def hemisphere_cameras(seed, n_views, radius, resolutions, fov_deg=60.0):
    """Cameras on the upper hemisphere (world -y is up) looking at the origin."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_views):
        d = rng.normal(size=3)
        d[1] = -abs(d[1])
        d /= np.linalg.norm(d)
        w, h = resolutions[i]
        cams.append(camera_look_at(radius * d, (0, 0, 0), w, h, fov_deg))
    return cams


def fallback_noise(seed, n_cand):
    """Standard normal draws for the two vanilla-split children of each candidate,
    shape [n_cand, 2, 3] (the offsets of Eq. 3 before scaling by s)."""
    rng = np.random.default_rng(seed)
    return _f32(rng.normal(size=(n_cand, 2, 3)))


def error_stage_inputs(seed, width, height, n_gauss, n_cells=None, bg_frac=0.05,
                       n_patches=None):
    """Stand-in inputs for the error-statistics stage at any image size.

    Returns (image [H,W,3] f32, target [H,W,3] f32, dominant [H,W] int32) shaped like
    a render: the dominant map is a Voronoi partition into cells owned by random
    Gaussian ids (a few cells left at -1), the image is smooth, and the target
    differs from it by elliptical error patches of random strength plus mild noise,
    so the thresholded error forms connected regions of many sizes.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    P = width * height
    if n_cells is None:
        n_cells = max(16, P // 400)
    if n_patches is None:
        n_patches = max(8, P // 2000)
    centres = np.stack([rng.uniform(0, width, n_cells), rng.uniform(0, height, n_cells)], 1)
    owner = rng.integers(0, n_gauss, size=n_cells).astype(np.int32)
    owner[rng.uniform(size=n_cells) < bg_frac] = -1
    yy, xx = np.mgrid[0:height, 0:width]
    pix = np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float64)
    _, nearest = cKDTree(centres).query(pix)
    dominant = owner[nearest].reshape(height, width).astype(np.int32)

    # Smooth base image: a few large blobs per channel.
    img = np.full((height, width, 3), 0.5)
    for _ in range(12):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        sx, sy = rng.uniform(0.1, 0.4) * width, rng.uniform(0.1, 0.4) * height
        amp = rng.uniform(-0.3, 0.3, size=3)
        g = np.exp(-0.5 * (((xx - cx) / sx) ** 2 + ((yy - cy) / sy) ** 2))
        img += g[..., None] * amp
    img = np.clip(img, 0.0, 1.0)
    tgt = img + rng.normal(0.0, 0.01, size=img.shape)
    for _ in range(n_patches):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        sx, sy = rng.uniform(1.5, 12.0), rng.uniform(1.5, 12.0)
        th = rng.uniform(0, math.pi)
        amp = rng.uniform(-0.8, 0.8, size=3)
        c, s = math.cos(th), math.sin(th)
        rad = 6.0 * max(sx, sy)  # the patch is negligible beyond six deviations
        x0, x1 = max(0, int(cx - rad)), min(width, int(cx + rad) + 1)
        y0, y1 = max(0, int(cy - rad)), min(height, int(cy + rad) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        dx, dy = xx[y0:y1, x0:x1] - cx, yy[y0:y1, x0:x1] - cy
        u = (c * dx + s * dy) / sx
        v = (-s * dx + c * dy) / sy
        g = np.exp(-0.5 * (u * u + v * v))
        tgt[y0:y1, x0:x1] += g[..., None] * amp
    tgt = np.clip(tgt, 0.0, 1.0)
    return _f32(img), _f32(tgt), dominant


def subscene_for_gradients(seed, n=64, width=32, height=32):
    """A small scene for finite-difference checks of the backward pass.

    Means are placed in front of a 32x32 camera at the origin, opacities stay
    below 0.9 (logit < 2.2) so the 0.99 alpha clamp is never reached, and scales
    are large enough that every Gaussian covers several pixels.
    """
    rng = np.random.default_rng(seed)
    z = rng.uniform(2.5, 4.0, n)
    x = rng.uniform(-0.45, 0.45, n) * z
    y = rng.uniform(-0.45, 0.45, n) * z
    sc = _attributes(rng, n, 3, np.stack([x, y, z], 1))
    sc["logscale"] = _f32(rng.normal(-2.3, 0.3, size=(n, 3)))
    sc["logit"] = _f32(rng.uniform(-1.5, 1.5, size=n))
    return sc, camera_origin_forward(width, height, 60.0)


def scene_initial_points(scene, frac, seed, init_scale=0.1, init_opacity=0.1):
    """A coarse initial model in the manner of a sparse point initialisation: the
    means of a random fraction of a scene's Gaussians, jittered by a tenth of the
    initial scale, with isotropic scales, identity rotations, one low opacity and a
    grey colour (zero SH)."""
    rng = np.random.default_rng(seed)
    n_all = scene["mean"].shape[0]
    n = max(1, int(round(frac * n_all)))
    idx = rng.choice(n_all, size=n, replace=False)
    mean = scene["mean"][idx].astype(np.float64) + rng.normal(0.0, 0.1 * init_scale, size=(n, 3))
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    quat = np.zeros((n, 4))
    quat[:, 0] = 1.0
    return {
        "mean": _f32(mean),
        "logit": _f32(np.full(n, math.log(init_opacity / (1.0 - init_opacity)))),
        "logscale": _f32(np.full((n, 3), math.log(init_scale))),
        "quat": _f32(quat),
        "sh": _f32(np.zeros((n, K, 3))),
        "sh_degree": deg,
    }


# Workload recipes. Scene seed 2k and target seed 2k+1 for config k.
CONFIGS = {
    0: dict(name="tiny plain step", n=2000, n_target=4000, sh_degree=0, scene="box",
            width=128, height=128, views=1, cand_frac=0.10),
    1: dict(name="single-view plain path", n=1_000_000, n_target=1_500_000, sh_degree=3,
            scene="clusters", width=1280, height=832, views=1, ring_radius=4.0, cand_frac=0.10),
    2: dict(name="hand backward", n=2_000_000, sh_degree=3, scene="clusters", width=1280,
            height=832, views=1, ring_radius=4.0),
    3: dict(name="batched uneven views", n=3_000_000, sh_degree=3, scene="clusters", views=16,
            hemisphere_radius=5.0),
    4: dict(name="densification-round stress", n=5_000_000, sh_degree=3, scene="clusters",
            width=1280, height=832, views=8, ring_radius=4.0, cand_frac=0.20),
}
