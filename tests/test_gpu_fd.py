"""The hand-written backward against central finite differences of the CUDA
forward itself (h = 1e-3), on the 64-Gaussian, 32x32 sub-scene whose opacities
stay below the alpha clamp. The loss is the mean L1 error of the float32 render,
summed in float64 on the host. Entries whose differences at h and h/2 disagree
straddle a kink of the forward (alpha cut-off, L1 sign) and are left out."""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV
from paper_2605_06876_b300 import ops

pytestmark = pytest.mark.gpu

H_STEP = 1e-3
FIELDS = [("mean", 3), ("logit", 1), ("logscale", 3), ("quat", 4), ("sh", 48)]


def _loss(scene, cam, target):
    g = ops.Gaussians.from_scene(scene, DEV)
    pr = ops.project(g, [cam])
    bins = ops.bin_sort(g.n, pr, [cam])
    img = ops.render(g.n, pr, bins, [cam])
    return float(np.abs(img.rgb.double().cpu().numpy() - target.reshape(-1, 3)).mean())


def _perturbed(scene, field, i, c, delta):
    sc = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    arr = sc[field]
    flat = arr.reshape(arr.shape[0], -1)
    flat[i, c] = np.float32(flat[i, c] + delta)
    return sc, float(flat[i, c])


def test_backward_matches_central_differences():
    sc, cam = scenes.subscene_for_gradients(0)
    tsub, _ = scenes.subscene_for_gradients(1, n=48)
    target = O.render(O.project(O.theta_of(tsub), 3, cam), cam)["rgb"].astype(np.float32)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, [cam])
    bins = ops.bin_sort(g.n, pr, [cam])
    img = ops.render(g.n, pr, bins, [cam])
    grad = ops.render_backward(g, pr, bins, img, [cam],
                               target=torch.as_tensor(target.reshape(-1, 3), device=DEV))
    torch.cuda.synchronize()
    gs = grad.to_scene()
    rng = np.random.default_rng(0)
    worst = {}
    for field, width in FIELDS:
        ga = gs[field].reshape(sc[field].shape[0], -1)
        scale = np.abs(ga).max()
        # the largest entries of the group plus random ones
        big = np.argsort(-np.abs(ga).ravel(), kind="stable")[:12]
        pick = np.unique(np.concatenate([big, rng.choice(ga.size, 12, replace=False)]))
        errs, skipped = [], 0
        for flat_idx in pick:
            i, c = divmod(int(flat_idx), ga.shape[1])
            fd = []
            for h in (H_STEP, 0.5 * H_STEP):
                sp, xp = _perturbed(sc, field, i, c, h)
                sm, xm = _perturbed(sc, field, i, c, -h)
                fd.append((_loss(sp, cam, target) - _loss(sm, cam, target)) / (xp - xm))
            # the forward is not smooth everywhere (the 1/255 alpha cut-off, the sign
            # of the L1 error): where the differences at h and h/2 disagree, the
            # interval straddles such a kink and says nothing about the derivative
            if abs(fd[0] - fd[1]) > 5e-3 * scale:
                skipped += 1
                continue
            errs.append(abs(fd[0] - ga[i, c]) / scale)
        assert skipped <= len(pick) // 4, (field, skipped, len(pick))
        errs = np.sort(errs)
        worst[field] = errs[-1]
        # float32 rendering noise: every smooth entry within 1% of the group's
        # largest gradient
        assert errs[-1] <= 1e-2, (field, errs)
    assert all(np.isfinite(list(worst.values())))
