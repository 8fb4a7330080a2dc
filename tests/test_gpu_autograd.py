"""The rasterizer behind torch.autograd (RasterizeGaussians): a loss written in
torch differentiates through adp_render_backward.

- torch's own mean L1 loss (torch.nn.functional.l1_loss) on the 64-Gaussian 32x32
  sub-scene: torch.autograd.grad equals the oracle's complex-step gradient of the
  mean L1 loss within 2e-3 of each parameter group's largest entry;
- a weighted quadratic loss summed in float64 (a different upstream gradient)
  against central differences of the same autograd forward at h = 1e-3 and h / 2
  (entries where the two differences disagree straddle a kink of the forward and
  are left out, at most a quarter per group).
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.autograd import rasterize

pytestmark = pytest.mark.gpu

GROUPS = {"mean": slice(0, 3), "logit": slice(3, 4), "logscale": slice(4, 7),
          "quat": slice(7, 11), "sh": slice(11, 59)}


def _theta_of_planes(planes, n, deg):
    g = ops.Gaussians.__new__(ops.Gaussians)
    g.n, g.sh_degree, g.rows = n, deg, None
    g.mean_logit, g.logscale, g.quat, g.sh = (t.detach() for t in planes)
    return O.theta_of(g.to_scene())


def _subscene():
    sc, cam = scenes.subscene_for_gradients(0)
    tsc, _ = scenes.subscene_for_gradients(1, n=48)
    target = O.render(O.project(O.theta_of(tsc), 3, cam), cam)["rgb"].astype(np.float32)
    return sc, cam, target


def test_autograd_l1_matches_oracle_gradient():
    sc, cam, target = _subscene()
    g = ops.Gaussians.from_scene(sc, DEV)
    planes = [t.requires_grad_(True) for t in g.tensors()]
    img = rasterize(g, [cam])
    loss = torch.nn.functional.l1_loss(img, torch.as_tensor(target, device=DEV))
    grads = torch.autograd.grad(loss, planes)
    got = _theta_of_planes(grads, g.n, 3)
    ref = O.grad(O.theta_of(sc), 3, cam, target.reshape(32, 32, 3))
    for name, sl in GROUPS.items():
        tol = 2e-3 * np.abs(ref[:, sl]).max() + 1e-12
        err = np.abs(got[:, sl] - ref[:, sl]).max()
        assert err <= tol, (name, err, tol)
    assert np.abs(ref).max() > 0


def test_autograd_quadratic_loss_matches_central_differences():
    sc, cam, target = _subscene()
    tgt = torch.as_tensor(target, device=DEV)
    w = torch.linspace(0.5, 1.5, 3, device=DEV)

    def loss_of(planes):
        g = ops.Gaussians.__new__(ops.Gaussians)
        g.n, g.sh_degree, g.rows = planes[0].shape[0], 3, None
        g.mean_logit, g.logscale, g.quat, g.sh = planes
        img = rasterize(g, [cam])
        # summed in float64 so that rounding of the sum stays far below the
        # differences at h = 1e-3 (the cast back is differentiable)
        d = img.double() - tgt.double()
        return ((d * d) * w.double()).sum() / img.shape[0]

    g0 = ops.Gaussians.from_scene(sc, DEV)
    planes = [t.clone().requires_grad_(True) for t in g0.tensors()]
    grads = torch.autograd.grad(loss_of(planes), planes)
    ga = _theta_of_planes(grads, g0.n, 3)
    base = O.theta_of(sc)
    rng = np.random.default_rng(2)

    def loss_at(theta):
        s = O.scene_of_theta(theta, 3)
        with torch.no_grad():
            return float(loss_of(ops.Gaussians.from_scene(s, DEV).tensors()).double().item())

    for name, sl in GROUPS.items():
        cols = np.arange(sl.start, sl.stop)
        scale = np.abs(ga[:, sl]).max()
        sub = ga[:, sl]
        big = np.argsort(-np.abs(sub).ravel(), kind="stable")[:8]
        pick = np.unique(np.concatenate([big, rng.choice(sub.size, 8, replace=False)]))
        errs, skipped = [], 0
        for flat in pick:
            i, c = divmod(int(flat), sub.shape[1])
            col = cols[c]
            fd = []
            for h in (1e-3, 5e-4):
                tp, tm = base.copy(), base.copy()
                tp[i, col] = np.float32(tp[i, col] + h)
                tm[i, col] = np.float32(tm[i, col] - h)
                fd.append((loss_at(tp) - loss_at(tm)) / (tp[i, col] - tm[i, col]))
            if abs(fd[0] - fd[1]) > 5e-3 * scale:
                skipped += 1
                continue
            errs.append(abs(fd[0] - sub[i, c]) / scale)
        assert skipped <= len(pick) // 4, (name, skipped, len(pick))
        assert max(errs) <= 1e-2, (name, sorted(errs)[-3:])
