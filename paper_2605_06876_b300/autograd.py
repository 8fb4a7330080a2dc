"""torch.autograd.Function around the rasterizer: the forward is adp_project,
adp_bin_sort and adp_render; the backward is adp_render_backward fed with the
upstream gradient dL/d(image), so any loss written in torch (the baselines' L1,
D-SSIM or another) differentiates through the hand-written kernels. The
Gaussian parameters are the four float4 plane tensors of ops.Gaussians."""
from __future__ import annotations

import torch

from . import _abi as A
from . import ops


class RasterizeGaussians(torch.autograd.Function):
    """image = rasterize(mean_logit, logscale, quat, sh) for fixed cameras.

    Inputs: mean_logit, logscale, quat [n, 4], sh [planes, n, 4] (float32,
    CUDA, contiguous); cams (camera dicts), params (AdpParams or None), bg (3
    floats). Output: the image of every view, [sum of W*H, 3], views
    concatenated row-major. Non-differentiable outputs of the forward (tile
    bins, transmittance, dominant map) are kept for the backward only."""

    @staticmethod
    def forward(ctx, mean_logit, logscale, quat, sh, cams, params, bg):
        n = mean_logit.shape[0]
        deg = {1: 0, 3: 1, 7: 2, 12: 3}[sh.shape[0]]
        g = ops.Gaussians.__new__(ops.Gaussians)
        g.n, g.sh_degree, g.rows = n, deg, None
        g.mean_logit, g.logscale, g.quat, g.sh = (mean_logit.detach(), logscale.detach(),
                                                  quat.detach(), sh.detach())
        params = params or A.default_params()
        pr = ops.project(g, cams, params)
        bins = ops.bin_sort(n, pr, cams, params)
        img = ops.render(n, pr, bins, cams, bg, params)
        ctx.state = (g, pr, bins, img, cams, params, bg)
        return img.rgb.clone()

    @staticmethod
    def backward(ctx, grad_rgb):
        g, pr, bins, img, cams, params, bg = ctx.state
        grad = ops.render_backward(g, pr, bins, img, cams, dL_drgb=grad_rgb.contiguous(), bg=bg,
                                   params=params)
        ctx.state = None
        return grad.mean_logit, grad.logscale, grad.quat, grad.sh, None, None, None


def rasterize(g: ops.Gaussians, cams, params=None, bg=(0.0, 0.0, 0.0)):
    """The differentiable image of g's planes (set requires_grad on them first)."""
    return RasterizeGaussians.apply(g.mean_logit, g.logscale, g.quat, g.sh, list(cams), params,
                                    tuple(float(x) for x in bg))
