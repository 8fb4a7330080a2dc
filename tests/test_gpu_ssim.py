"""GPU parity of the D-SSIM loss term and its gradient against the FP64 oracle, on
two views of uneven, ragged sizes and at the full 1280x832 size; the gradient feeds
the backward through its upstream-gradient input."""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, np_
from paper_2605_06876_b300 import ops

pytestmark = pytest.mark.gpu


def _images(seed, W, H):
    img, tgt, _ = scenes.error_stage_inputs(seed, W, H, 1)
    return img.reshape(-1, 3), tgt.reshape(-1, 3)


@pytest.mark.parametrize("sizes", [[(97, 61), (40, 33)], [(1280, 832)]])
def test_dssim_matches_the_oracle(sizes):
    cams, imgs, tgts = [], [], []
    for v, (W, H) in enumerate(sizes):
        cams.append(scenes.camera_origin_forward(W, H))
        i, t = _images(50 + v, W, H)
        imgs.append(i)
        tgts.append(t)
    lam = 0.2
    dL, loss = ops.dssim_loss_grad(torch.as_tensor(np.concatenate(imgs), device=DEV),
                                   torch.as_tensor(np.concatenate(tgts), device=DEV), cams, lam)
    torch.cuda.synchronize()
    got, got_loss = np_(dL), np_(loss)
    off = 0
    for v, (W, H) in enumerate(sizes):
        l1, s, g, scale = O.dssim_loss_grad(imgs[v], tgts[v], W, H, lam, return_scale=True)
        P = W * H
        gv = got[off:off + P]
        # the three window-sum terms of each entry nearly cancel in smooth regions, so
        # a float32 result is exact to a small multiple of their summed magnitude
        # (float32 rounding is 6e-8; 121-term window sums and a few products on top)
        err = np.abs(gv - g)
        bound = 2e-5 * scale + 1e-3 * (1 - lam) / (3.0 * P) * 1e-3
        assert np.all(err <= bound), (v, (err / np.maximum(scale, 1e-30)).max())
        np.testing.assert_allclose(got_loss[v][0], l1, rtol=1e-5)
        # the variance terms q11 - m1^2 lose up to float32 rounding (6e-8) times m1^2
        # (about 0.25) against C2 = 9e-4: about 2e-5 of each pixel's SSIM
        np.testing.assert_allclose(got_loss[v][1], s, rtol=5e-5)
        off += P


def test_backward_takes_the_dssim_gradient():
    from gpu_util import small_cluster_inputs

    sc, cams = small_cluster_inputs(3000, 128, 96, seed=52)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams)
    _, tgt = _images(53, 128, 96)
    tgt = torch.as_tensor(tgt, device=DEV)
    # lambda = 0 reduces to the built-in L1 gradient
    dL0, _ = ops.dssim_loss_grad(img.rgb, tgt, cams, 0.0)
    a = ops.render_backward(g, pr, bins, img, cams, dL_drgb=dL0)
    b = ops.render_backward(g, pr, bins, img, cams, target=tgt)
    dL, _ = ops.dssim_loss_grad(img.rgb, tgt, cams, 0.2)
    c = ops.render_backward(g, pr, bins, img, cams, dL_drgb=dL)
    torch.cuda.synchronize()
    for ta, tb, tc in zip(a.tensors(), b.tensors(), c.tensors()):
        sc_ = tb.abs().max().item() + 1e-30
        assert (ta - tb).abs().max().item() <= 1e-5 * sc_
        assert torch.isfinite(tc).all()
    assert any((tc - tb).abs().max().item() > 1e-3 * (tb.abs().max().item() + 1e-30)
               for tb, tc in zip(b.tensors(), c.tensors()))


def test_plain_step_with_the_dssim_loss_replays():
    from gpu_util import small_cluster_inputs
    from paper_2605_06876_b300.pipeline import PlainStep

    sc, cams = small_cluster_inputs(8000, 160, 112, seed=54)
    tg = ops.Gaussians.from_scene(scenes.scene_clusters(55, 12000, 3), DEV)
    prt = ops.project(tg, cams)
    target = ops.render(tg.n, prt, ops.bin_sort(tg.n, prt, cams), cams).rgb.clone()
    st = PlainStep(ops.Gaussians.from_scene(sc, DEV), cams, target, 0.1, dssim_lambda=0.2)
    noise = torch.as_tensor(scenes.fallback_noise(56, st.k), device=DEV)
    st.step(noise)
    torch.cuda.synchronize()
    first = np_(st.loss).copy()
    assert 0.0 < first[0, 0] < 1.0 and 0.0 < first[0, 1] < 1.0
    st.capture(noise)
    st.replay()
    torch.cuda.synchronize()
    # the replayed step renders the Adam-updated scene: a loss of the same order
    again = np_(st.loss)
    assert np.all(np.isfinite(again)) and abs(again[0, 1] - first[0, 1]) < 0.05
