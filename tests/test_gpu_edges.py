"""Degenerate inputs of the plain step through every entry point, against the FP64
oracle where it applies and against what the case fixes otherwise:

- no Gaussian at all: every call succeeds, the image is the background, nothing is
  counted, selected, labelled or split, and the new population is empty;
- every Gaussian behind the camera: the background image, zero counts and masses,
  the top-k of all-equal masses (the lowest ids), and the oracle's split;
- no candidate (k = 0) and every Gaussian a candidate (k = n);
- ragged images (1x1, 17x3), smaller than one tile.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, compare_render, np_
from paper_2605_06876_b300 import ops

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)


def _gpu_plain(sc, cams, target, k, noise):
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams, BG)
    maps, count, mass = ops.error_stats(img.rgb, target, img.dominant, g.n, cams)
    cand = ops.select_topk(mass, g.n, k)
    regs = ops.error_regions(maps, img.dominant, target, g.n, cams, cand)
    plan = ops.split_plan(g, cams, regs, cand, count)
    out, _, _ = ops.split_apply(g, plan, regs, cand, noise, with_state=False)
    grad = ops.render_backward(g, pr, bins, img, cams, bg=BG, target=target)
    m, v = g.zeros_like(), g.zeros_like()
    ops.adam_step(g, grad, m, v, 1)
    torch.cuda.synchronize()
    return dict(g=g, g0=ops.Gaussians.from_scene(sc, DEV), img=img, maps=maps, count=count,
                mass=mass, cand=cand, regs=regs, plan=plan, out=out, grad=grad)


def _targets(cams, seed):
    rng = np.random.default_rng(seed)
    return [rng.random((c["height"], c["width"], 3)).astype(np.float32) for c in cams]


def _check_against_oracle(sc, cams, targets, k, r, noise):
    """The GPU step against the oracle's. The full GPU path: its image per view
    (tie-excused) and its masses within float32 rounding of the image. Then,
    stage-isolated from the oracle's own float32 image and dominant map (so both
    sides decide from the same values): the counts, masses, candidates, region
    table, statuses, child counts and the new population (kept rows bit for bit,
    appended rows within the split's bounds)."""
    orc = O.plain_step(sc, cams, targets, k_cand=k, noise=noise.astype(np.float64), bg=BG)
    n = sc["mean"].shape[0]
    off = 0
    for v, cam in enumerate(cams):
        P = cam["width"] * cam["height"]
        img = r["img"]
        o = orc["views"][v]["render"]
        compare_render(np_(img.rgb)[off:off + P], np_(img.T)[off:off + P],
                       np_(img.n_contrib)[off:off + P], np_(img.dominant)[off:off + P], o,
                       f"view {v}")
        off += P
    np.testing.assert_allclose(np_(r["mass"])[:n], orc["mass"], rtol=1e-4, atol=1e-6)
    # stage-isolated from the oracle's image
    g = r["g0"]
    img_o = torch.as_tensor(np.concatenate([vw["img32"].reshape(-1, 3) for vw in orc["views"]]),
                            device=DEV)
    dom_o = torch.as_tensor(np.concatenate([vw["render"]["dominant"] for vw in orc["views"]])
                            .astype(np.int32), device=DEV)
    tgt = torch.as_tensor(np.concatenate([t.reshape(-1, 3) for t in targets]), device=DEV)
    maps, count, mass = ops.error_stats(img_o, tgt, dom_o, n, cams)
    cand = ops.select_topk(mass, n, k)
    regs = ops.error_regions(maps, dom_o, tgt, n, cams, cand)
    plan = ops.split_plan(g, cams, regs, cand, count)
    out, _, _ = ops.split_apply(g, plan, regs, cand, torch.as_tensor(noise, device=DEV),
                                with_state=False)
    torch.cuda.synchronize()
    assert np.array_equal(np_(count)[:n], orc["count"])
    assert np.array_equal(np_(mass)[:n], orc["mass"])
    assert np.array_equal(np_(cand)[:k], orc["cand"])
    rgs, rg = regs.to_numpy(), orc["regions"]
    for key in ("view", "parent", "label", "band", "moments"):
        assert np.array_equal(rgs[key], rg[key]), key
    sp = orc["split"]
    assert np.array_equal(np_(plan.status), sp["status"])
    assert np.array_equal(np_(plan.n_children), sp["n_children"])
    assert plan.new_n == sp["new_n"] == out.n
    got, ref = O.theta_of(out.to_scene()), sp["theta"]
    cl = orc["cand"].tolist()
    nk = sum(1 for i in range(n) if i not in set(cl) or sp["status"][cl.index(i)] == O.RESET)
    assert np.array_equal(got[:nk], ref[:nk])
    np.testing.assert_allclose(got[nk:, :4], ref[nk:, :4], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(got[nk:, 11:], ref[nk:, 11:], rtol=1e-5, atol=1e-5)
    return orc


def test_no_gaussian():
    sc = scenes.scene_box(0, 50, 0)
    sc = {k: (v[:0] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    cams = [scenes.camera_origin_forward(40, 24)]
    target = torch.as_tensor(_targets(cams, 1)[0].reshape(-1, 3), device=DEV)
    r = _gpu_plain(sc, cams, target, 0, torch.zeros((1, 2, 3), device=DEV))
    want = torch.tensor(BG, device=DEV).expand(40 * 24, 3)
    assert torch.equal(r["img"].rgb, want)
    assert torch.equal(r["img"].T, torch.ones(40 * 24, device=DEV))
    assert bool((r["img"].dominant == -1).all()) and bool((r["img"].n_contrib == 0).all())
    assert int(r["regs"].count.item()) == 0
    assert r["plan"].new_n == 0 and r["out"].n == 0


def test_every_gaussian_behind_the_camera():
    sc = scenes.scene_box(2, 400, 0)
    sc = dict(sc, mean=(sc["mean"] - np.float32([0, 0, 12])).astype(np.float32))
    cams = [scenes.camera_origin_forward(48, 40)]
    targets = _targets(cams, 3)
    k = 40
    noise = scenes.fallback_noise(4, k)
    r = _gpu_plain(sc, cams, torch.as_tensor(targets[0].reshape(-1, 3), device=DEV), k,
                   torch.as_tensor(noise, device=DEV))
    want = torch.tensor(BG, device=DEV).expand(48 * 40, 3)
    assert torch.equal(r["img"].rgb, want)
    assert not bool(r["count"][:400].any()) and not bool(r["mass"][:400].any())
    assert np.array_equal(np_(r["cand"])[:k], np.arange(k, dtype=np.int32))  # ties: lowest ids
    assert not any(bool(t.any()) for t in r["grad"].tensors())  # nothing rendered
    _check_against_oracle(sc, cams, targets, k, r, noise)


@pytest.mark.parametrize("k", [0, 300])
def test_no_candidate_and_every_gaussian_a_candidate(k):
    sc = scenes.scene_box(5, 300, 0)
    cams = [scenes.camera_origin_forward(64, 48)]
    targets = _targets(cams, 6)
    noise = scenes.fallback_noise(7, max(k, 1))
    r = _gpu_plain(sc, cams, torch.as_tensor(targets[0].reshape(-1, 3), device=DEV), k,
                   torch.as_tensor(noise, device=DEV))
    if k == 0:
        assert r["plan"].new_n == 300
        for a, b in zip(r["out"].tensors(), ops.Gaussians.from_scene(sc, DEV).tensors()):
            assert torch.equal(a, b)
    _check_against_oracle(sc, cams, targets, k, r, noise)


@pytest.mark.parametrize("size", [(1, 1), (17, 3), (3, 17)])
def test_ragged_images_smaller_than_a_tile(size):
    W, H = size
    sc = scenes.scene_box(8, 600, 0)
    cams = [scenes.camera_origin_forward(W, H)]
    targets = _targets(cams, 9)
    k = 30
    noise = scenes.fallback_noise(10, k)
    r = _gpu_plain(sc, cams, torch.as_tensor(targets[0].reshape(-1, 3), device=DEV), k,
                   torch.as_tensor(noise, device=DEV))
    _check_against_oracle(sc, cams, targets, k, r, noise)
