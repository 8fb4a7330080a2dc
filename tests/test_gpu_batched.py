"""GPU parity of the batched step (adp_train_step_batched): one persistent fused
forward + L1-error + backward kernel over the (view, tile) work queue of many
views of uneven size.

- Against the one-stage calls on the same views: projection, bins, image,
  dominant map, error maps, counts and masses bit for bit; the gradient (float
  atomics in another order) within 1e-5 of each parameter group's largest entry.
- Each view of the batch against the view launched alone: image and error maps
  bit for bit (the raw L1 min/max are per view).
- Against the FP64 oracle: the gradient of a two-view 64-Gaussian sub-scene (the
  sum of the views' mean L1 losses) within 2e-3 of each group's largest entry,
  and sampled pixels of the 3M-Gaussian, 16-view uneven workload.
- A replay of the captured graph reproduces the eager call.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, compare_render, np_, small_cluster_inputs
from paper_2605_06876_b300 import _abi as A
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.pipeline import BatchedStep

pytestmark = pytest.mark.gpu

GROUPS = {"mean": slice(0, 3), "logit": slice(3, 4), "logscale": slice(4, 7),
          "quat": slice(7, 11), "sh": slice(11, 59)}


def _uneven_cams(seed=31):
    _, cams = small_cluster_inputs(10, 320, 208, views=2, seed=seed)
    cams.append(scenes.camera_look_at((0, -2.5, -3.5), (0, 0, 0), 211, 133))
    cams.append(scenes.camera_look_at((3.0, 0.5, -2.0), (0, 0, 0), 144, 260))
    return cams


def _target(cams, seed=32, n=30000):
    tg = ops.Gaussians.from_scene(scenes.scene_clusters(seed, n, 3), DEV)
    prt = ops.project(tg, cams)
    return ops.render(tg.n, prt, ops.bin_sort(tg.n, prt, cams), cams).rgb.clone()


def _separate(g, cams, target, params=None):
    """The one-stage calls on the same views."""
    pr = ops.project(g, cams, params)
    bins = ops.bin_sort(g.n, pr, cams, params)
    img = ops.render(g.n, pr, bins, cams, params=params)
    maps, count, mass = ops.error_stats(img.rgb, target, img.dominant, g.n, cams, params)
    grad = ops.render_backward(g, pr, bins, img, cams, target=target, params=params,
                               grad=ops.Gaussians(g.n, g.sh_degree, DEV, zero=False,
                                                  row_mask=True))
    torch.cuda.synchronize()
    return pr, bins, img, maps, count, mass, grad


def _grad_close(a, b, rel):
    ta, tb = O.theta_of(a.dense().to_scene()), O.theta_of(b.dense().to_scene())
    for name, sl in GROUPS.items():
        tol = rel * np.abs(tb[:, sl]).max() + 1e-12
        err = np.abs(ta[:, sl] - tb[:, sl]).max()
        assert err <= tol, (name, err, tol)


@pytest.mark.parametrize("batch", [256, 64])
def test_batched_equals_the_one_stage_calls(batch):
    sc, _ = small_cluster_inputs(20000, 8, 8, seed=30)
    cams = _uneven_cams()
    target = _target(cams)
    g = ops.Gaussians.from_scene(sc, DEV)
    params = A.default_params(batch=batch)
    status = ops.status_word(DEV)
    pr, bins, img, maps, count, mass, grad = ops.train_step_batched(g, cams, target, params,
                                                                    status=status)
    torch.cuda.synchronize()
    ops.check_status(status)
    r = _separate(g, cams, target, params)
    K = int(r[1].n_inst.item())
    assert int(bins.n_inst.item()) == K
    assert torch.equal(bins.ranges, r[1].ranges) and torch.equal(bins.inst[:K], r[1].inst[:K])
    for x, y in zip((img.rgb, img.T, img.n_contrib, img.last, img.dominant),
                    (r[2].rgb, r[2].T, r[2].n_contrib, r[2].last, r[2].dominant)):
        assert torch.equal(x, y)
    for x, y in zip((maps.E, maps.mask, maps.minmax), (r[3].E, r[3].mask, r[3].minmax)):
        assert torch.equal(x, y)
    assert torch.equal(count, r[4]) and torch.equal(mass, r[5])
    assert torch.equal(grad.rows, r[6].rows)
    _grad_close(grad, r[6], 1e-5)


def test_each_view_of_the_batch_equals_the_view_alone():
    sc, _ = small_cluster_inputs(20000, 8, 8, seed=33)
    cams = _uneven_cams(34)
    target = _target(cams, 35)
    g = ops.Gaussians.from_scene(sc, DEV)
    _, _, img, maps, count, mass, grad = ops.train_step_batched(g, cams, target)
    torch.cuda.synchronize()
    off = 0
    grads = []
    for cam in cams:
        P = cam["width"] * cam["height"]
        _, _, i1, m1, _, _, g1 = ops.train_step_batched(g, [cam], target[off:off + P])
        torch.cuda.synchronize()
        assert torch.equal(img.rgb[off:off + P], i1.rgb)
        assert torch.equal(img.dominant[off:off + P], i1.dominant)
        assert torch.equal(maps.E[off:off + P], m1.E) and torch.equal(maps.mask[off:off + P], m1.mask)
        grads.append(O.theta_of(g1.dense().to_scene()))
        off += P
    # the views' mean L1 losses add up, and so do their gradients
    total = O.theta_of(grad.dense().to_scene())
    summed = np.sum(grads, axis=0)
    for name, sl in GROUPS.items():
        tol = 1e-4 * np.abs(summed[:, sl]).max() + 1e-12
        assert np.abs(total[:, sl] - summed[:, sl]).max() <= tol, name


def test_batched_gradient_matches_oracle_two_views():
    """64 Gaussians seen by two 32x32 cameras: the gradient of the sum of the two
    views' mean L1 losses against the sum of the oracle's complex-step gradients."""
    sc, cam = scenes.subscene_for_gradients(0)
    cam2 = scenes.camera_look_at((0.4, -0.2, 0.1), (0.0, 0.0, 3.2), 32, 32)
    cams = [cam, cam2]
    tsc, _ = scenes.subscene_for_gradients(1, n=48)
    th_t, th = O.theta_of(tsc), O.theta_of(sc)
    targets = [O.render(O.project(th_t, 3, c), c)["rgb"].astype(np.float32) for c in cams]
    g = ops.Gaussians.from_scene(sc, DEV)
    tgt = torch.as_tensor(np.concatenate(targets), device=DEV)
    *_, grad = ops.train_step_batched(g, cams, tgt)
    torch.cuda.synchronize()
    got = O.theta_of(grad.dense().to_scene())
    ref = sum(O.grad(th, 3, c, t.reshape(32, 32, 3)) for c, t in zip(cams, targets))
    for name, sl in GROUPS.items():
        tol = 2e-3 * np.abs(ref[:, sl]).max() + 1e-12
        assert np.abs(got[:, sl] - ref[:, sl]).max() <= tol, (name, np.abs(got[:, sl] - ref[:, sl]).max(), tol)
    assert np.abs(ref).max() > 0


def test_captured_batched_step_replays_the_eager_one():
    sc, _ = small_cluster_inputs(20000, 8, 8, seed=36)
    cams = _uneven_cams(37)
    target = _target(cams, 38)
    g = ops.Gaussians.from_scene(sc, DEV)
    st = BatchedStep(g, cams, target)
    st.run()
    torch.cuda.synchronize()
    ref = (st.img.rgb.clone(), st.maps.E.clone(), st.count.clone(), st.mass.clone(),
           st.grad.dense())
    st.img.rgb.zero_()
    st.maps.E.zero_()
    st.capture()
    st.replay()
    st.replay()
    torch.cuda.synchronize()
    assert st.fits()
    assert torch.equal(st.img.rgb, ref[0]) and torch.equal(st.maps.E, ref[1])
    assert torch.equal(st.count, ref[2]) and torch.equal(st.mass, ref[3])
    _grad_close(st.grad, ref[4], 1e-5)


def test_batched_3m_uneven_16_views_sampled_pixels():
    """The batched-views workload: 3,000,000 Gaussians, 16 cameras on a radius-5
    hemisphere with resolutions between 640x416 and 1600x1056, in one fused call.
    Its image equals the one-stage render of the same launch, and sampled pixels
    of the smallest and the largest view match the oracle's brute force."""
    cfg = scenes.CONFIGS[3]
    sc = scenes.scene_clusters(6, cfg["n"], cfg["sh_degree"])
    res = scenes.uneven_resolutions(7, cfg["views"])
    cams = scenes.hemisphere_cameras(7, cfg["views"], cfg["hemisphere_radius"], res)
    g = ops.Gaussians.from_scene(sc, DEV)
    P = ops.n_pixels(cams)
    target = torch.rand((P, 3), device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    pr, bins, img, maps, count, mass, grad = ops.train_step_batched(g, cams, target)
    torch.cuda.synchronize()
    assert int(bins.n_inst.item()) <= bins.capacity
    ref = ops.render(g.n, pr, bins, cams)
    torch.cuda.synchronize()
    assert torch.equal(img.rgb, ref.rgb) and torch.equal(img.dominant, ref.dominant)
    del ref, grad
    offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    sizes = [c["width"] * c["height"] for c in cams]
    theta = O.theta_of(sc)
    rng = np.random.default_rng(5)
    for v in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        cam = cams[v]
        pix = rng.choice(sizes[v], 60, replace=False)
        o = O.render(O.project(theta, 3, cam), cam, pixels=pix)
        idx = torch.as_tensor(offs[v] + pix, device=DEV)
        compare_render(np_(img.rgb[idx]), np_(img.T[idx]), np_(img.n_contrib[idx]),
                       np_(img.dominant[idx]), o,
                       f"batched 3M Gaussians, view {v} {cam['width']}x{cam['height']}")


def _one_stage_image(g, cams, target, bg):
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams, bg)
    maps, count, mass = ops.error_stats(img.rgb, target, img.dominant, g.n, cams)
    torch.cuda.synchronize()
    return img, maps, count, mass


@pytest.mark.parametrize("case", ["empty", "behind", "one_pixel", "max_views"])
def test_batched_edge_cases(case):
    """Degenerate inputs of the batched call against the one-stage calls: no
    Gaussian at all, every Gaussian behind every camera, a 1x1 view beside ragged
    ones, and the maximum number of views (ADP_MAX_VIEWS, small ones)."""
    bg = (0.25, 0.5, 0.75)
    sc, _ = small_cluster_inputs(4000, 8, 8, seed=40)
    if case == "empty":
        sc = {k: (v[:0] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        cams = _uneven_cams(41)
    elif case == "behind":
        sc = dict(sc, mean=(sc["mean"] * np.float32(0.1) + np.float32([0, 0, -30])).astype(np.float32))
        cams = [scenes.camera_origin_forward(97, 61), scenes.camera_origin_forward(64, 64)]
    elif case == "one_pixel":
        cams = [scenes.camera_look_at((0, 0, -4), (0, 0, 0), 1, 1),
                scenes.camera_look_at((0.3, 0, -4), (0, 0, 0), 37, 19)]
    else:
        cams = [scenes.camera_look_at((4 * np.cos(a), -0.5, 4 * np.sin(a)), (0, 0, 0), 48, 32)
                for a in np.linspace(0, 2 * np.pi, A.ADP_MAX_VIEWS, endpoint=False)]
    P = ops.n_pixels(cams)
    target = torch.rand((P, 3), device=DEV, generator=torch.Generator(DEV).manual_seed(4))
    g = ops.Gaussians.from_scene(sc, DEV)
    status = ops.status_word(DEV)
    pr, bins, img, maps, count, mass, grad = ops.train_step_batched(g, cams, target, bg=bg,
                                                                    status=status)
    torch.cuda.synchronize()
    ops.check_status(status)
    ref, rmaps, rcount, rmass = _one_stage_image(g, cams, target, bg)
    for x, y in zip((img.rgb, img.T, img.n_contrib, img.dominant), (ref.rgb, ref.T, ref.n_contrib,
                                                                     ref.dominant)):
        assert torch.equal(x, y)
    assert torch.equal(maps.E, rmaps.E) and torch.equal(maps.mask, rmaps.mask)
    if g.n:
        assert torch.equal(count, rcount) and torch.equal(mass, rmass)
    if case in ("empty", "behind"):  # nothing rendered: the background everywhere
        want = torch.tensor(bg, device=DEV).expand(P, 3)
        assert torch.equal(img.rgb, want) and bool((img.dominant == -1).all())
        if g.n:
            assert not bool(grad.rows.any()) and not bool(count.any())


def test_batched_instance_overflow_is_reported():
    """Too small an instance capacity (1,024 for about a million instances): the
    call runs to its end without a device error, writes nothing past the capacity
    and reports the count it needs, which equals the count an ample capacity sees."""
    sc, _ = small_cluster_inputs(20000, 8, 8, seed=44)
    cams = _uneven_cams(45)
    target = _target(cams, 46)
    g = ops.Gaussians.from_scene(sc, DEV)
    small = BatchedStep(g, cams, target, bins_margin=0.0)
    assert small.bins.capacity == 1024
    small.run()
    torch.cuda.synchronize()
    assert not small.fits()  # fits() also checks the status word
    ample = BatchedStep(g, cams, target)
    ample.run()
    torch.cuda.synchronize()
    assert ample.fits()
    assert int(small.bins.n_inst.item()) == int(ample.bins.n_inst.item()) > 1024
