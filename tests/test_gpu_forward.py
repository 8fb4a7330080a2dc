"""GPU parity of projection, binning and compositing against the FP64 oracle.

Tolerances: colour max-abs <= 2e-4 on [0, 1], T within 1e-4, contributor counts
exact, except at tie pixels (a contributor's alpha within 1e-6 of 1/255 or of the
0.99 clamp, or a stop test within 1e-6 of 1e-4; for the dominant id also a weight
margin below 1e-6, where it must be one of the two best); every disagreement must
be at a tie and the excused pixels at most 1e-4 of the pixels. Integer work (tile
lists, ranges) bit-exact given identical keys.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import (DEV, c0_inputs, compare_render, gpu_forward, np_, oracle_projected_to_gpu,
                      small_cluster_inputs)
from paper_2605_06876_b300 import _abi, ops

pytestmark = pytest.mark.gpu


def _compare_render(img, ord_, label):
    return compare_render(np_(img.rgb), np_(img.T), np_(img.n_contrib), np_(img.dominant), ord_,
                          label)


def test_project_matches_oracle():
    sc, cams = small_cluster_inputs(5000, 200, 130, views=3)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    th = O.theta_of(sc)
    n = g.n
    for v, cam in enumerate(cams):
        o = O.project(th, 3, cam)
        sl = slice(v * n, (v + 1) * n)
        xyod, con, rgb = np_(pr.xyod[sl]), np_(pr.conic[sl]), np_(pr.rgb[sl])
        tiles, rect = np_(pr.tiles[sl]), np_(pr.rect[sl])
        vis = (o["tiles"] > 0) & (tiles > 0)
        # visibility agrees except at boxes grazing the image border
        assert (o["tiles"] > 0).sum() > 100
        assert np.mean((o["tiles"] > 0) != (tiles > 0)) < 1e-3
        np.testing.assert_allclose(xyod[vis, :2], o["mean2d"][vis], rtol=1e-5, atol=2e-3)
        np.testing.assert_allclose(xyod[vis, 2], o["opacity"][vis], rtol=1e-5)
        np.testing.assert_allclose(xyod[vis, 3], o["depth"][vis], rtol=1e-6)
        np.testing.assert_allclose(con[vis, :3], o["conic"][vis], rtol=2e-3,
                                   atol=2e-4 * np.abs(o["conic"][vis]).max())
        np.testing.assert_allclose(rgb[vis, :3], o["rgb"][vis], atol=2e-5)
        same = np.all(rect[vis] == o["rect"][vis], 1)
        assert same.mean() > 0.995


def _reaching(orp, ids, tx, ty, W, H):
    """Ids whose alpha (float32 records, FP64 arithmetic) reaches 1/255 at some
    pixel centre of tile (tx, ty): brute force over the tile's pixels."""
    xs = np.arange(tx * 16, min(tx * 16 + 16, W), dtype=np.float64)
    ys = np.arange(ty * 16, min(ty * 16 + 16, H), dtype=np.float64)
    X, Y = np.meshgrid(xs, ys)
    out = []
    for i in ids:
        mx, my = np.float32(orp["mean2d"][i]).astype(np.float64)
        A, B, C = np.float32(orp["conic"][i]).astype(np.float64)
        o = float(np.float32(orp["opacity"][i]))
        dx, dy = mx - X, my - Y
        a = o * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
        if a.max() >= 1 / 255 * (1 + 1e-5):
            out.append(i)
    return out


@pytest.mark.parametrize("views,n", [(1, 8000), (1, 20000), (3, 8000)])
def test_bin_sort_tile_lists_given_identical_keys(views, n):
    """Fed the oracle's own float32 records, every GPU tile list is the oracle's
    per-tile (depth, id) list by rectangle with the Gaussians that cannot reach
    the tile removed: it keeps the order, it is a subsequence of the rectangle
    list, and it contains every Gaussian whose alpha reaches 1/255 at one of the
    tile's pixel centres (brute force). The instance count is the rectangle
    count (capacity semantics). The sizes cover the one-block depth sort (8,000
    records) and the multi-launch radix passes with an even pass count (20,000)
    and, with the extra view pass, an odd one (3 x 8,000)."""
    sc, cams = small_cluster_inputs(n, 240, 160, views=views, seed=3)
    th = O.theta_of(sc)
    orps = [O.project(th, 3, c) for c in cams]
    assert th.shape[0] == n
    pr = oracle_projected_to_gpu(orps, n)
    bins = ops.bin_sort(n, pr, cams)
    torch.cuda.synchronize()
    inst, ranges = np_(bins.inst), np_(bins.ranges)
    K = int(bins.n_inst.item())
    assert K == sum(int(o["tiles"].sum()) for o in orps)
    t0 = 0
    kept = total = 0
    for v, cam in enumerate(cams):
        W, H = cam["width"], cam["height"]
        tx, ty = (W + 15) // 16, (H + 15) // 16
        start, ref = O.tile_lists(orps[v]["depth"].astype(np.float32), orps[v]["rect"],
                                  orps[v]["tiles"], tx, ty)
        for t in range(tx * ty):
            s_, e = ranges[t0 + t]
            got = list(inst[s_:e]) if e > s_ else []
            full = list(ref[start[t]:start[t + 1]])
            it = iter(full)
            assert all(g in it for g in got), (v, t)  # ordered subsequence
            need = _reaching(orps[v], full, t % tx, t // tx, W, H)
            assert set(need) <= set(got), (v, t, set(need) - set(got))
            kept += len(got)
            total += len(full)
        t0 += tx * ty
    assert kept < total  # the rectangle overestimates rotated ellipses


def test_bin_sort_overflow_reports_required_capacity():
    sc, cams = small_cluster_inputs(3000, 160, 96, seed=4)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    need = int(pr.tiles.sum().item())
    small = ops.Bins.alloc(need // 2, ops.n_tiles(cams), DEV)
    ops.bin_sort(g.n, pr, cams, bins=small, grow=False)
    torch.cuda.synchronize()
    assert int(small.n_inst.item()) == need
    assert int(np_(small.ranges).max()) == 0  # nothing binned past the capacity
    full = ops.bin_sort(g.n, pr, cams)
    assert int(full.n_inst.item()) == need


def test_render_c0_matches_oracle():
    sc, cam, _ = c0_inputs()
    g, pr, bins, img = gpu_forward(sc, [cam])
    o = O.render(O.project(O.theta_of(sc), 0, cam), cam)
    _compare_render(img, o, "tiny workload 128x128")


def test_render_stage_isolated_and_background():
    """Given the oracle's records (float32), compositing agrees with the oracle
    per pixel, with a non-black background."""
    sc, cams = small_cluster_inputs(20000, 320, 208, seed=5)
    cam = cams[0]
    th = O.theta_of(sc)
    orp = O.project(th, 3, cam)
    n = th.shape[0]
    pr = oracle_projected_to_gpu([orp], n)
    bg = (0.2, 0.5, 0.8)
    bins = ops.bin_sort(n, pr, cams)
    img = ops.render(n, pr, bins, cams, bg)
    torch.cuda.synchronize()
    # the oracle composites the same float32-rounded records in FP64
    orp32 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype == np.float64 else v)
             for k, v in orp.items()}
    _compare_render(img, O.render(orp32, cam, bg=bg), "20k Gaussians 320x208, oracle records")


@pytest.mark.parametrize("shape", [(8, 32), (32, 8)])
def test_tile_shape_invariance(shape):
    """The per-pixel contributor sequence does not depend on the tiling, so other
    tile shapes give bit-identical images and dominant maps."""
    sc, cams = small_cluster_inputs(20000, 330, 210, seed=6)
    _, _, _, ref = gpu_forward(sc, cams)
    p = _abi.default_params(tile_w=shape[0], tile_h=shape[1])
    _, _, _, got = gpu_forward(sc, cams, p)
    for a, b in zip((ref.rgb, ref.T, ref.dominant, ref.n_contrib),
                    (got.rgb, got.T, got.dominant, got.n_contrib)):
        assert torch.equal(a, b)


def test_batched_views_equal_views_alone():
    """Each view of a multi-view launch equals that view rendered alone, bitwise."""
    sc, cams = small_cluster_inputs(20000, 256, 160, views=4, seed=7)
    cams[1] = scenes.camera_look_at((0, -2, -4), (0, 0, 0), 300, 180)
    _, _, _, allv = gpu_forward(sc, cams)
    off = 0
    for cam in cams:
        _, _, _, one = gpu_forward(sc, [cam])
        P = cam["width"] * cam["height"]
        assert torch.equal(allv.rgb[off:off + P], one.rgb)
        assert torch.equal(allv.dominant[off:off + P], one.dominant)
        off += P


def test_full_size_sampled_pixels():
    """1M Gaussians at 1280x832 (the single-view workload): 400 sampled pixels
    agree with the oracle's brute-force per-pixel compositing over all Gaussians."""
    cfg = scenes.CONFIGS[1]
    sc = scenes.scene_clusters(2, cfg["n"], cfg["sh_degree"])
    cam = scenes.ring_cameras(3, 1, cfg["ring_radius"], cfg["width"], cfg["height"])[0]
    g, pr, bins, img = gpu_forward(sc, [cam])
    rng = np.random.default_rng(0)
    pix = rng.choice(cfg["width"] * cfg["height"], 400, replace=False)
    o = O.render(O.project(O.theta_of(sc), 3, cam), cam, pixels=pix)
    sub = ops.Image(*(t[torch.as_tensor(pix, device=DEV)] for t in
                      (img.rgb, img.T, img.n_contrib, img.last, img.dominant)))
    _compare_render(sub, o, "1M Gaussians 1280x832, sampled")


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_multi_view_projection_equals_single_view(deg):
    """The several-view projection kernel (one screening of each Gaussian for all
    views, survivors projected per block) against the one-view kernel, per SH
    degree: every view's records, bit for bit."""
    sc = scenes.scene_clusters(60 + deg, 30000, deg)
    cams = scenes.ring_cameras(61, 3, 4.0, 160, 96)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    torch.cuda.synchronize()
    n = g.n
    for v, cam in enumerate(cams):
        p1 = ops.project(g, [cam])
        torch.cuda.synchronize()
        t1 = np_(p1.tiles)
        assert np.array_equal(t1, np_(pr.tiles)[v * n:(v + 1) * n])
        vis = t1 > 0
        assert vis.sum() > 1000
        for name in ("xyod", "conic", "rgb", "rect"):
            a = np_(getattr(p1, name))[:n][vis]
            b = np_(getattr(pr, name))[v * n:(v + 1) * n][vis]
            assert np.array_equal(a, b), (v, name)


def test_large_binning_equals_per_view_binning():
    """16 views of 150,000 Gaussians (2.4M records, one launch of every binning
    kernel over all views): every (view, tile) list equals that view's list binned
    alone, entry for entry."""
    sc = scenes.scene_clusters(70, 150_000, 3)
    cams = scenes.ring_cameras(71, 16, 4.0, 320, 208)
    g = ops.Gaussians.from_scene(sc, DEV)
    assert g.n * len(cams) >= 1 << 21
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    torch.cuda.synchronize()
    ranges = np_(bins.ranges).reshape(-1, 2)
    inst = np_(bins.inst)
    per_view_tiles = ranges.shape[0] // len(cams)
    for v, cam in enumerate(cams):
        p1 = ops.project(g, [cam])
        b1 = ops.bin_sort(g.n, p1, [cam])
        torch.cuda.synchronize()
        r1 = np_(b1.ranges).reshape(-1, 2)
        i1 = np_(b1.inst)
        assert r1.shape[0] == per_view_tiles
        for t in range(per_view_tiles):
            a0, a1 = ranges[v * per_view_tiles + t]
            c0, c1 = r1[t]
            assert np.array_equal(inst[a0:a1], i1[c0:c1]), (v, t)
