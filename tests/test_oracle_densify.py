"""Pins of the oracle's densification pieces (Sec. 3, Eq. 2): the image-space
gradient against central differences of the oracle's own real-valued render, the
NDC scaling, and the split/clone rule on hand-built cases."""
import math

import numpy as np

import oracle as O
import scenes


def _l1(proj, cam, target):
    r = O.render(proj, cam)
    return float(np.abs(r["rgb"] - target.reshape(-1, 3)).sum() / target.size)


def test_mean2d_gradient_matches_central_differences_of_the_render():
    sc, cam = scenes.subscene_for_gradients(2, n=24)
    tsub, _ = scenes.subscene_for_gradients(3, n=16)
    target = O.render(O.project(O.theta_of(tsub), 3, cam), cam)["rgb"].astype(np.float32)
    theta = O.theta_of(sc)
    proj = O.project(theta, 3, cam)
    vis = np.nonzero(proj["tiles"] > 0)[0][:8].astype(np.int32)
    _, m2 = O.grad(theta, 3, cam, target, sel=vis, return_mean2d=True)
    h = 1e-6
    checked = 0
    for r, i in enumerate(vis):
        for c in range(2):
            fd = []
            for sgn in (1.0, -1.0):
                p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in proj.items()}
                p["mean2d"][i, c] += sgn * h
                fd.append(_l1(p, cam, target))
            d = (fd[0] - fd[1]) / (2 * h)
            assert abs(d - m2[r, c]) <= 1e-6 * max(1.0, abs(d)) + 1e-9, (i, c, d, m2[r, c])
            checked += abs(d) > 0
    assert checked >= 4


def test_ndc_scaling():
    g = np.array([[3.0, 4.0], [0.0, 0.0], [-2.0, 1.0]])
    out = O.densify_stat_ndc(g, 200, 100)
    np.testing.assert_allclose(out, [math.hypot(300.0, 200.0), 0.0, math.hypot(200.0, 50.0)])


def test_split_and_clone_rule():
    tau_g, tau_s = np.float32(2e-4), 0.05
    ln = math.log(tau_s)
    # accum / visits: exactly at the threshold, above, below, never visited
    accum = np.array([4e-4, 6e-4, 1e-4, 5.0, 4e-4, 4e-4], np.float32)
    visits = np.array([2, 1, 1, 0, 2, 2], np.int32)
    big, small = ln + 0.5, ln - 0.5
    ls = np.array([[big, -9, -9], [small, small, small], [big, big, big], [big, 0, 0],
                   [small, np.float32(ln), small], [np.nextafter(np.float32(ln), 1.0), -9, -9]],
                  np.float32)
    split, clone = O.densify_select(accum, visits, ls, tau_g, tau_s)
    # 0: g = 2e-4 >= tau_g (float32 division), large -> split; 1: small -> clone;
    # 2: g below; 3: never visited; 4: max log s equal to ln tau_s (not greater) -> clone;
    # 5: just above ln tau_s -> split
    g0 = np.float32(4e-4) / np.float32(2)
    assert g0 >= tau_g
    assert split.tolist() == [0, 5] and clone.tolist() == [1, 4]
    # disjoint and ascending by construction
    assert not set(split) & set(clone)


def test_clone_rows_copy_the_kept_rows():
    theta_new = np.arange(5 * 3, dtype=np.float64).reshape(5, 3)
    # population of 6 before the split: candidates 1 (removed) and 4 (RESET, kept)
    out = O.clone_rows(theta_new, 6, np.array([O.FALLBACK, O.RESET]), np.array([1, 4]),
                       np.array([0, 3, 5]))
    # kept ids 0, 2, 3, 4, 5 -> rows 0..4; clones of ids 0, 3, 5 -> rows 0, 2, 4
    assert out.shape == (8, 3)
    np.testing.assert_array_equal(out[5:], theta_new[[0, 2, 4]])
