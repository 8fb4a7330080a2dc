"""Pins of the oracle's AdpSplit operator: child initialisation (Eqs. 9-10 and
Appendix A), cross-view merge (Eqs. 11-12), cap, statuses, parent copy, fallback
split (Eqs. 3-4) and the order of the new population."""
import json
import math
import os

import numpy as np
import pytest

import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_split_defaults_follow_the_paper(orc):
    g = json.load(open(os.path.join(GOLDEN, "paper_defaults.json")))
    sp = orc.SplitParams()
    for k in ("tau_l1", "r_erode", "m_min", "n_levels", "n_max", "gamma_d", "gamma_c"):
        assert getattr(sp, k) == g[k], k


def _parent(mean, logscale, quat, logit=0.3, deg=0):
    K = (deg + 1) ** 2
    th = np.zeros(11 + 3 * K)
    th[0:3] = mean
    th[3] = logit
    th[4:7] = logscale
    th[7:11] = quat
    return th


def _stats(cx, cy, e1=(1.0, 0.0), s1=3.0, s2=1.5, rgb=(0.2, 0.5, 0.9)):
    e = np.array(e1, float) / np.linalg.norm(e1)
    return np.array([cx, cy, 0, 0, 0, e[0], e[1], s1, s2, *rgb])


def _golden_section(f, a, b, iters=200):
    g = (math.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(iters):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def test_tstar_is_the_mahalanobis_closest_ray_point(orc):
    """t* minimises (l(t) - mu)^T Sigma^-1 (l(t) - mu) along the centroid ray:
    it matches a golden-section search and the derivative vanishes there."""
    rng = np.random.default_rng(0)
    cam = scenes.camera_look_at((1.0, -0.5, -4.0), (0, 0, 0), 120, 90)
    for _ in range(10):
        th = _parent(rng.normal(0, 0.3, 3), rng.normal(-2, 0.5, 3), rng.normal(size=4))
        st = _stats(rng.uniform(20, 100), rng.uniform(10, 80))
        ch = orc.child_proposal(th, cam, st, eps_t=0.0)
        R = np.asarray(cam["R"], np.float64).reshape(3, 3)
        o = -R.T @ np.asarray(cam["t"], np.float64)
        dcam = np.array([(st[0] - float(cam["px"])) / float(cam["fx"]), (st[1] - float(cam["py"])) / float(cam["fy"]), 1.0])
        d = R.T @ dcam
        d /= np.linalg.norm(d)
        Rp = orc.quat_to_rot(th[7:11])[0]
        Ainv = Rp @ np.diag(np.exp(-2 * th[4:7])) @ Rp.T
        f = lambda t: (o + t * d - th[:3]) @ Ainv @ (o + t * d - th[:3])
        t_num = _golden_section(f, -50, 50)
        assert abs(ch["tstar"] - t_num) < 1e-6 * max(1, abs(t_num))
        grad = 2 * d @ Ainv @ (o + ch["tstar"] * d - th[:3])
        assert abs(grad) < 1e-8 * (1 + abs(d @ Ainv @ d))
        np.testing.assert_allclose(ch["mu"], o + ch["tstar"] * d, atol=1e-12)


def test_tstar_isotropic_parent_is_the_orthogonal_projection(orc):
    """For an isotropic parent, Eq. 10 reduces to t* = b.d / (1 + eps s^2)."""
    cam = scenes.camera_origin_forward(64, 64)
    th = _parent([0.3, -0.2, 4.0], [math.log(0.1)] * 3, [1, 0, 0, 0])
    st = _stats(40.0, 25.0)
    for eps in (0.0, 1e-8, 1e-2):
        ch = orc.child_proposal(th, cam, st, eps_t=eps)
        d = np.array([(40 - float(cam["px"])) / float(cam["fx"]), (25 - float(cam["py"])) / float(cam["fy"]), 1.0])
        d /= np.linalg.norm(d)
        ref = (th[:3] @ d) / (1 + eps * 0.01)
        assert abs(ch["tstar"] - ref) < 1e-12


def _project(cam, X):
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    p = R @ X + np.asarray(cam["t"], np.float64)
    return np.array([float(cam["fx"]) * p[0] / p[2] + float(cam["px"]), float(cam["fy"]) * p[1] / p[2] + float(cam["py"])])


def test_child_geometry(orc):
    """The child sits on the centroid ray (projects back to the centroid); R is
    a proper rotation whose third column is the camera forward axis and whose
    first two lie in the image plane; scales never exceed the parent's largest
    scale; an unclipped first axis spans sigma1 pixels along e1; colour decodes
    back to the target RGB."""
    rng = np.random.default_rng(1)
    cam = scenes.camera_look_at((0.5, -1.0, -5.0), (0, 0, 0), 200, 150)
    zv = np.asarray(cam["R"], np.float64).reshape(3, 3)[2]
    for _ in range(20):
        th = _parent(rng.normal(0, 0.5, 3), rng.normal(-1.5, 0.5, 3), rng.normal(size=4))
        ang = rng.uniform(0, np.pi)
        st = _stats(rng.uniform(30, 170), rng.uniform(20, 130), (math.cos(ang), math.sin(ang)),
                    s1=rng.uniform(1, 6), s2=rng.uniform(0.2, 1))
        ch = orc.child_proposal(th, cam, st)
        R = ch["R"]
        # the camera rows are float32 values, orthonormal to ~1e-8
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-7)
        np.testing.assert_allclose(R[:, :2].T @ R[:, :2], np.eye(2), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-7
        np.testing.assert_allclose(R[:, 2], zv, atol=1e-15)
        assert abs(R[:, 0] @ zv) < 1e-7 and abs(R[:, 1] @ zv) < 1e-7
        assert np.all(ch["s"] <= np.exp(th[4:7]).max() * (1 + 1e-12))
        assert ch["s"][2] == ch["s"][1] and ch["s"][0] >= 0
        if ch["tstar"] > 0:
            np.testing.assert_allclose(_project(cam, ch["mu"]), st[:2], atol=1e-8)
        np.testing.assert_allclose(ch["rgb"], st[9:12])
    # unclipped case: the first axis covers sigma1 pixels along e1 (to first order)
    th = _parent([0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1, 0, 0, 0])
    st = _stats(100.0, 75.0, (0.6, 0.8), s1=2.0, s2=1.0)
    ch = orc.child_proposal(th, cam, st)
    a1 = ch["R"][:, 0] * ch["s"][0]
    h = 1e-4
    dpix = (_project(cam, ch["mu"] + h * a1) - _project(cam, ch["mu"] - h * a1)) / (2 * h)
    np.testing.assert_allclose(np.abs(dpix), 2.0 * np.array([0.6, 0.8]), rtol=1e-3)


def test_child_clip_bound(orc):
    """A huge region against a tiny parent: each axis component is clipped to
    s_max |e|, so s1 = s2 = s_max."""
    cam = scenes.camera_origin_forward(64, 64)
    th = _parent([0, 0, 5.0], [math.log(0.01)] * 3, [1, 0, 0, 0])
    ch = orc.child_proposal(th, cam, _stats(32, 32, (1, 1), s1=500, s2=400))
    np.testing.assert_allclose(ch["s"], [0.01, 0.01, 0.01], rtol=1e-12)


def _cov(R, s):
    R = np.asarray(R).reshape(3, 3)
    return R @ np.diag(np.asarray(s) ** 2) @ R.T


def test_merge_singleton_is_identity(orc):
    rng = np.random.default_rng(2)
    R = orc.quat_to_rot(rng.normal(size=4))
    s = np.array([[0.3, 0.1, 0.1]])
    mg = orc.merge(np.array([[1.0, 2.0, 3.0]]), R, s, np.array([[0.1, 0.2, 0.3]]))
    assert mg["n_groups"] == 1
    np.testing.assert_allclose(mg["Sigma"][0], _cov(R[0], s[0]), atol=1e-14)
    np.testing.assert_allclose(mg["mu"][0], [1, 2, 3])


def test_merge_transitive_enclosing_and_exact_means(orc):
    """A-B and B-C are within gamma_d but A-C is not: all three merge (Eq. 11 is
    applied transitively). The merged centre and colour are exact means, and the
    merged ellipsoid reaches every member's 1-sigma extent along each eigenaxis
    of the mean covariance (Eq. 12)."""
    s = np.array([[0.5, 0.5, 0.5]] * 3 + [[0.5, 0.5, 0.5]])
    R = np.stack([np.eye(3)] * 4)
    mu = np.array([[0, 0, 0], [0.9, 0, 0], [1.8, 0, 0], [10, 0, 0]], float)
    rgb = np.array([[0.5, 0.5, 0.5], [0.55, 0.5, 0.5], [0.6, 0.5, 0.5], [0.5, 0.5, 0.5]])
    # symmetric distances: A-B = 1.8/... = 0.9/0.5*2 = 3.6 > 2 with these scales, so widen
    s[:3] = [[1.0, 0.3, 0.3]] * 3
    mg = orc.merge(mu, R, s, rgb)
    # A-B: 0.9 + 0.9 = 1.8 <= 2; B-C same; A-C: 1.8 + 1.8 = 3.6 > 2
    assert list(mg["group_of"]) == [0, 0, 0, 1]
    np.testing.assert_allclose(mg["mu"][0], mu[:3].mean(0), atol=1e-15)
    np.testing.assert_allclose(mg["rgb"][0], rgb[:3].mean(0), atol=1e-15)
    Sig = mg["Sigma"][0]
    lam, E = np.linalg.eigh(Sig)
    for m in range(3):
        Sm = _cov(R[m], s[m])
        for r in range(3):
            e = E[:, r]
            reach = abs(e @ (mu[m] - mg["mu"][0])) + math.sqrt(e @ Sm @ e)
            assert lam[r] >= reach ** 2 * (1 - 1e-9)
    # colour difference above gamma_c blocks the edge
    rgb2 = rgb.copy()
    rgb2[1, 0] = 0.8
    mg2 = orc.merge(mu, R, s, rgb2)
    assert mg2["n_groups"] == 4


def test_merge_boundary_is_inclusive(orc):
    """Both thresholds of Eq. 11 are inclusive (<=)."""
    R = np.stack([np.eye(3)] * 2)
    s = np.array([[1.0, 1, 1], [1.0, 1, 1]])
    mu = np.array([[0, 0, 0], [1.0, 0, 0]])
    rgb = np.array([[0.5, 0.5, 0.5], [0.625, 0.5, 0.5]])
    assert orc.merge(mu, R, s, rgb, gamma_d=2.0, gamma_c=0.125)["n_groups"] == 1
    assert orc.merge(mu, R, s, rgb, gamma_d=1.999, gamma_c=0.125)["n_groups"] == 2
    assert orc.merge(mu, R, s, rgb, gamma_d=2.0, gamma_c=0.124)["n_groups"] == 2


def _toy_split_inputs(orc, n=12, deg=1):
    rng = np.random.default_rng(5)
    cams = [scenes.camera_look_at((4 * math.cos(a), 0, 4 * math.sin(a)), (0, 0, 0), 80, 60)
            for a in (0.3, 1.1)]
    sc = scenes.scene_box(3, n, deg)
    sc["mean"][:] = (rng.normal(0, 0.3, (n, 3))).astype(np.float32)
    sc["logscale"][:] = np.float32(-1.0)
    theta = orc.theta_of(sc)
    # candidates 1, 4, 6, 9: 1 has no attributed pixels (fallback), 4 has pixels
    # but no region (reset), 6 and 9 have regions (adaptive)
    cand = np.array([1, 4, 6, 9], np.int32)
    count = np.zeros(n, np.int32)
    count[[4, 6, 9, 2]] = [10, 50, 30, 7]
    regs = {"view": [], "parent": [], "label": [], "stats": []}
    for (v, p, lab, cx, cy) in [(0, 6, 100, 30, 20), (0, 6, 900, 50, 40), (1, 6, 77, 40, 30),
                                (1, 9, 5, 20, 10), (0, 2, 60, 10, 10)]:
        regs["view"].append(v)
        regs["parent"].append(p)
        regs["label"].append(lab)
        regs["stats"].append(_stats(cx, cy, (0.8, 0.6), s1=4, s2=2, rgb=rng.uniform(0, 1, 3)))
    regs = {k: np.ascontiguousarray(np.array(v, np.int32 if k != "stats" else np.float64))
            for k, v in regs.items()}
    noise = scenes.fallback_noise(9, 4).astype(np.float64)
    return theta, deg, cams, regs, cand, count, noise


def test_split_statuses_and_population_order(orc):
    theta, deg, cams, regs, cand, count, noise = _toy_split_inputs(orc)
    n, P = theta.shape
    am = np.random.default_rng(1).normal(size=theta.shape)
    av = np.abs(np.random.default_rng(2).normal(size=theta.shape))
    out = orc.split(theta, deg, cams, regs, cand, count, noise, adam_m=am, adam_v=av)
    assert list(out["status"]) == [orc.FALLBACK, orc.RESET, orc.ADAPTIVE, orc.ADAPTIVE]
    N6, N9 = out["n_children"][2], out["n_children"][3]
    assert 1 <= N6 <= 3 and N9 == 1
    assert out["new_n"] == (n - 4) + 1 + 2 + (1 + N6) + (1 + N9)
    th = out["theta"]
    # kept in id order: non-candidates and the RESET candidate 4, Adam state kept
    kept = [i for i in range(n) if i not in (1, 6, 9)]
    assert np.array_equal(th[:len(kept)], theta[kept])
    assert np.array_equal(out["m"][:len(kept)], am[kept]) and np.array_equal(out["v"][:len(kept)], av[kept])
    assert not out["m"][len(kept):].any() and not out["v"][len(kept):].any()
    o = len(kept)
    # candidate 1: vanilla split into two (Eqs. 3-4) with the given noise
    Rp = orc.quat_to_rot(theta[1, 7:11])[0]
    s = np.exp(theta[1, 4:7])
    for c in range(2):
        np.testing.assert_allclose(th[o + c, :3], theta[1, :3] + Rp @ (s * noise[0, c]), atol=1e-14)
        np.testing.assert_allclose(np.exp(th[o + c, 4:7]), s / (0.8 * 2), rtol=1e-14)
        assert np.array_equal(th[o + c, 7:], theta[1, 7:]) and th[o + c, 3] == theta[1, 3]
    o += 2
    # candidate 6: parent copy with opacity o/(N+1), scale unchanged, then children
    for (i, N) in ((6, N6), (9, N9)):
        op = 1 / (1 + math.exp(-theta[i, 3]))
        np.testing.assert_allclose(1 / (1 + math.exp(-th[o, 3])), op / (N + 1), rtol=1e-13)
        assert np.array_equal(th[o, 4:], theta[i, 4:]) and np.array_equal(th[o, :3], theta[i, :3])
        for k in range(1, N + 1):
            assert th[o + k, 3] == theta[i, 3]  # children inherit the opacity
            assert np.all(th[o + k, 14:] == 0)  # higher SH bands zero
        o += 1 + N
    assert o == out["new_n"]


def test_split_cap_keeps_largest_extents(orc):
    """Many far-apart regions of one parent: n_max of them survive, those with
    the largest sqrt(det Sigma), emitted in first-member order."""
    cam = scenes.camera_origin_forward(200, 200)
    th = _parent([0, 0, 5.0], [0.0] * 3, [1, 0, 0, 0])[None]
    rng = np.random.default_rng(4)
    M = 12
    st = np.stack([_stats(15 + 15 * k, 100, (1, 0), s1=rng.uniform(1, 5), s2=rng.uniform(0.5, 1),
                          rgb=rng.uniform(0, 1, 3)) for k in range(M)])
    regs = dict(view=np.zeros(M, np.int32), parent=np.zeros(M, np.int32),
                label=np.arange(M, dtype=np.int32) * 3, stats=st)
    sp = orc.SplitParams(n_max=5, gamma_d=1e-9)
    out = orc.split(th, 0, [cam], regs, np.array([0], np.int32), np.array([99], np.int32),
                    np.zeros((1, 2, 3)), sp)
    assert out["n_children"][0] == 5
    props = [orc.child_proposal(th[0], cam, st[k]) for k in range(M)]
    ext = np.array([np.prod(p["s"]) for p in props])
    keep = sorted(np.argsort(-ext, kind="stable")[:5])
    kids = out["theta"][1:]
    for j, k in enumerate(keep):
        np.testing.assert_allclose(kids[j, :3], props[k]["mu"], atol=1e-12)
        Sk = _cov(orc.quat_to_rot(kids[j, 7:11])[0], np.exp(kids[j, 4:7]))
        np.testing.assert_allclose(Sk, _cov(props[k]["R"], props[k]["s"]), atol=1e-12)
        dc = kids[j, 11:14]
        np.testing.assert_allclose(dc / (2 * math.sqrt(math.pi)) + 0.5, props[k]["rgb"], atol=1e-12)
