"""Pins of the oracle's forward path (projection, colour, compositing, dominant map).

Each test checks the oracle against something independent of it: a closed form, a
library routine, a numerical derivative or brute force.
"""
import math

import numpy as np
import pytest

import scenes


def _one(mean, logscale, quat, logit, dc=(0.0, 0.0, 0.0), deg=0, rest=None):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0] = dc
    if rest is not None:
        sh[0, 1:] = rest
    return {"mean": np.array([mean], np.float32), "logit": np.array([logit], np.float32),
            "logscale": np.array([logscale], np.float32), "quat": np.array([quat], np.float32),
            "sh": sh, "sh_degree": deg}


def _scene(items, deg=0):
    keys = ["mean", "logit", "logscale", "quat", "sh"]
    return {**{k: np.concatenate([it[k] for it in items]) for k in keys}, "sh_degree": deg}


# ----------------------------------------------------------------- SH basis

def test_sh_basis_orthonormal_on_sphere(orc):
    """The 16 real SH basis functions are orthonormal on the unit sphere
    (Gauss-Legendre in cos(theta) x uniform phi quadrature, exact for these
    polynomial degrees)."""
    nt, nphi = 24, 48
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wt = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = orc.sh_basis(3, dirs)
    G = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_matches_scipy_up_to_sign(orc):
    """|Y_k| equals the magnitude of scipy's real spherical harmonic of the
    same (l, m) (index k = l^2 + l + m)."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = orc.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            c = sp.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            np.testing.assert_allclose(np.abs(Y[:, k]), np.abs(ref), atol=1e-12)
    # degree-1 orientation of the 3DGS basis: (-y, z, -x) up to positive factors
    assert np.all(np.sign(Y[:, 1]) == -np.sign(d[:, 1]))
    assert np.all(np.sign(Y[:, 2]) == np.sign(d[:, 2]))
    assert np.all(np.sign(Y[:, 3]) == -np.sign(d[:, 0]))


# ----------------------------------------------------------------- rotations

def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_quat_to_rot_matches_sandwich_product(orc):
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.normal(size=4)
        R = orc.quat_to_rot(q)[0]
        qn = q / np.linalg.norm(q)
        qc = qn * np.array([1, -1, -1, -1])
        v = rng.normal(size=3)
        rv = _qmul(_qmul(qn, np.r_[0.0, v]), qc)[1:]
        np.testing.assert_allclose(R @ v, rv, atol=1e-12)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12
        q2 = orc.rot_to_quat(R)[0]
        np.testing.assert_allclose(orc.quat_to_rot(q2)[0], R, atol=1e-12)


# ----------------------------------------------------------------- projection

def test_projection_isotropic_on_axis_closed_form(orc):
    """One isotropic Gaussian on the optical axis: Sigma2D = (f s / z)^2 I + 0.3 I,
    centred on the principal point."""
    cam = scenes.camera_origin_forward(65, 49, 60.0)
    z, s = 3.0, 0.05
    sc = _one([0, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], 0.5)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    f = float(cam["fx"])
    s32 = float(np.float32(math.log(s)))
    var = (f * math.exp(s32) / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0, var], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0, 1 / var], rtol=1e-12)
    np.testing.assert_allclose(pr["mean2d"][0], [cam["px"], cam["py"]], atol=1e-12)
    assert pr["depth"][0] == z
    np.testing.assert_allclose(pr["opacity"][0], 1 / (1 + math.exp(-float(np.float32(0.5)))))


def _pixel_of(cam, X):
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    p = R @ X + np.asarray(cam["t"], np.float64)
    return np.array([cam["fx"] * p[0] / p[2] + cam["px"], cam["fy"] * p[1] / p[2] + cam["py"]])


def test_projection_matches_numerical_jacobian(orc):
    """EWA: Sigma2D = J Sigma J^T + 0.3 I with J the Jacobian of the world->pixel
    map at the mean, here taken by central differences (rotated camera,
    anisotropic rotated Gaussian, inside the clamp range)."""
    rng = np.random.default_rng(1)
    cam = scenes.camera_look_at((2.0, -0.5, -3.0), (0.1, 0.2, 0.3), 160, 96)
    for _ in range(10):
        mean = rng.normal(0, 0.4, 3)
        ls = rng.normal(-2.5, 0.4, 3)
        q = rng.normal(size=4)
        sc = _one(mean, ls, q, 1.0)
        th = orc.theta_of(sc)
        pr = orc.project(th, 0, cam)
        X = th[0, 0:3]
        h = 1e-6
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (_pixel_of(cam, X + e) - _pixel_of(cam, X - e)) / (2 * h)
        Rg = orc.quat_to_rot(th[0, 7:11])[0]
        S = Rg @ np.diag(np.exp(2 * th[0, 4:7])) @ Rg.T
        C2 = J @ S @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][0], [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-6)
        np.testing.assert_allclose(pr["mean2d"][0], _pixel_of(cam, X), rtol=1e-12)
        inv = np.linalg.inv(C2)
        np.testing.assert_allclose(pr["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)


def test_colour_dc_only_closed_form(orc):
    """Degree 0: colour = max(0, dc / (2 sqrt(pi)) + 0.5) per channel."""
    cam = scenes.camera_origin_forward(32, 32)
    dc = np.array([1.2, -0.4, -2.5], np.float32)
    sc = _one([0.1, 0, 3], [-3] * 3, [1, 0, 0, 0], 0.0, dc=dc)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    ref = np.maximum(0.0, dc.astype(np.float64) / (2 * math.sqrt(math.pi)) + 0.5)
    np.testing.assert_allclose(pr["rgb"][0], ref, rtol=1e-14)
    assert list(pr["clamped"][0]) == [0, 0, 1]


def test_colour_view_direction(orc):
    """Degree 3: colour = 0.5 + sum_k sh_k Y_k(d) with d the unit vector from the
    camera centre (-R^T t) to the mean."""
    rng = np.random.default_rng(2)
    cam = scenes.camera_look_at((1.5, -1.0, -4.0), (0, 0, 0), 64, 64)
    rest = rng.normal(0, 0.2, (15, 3)).astype(np.float32)
    sc = _one([0.2, -0.1, 0.3], [-3] * 3, [1, 0, 0, 0], 0.0, dc=(0.3, 0.2, 0.1), deg=3, rest=rest)
    th = orc.theta_of(sc)
    pr = orc.project(th, 3, cam)
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    centre = -R.T @ np.asarray(cam["t"], np.float64)
    d = th[0, :3] - centre
    d /= np.linalg.norm(d)
    Y = orc.sh_basis(3, d[None])[0]
    ref = np.maximum(0, 0.5 + Y @ th[0, 11:].reshape(16, 3))
    np.testing.assert_allclose(pr["rgb"][0], ref, rtol=1e-13)


def test_box_contains_support_and_rect(orc):
    """Every pixel with alpha_raw >= 1/255 lies inside the Gaussian's pixel box
    (checked by brute force over the image), and the tile rectangle is the box
    divided by the tile size."""
    sc = scenes.scene_box(11, 300, 0)
    cam = scenes.camera_origin_forward(96, 80)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    yy, xx = np.mgrid[0:80, 0:96]
    for i in range(300):
        if pr["tiles"][i] == 0:
            continue
        dx = pr["mean2d"][i, 0] - xx
        dy = pr["mean2d"][i, 1] - yy
        A, B, Cc = pr["conic"][i]
        a = pr["opacity"][i] * np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
        ys, xs = np.nonzero(a >= 1 / 255)
        b = pr["box"][i]
        if len(xs):
            assert xs.min() >= b[0] and xs.max() <= b[1] and ys.min() >= b[2] and ys.max() <= b[3]
        r = pr["rect"][i]
        assert list(r) == [b[0] // 16, b[1] // 16, b[2] // 16, b[3] // 16]
        assert pr["tiles"][i] == (r[1] - r[0] + 1) * (r[3] - r[2] + 1)


def test_culling_rules(orc):
    cam = scenes.camera_origin_forward(32, 32)
    behind = _one([0, 0, 0.1], [-3] * 3, [1, 0, 0, 0], 0.0)
    faint = _one([0, 0, 3], [-3] * 3, [1, 0, 0, 0], -6.0)  # opacity < 1/255
    off = _one([50, 0, 3], [-3] * 3, [1, 0, 0, 0], 0.0)
    ok = _one([0, 0, 3], [-3] * 3, [1, 0, 0, 0], 0.0)
    pr = orc.project(orc.theta_of(_scene([behind, faint, off, ok])), 0, cam)
    assert list(pr["tiles"] > 0) == [False, False, False, True]


# ----------------------------------------------------------------- compositing

def test_single_splat_analytic_footprint(orc):
    """One Gaussian: pixel = c min(0.99, o exp(-0.5 d^T C d)) where that reaches
    1/255, else the (black) background; T = 1 - alpha."""
    cam = scenes.camera_origin_forward(41, 37)
    sc = _one([0.05, -0.03, 2.5], [-2.2, -2.6, -2.4], [0.9, 0.2, -0.1, 0.3], 1.5, dc=(1.0, 0.5, -1.0))
    pr = orc.project(orc.theta_of(sc), 0, cam)
    rd = orc.render(pr, cam)
    yy, xx = np.mgrid[0:37, 0:41]
    A, B, Cc = pr["conic"][0]
    dx, dy = pr["mean2d"][0, 0] - xx, pr["mean2d"][0, 1] - yy
    a = pr["opacity"][0] * np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
    a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0).reshape(-1)
    np.testing.assert_allclose(rd["rgb"], a[:, None] * pr["rgb"][0][None, :], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(rd["T"], 1 - a, rtol=1e-13)
    assert np.all(rd["dominant"][a > 0] == 0) and np.all(rd["dominant"][a == 0] == -1)
    # distance to the 1/255 cut-off: |alpha_raw - 1/255| where the pixel tests the
    # Gaussian (contributes, or misses by at most the capture window), else none
    cfg = orc.Config(tie_capture=3e-3)
    rw = orc.render(pr, cam, cfg=cfg)
    ar = (pr["opacity"][0] * np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)).reshape(-1)
    box = pr["box"][0]
    inbox = ((xx >= box[0]) & (xx <= box[1]) & (yy >= box[2]) & (yy <= box[3])).reshape(-1)
    tested = inbox & (ar >= 1 / 255 - cfg.tie_capture)
    assert tested.sum() > a.astype(bool).sum()  # some near misses are reported
    np.testing.assert_allclose(rw["dist"][tested, 0], np.abs(ar[tested] - 1 / 255), rtol=1e-12)
    assert np.all(rw["dist"][~tested, 0] > 1e299)
    assert np.array_equal(rw["rgb"], rd["rgb"])  # near misses are never blended


def _stack(opacities, dcs, w=33, h=33):
    """Large isotropic Gaussians centred on the middle pixel, at increasing depth:
    at that pixel alpha_i equals opacity_i exactly."""
    items = []
    for k, (o, dc) in enumerate(zip(opacities, dcs)):
        logit = math.log(o / (1 - o))
        items.append(_one([0, 0, 2.0 + k], [0.0] * 3, [1, 0, 0, 0], logit, dc=dc))
    sc = _scene(items)
    return sc, scenes.camera_origin_forward(w, h)


def test_three_splat_transmittance_product(orc):
    ops = [0.3, 0.5, 0.7]
    dcs = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    sc, cam = _stack(ops, dcs)
    th = orc.theta_of(sc)
    pr = orc.project(th, 0, cam)
    c = pr["rgb"]
    a = pr["opacity"]
    centre = 16 * 33 + 16
    rd = orc.render(pr, cam, pixels=[centre])
    ref = a[0] * c[0] + (1 - a[0]) * a[1] * c[1] + (1 - a[0]) * (1 - a[1]) * a[2] * c[2]
    np.testing.assert_allclose(rd["rgb"][0], ref, rtol=1e-14)
    np.testing.assert_allclose(rd["T"][0], (1 - a[0]) * (1 - a[1]) * (1 - a[2]), rtol=1e-14)
    # weights w = (0.3, 0.35, 0.245): the second Gaussian dominates (Eq. 5)
    assert rd["dominant"][0] == 1 and rd["second"][0] == 0
    assert rd["n_contrib"][0] == 3


def test_threshold_distances_of_a_stack(orc):
    """The distances behind the tie flags, by hand at the centre pixel of the
    three-splat stack (alpha_i = opacity_i exactly): to 1/255 the smallest
    |alpha - 1/255|, to the stop threshold the smallest |T (1 - alpha) - 1e-4| over
    the three stop tests, to the clamp the smallest |alpha - 0.99|, and the margin
    w_best - w_second of the weights (0.3, 0.35, 0.245)."""
    sc, cam = _stack([0.3, 0.5, 0.7], [(1.0, 0.0, 0.0)] * 3)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    a = pr["opacity"]
    rd = orc.render(pr, cam, pixels=[16 * 33 + 16])
    tests = [1 - a[0], (1 - a[0]) * (1 - a[1]), (1 - a[0]) * (1 - a[1]) * (1 - a[2])]
    w = sorted([a[0], (1 - a[0]) * a[1], (1 - a[0]) * (1 - a[1]) * a[2]])
    want = [min(abs(x - 1 / 255) for x in a), min(abs(t - 1e-4) for t in tests),
            min(abs(x - 0.99) for x in a), w[-1] - w[-2]]
    np.testing.assert_allclose(rd["dist"][0], want, rtol=1e-12)
    assert rd["tie"][0] == 0
    # bands wider than a distance set that distance's bit
    wide = orc.render(pr, cam, pixels=[16 * 33 + 16],
                      cfg=orc.Config(tie_stop=0.2, tie_margin=0.06))
    assert wide["tie"][0] == 2 | 8
    assert np.array_equal(orc.tie_bits(rd["dist"], stop=0.2, margin=0.06), wide["tie"])


def test_stop_distance_covers_the_stopping_test(orc):
    """alpha = 0.95 five times: the stop tests are 0.05, 0.0025, 1.25e-4 and the
    failing 6.25e-6; the nearest to 1e-4 is 1.25e-4 (distance 2.5e-5), and no test
    after the stop counts."""
    sc, cam = _stack([0.95] * 5, [(1.0, 1.0, 1.0)] * 5)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    a = pr["opacity"][0]
    rd = orc.render(pr, cam, pixels=[16 * 33 + 16])
    tests = [(1 - a) ** k for k in (1, 2, 3, 4)]
    np.testing.assert_allclose(rd["dist"][0, 1], min(abs(t - 1e-4) for t in tests), rtol=1e-12)
    assert rd["tie"][0] == 0
    near = orc.render(pr, cam, pixels=[16 * 33 + 16], cfg=orc.Config(tie_stop=3e-5))
    assert near["tie"][0] == 2


def test_early_stop_before_blending(orc):
    """alpha = 0.95 five times: T runs 1, .05, .0025, 1.25e-4; the fourth
    Gaussian would leave 6.25e-6 < 1e-4, so it and the rest are not blended."""
    sc, cam = _stack([0.95] * 5, [(1.0, 1.0, 1.0)] * 5)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    rd = orc.render(pr, cam, pixels=[16 * 33 + 16])
    a = pr["opacity"][0]
    assert rd["n_contrib"][0] == 3
    np.testing.assert_allclose(rd["T"][0], (1 - a) ** 3, rtol=1e-14)
    np.testing.assert_allclose(rd["rgb"][0], pr["rgb"][0] * (1 - (1 - a) ** 3), rtol=1e-13)


def test_alpha_clamp(orc):
    sc, cam = _stack([0.995], [(1.0, 1.0, 1.0)])
    pr = orc.project(orc.theta_of(sc), 0, cam)
    rd = orc.render(pr, cam, pixels=[16 * 33 + 16])
    np.testing.assert_allclose(rd["T"][0], 0.01, rtol=1e-12)


def test_weights_sum_to_one_minus_transmittance(orc):
    """With every colour 1 and a black background the pixel value is
    sum_i T_i alpha_i = 1 - T_final <= 1 (Eq. 1)."""
    sc = scenes.scene_box(5, 400, 0)
    sc["sh"][:] = np.float32(math.sqrt(math.pi))  # decodes to colour 1.0
    cam = scenes.camera_origin_forward(48, 48)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    c = pr["rgb"][pr["tiles"] > 0]
    np.testing.assert_allclose(c, 1.0, rtol=1e-7)  # sqrt(pi) rounded to float32
    rd = orc.render(pr, cam)
    np.testing.assert_allclose(rd["rgb"][:, 0], c[0, 0] * (1 - rd["T"]), rtol=1e-12, atol=1e-15)
    assert np.all(1 - rd["T"] <= 1) and np.all(rd["T"] >= 0)


def test_bucketed_render_equals_brute_force(orc):
    sc = scenes.scene_box(9, 600, 0)
    cam = scenes.camera_origin_forward(70, 50)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    full = orc.render(pr, cam, bg=(0.1, 0.2, 0.3))
    brute = orc.render(pr, cam, bg=(0.1, 0.2, 0.3), pixels=np.arange(70 * 50))
    for k in ("rgb", "T", "n_contrib", "dominant", "second", "tie"):
        assert np.array_equal(full[k], brute[k]), k


def test_dominant_is_argmax_of_weights(orc):
    """Brute force: recompute every contributor's weight T alpha per pixel in
    numpy and take the argmax."""
    sc = scenes.scene_box(13, 120, 0)
    cam = scenes.camera_origin_forward(24, 24)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    rd = orc.render(pr, cam)
    vis = np.nonzero(pr["tiles"] > 0)[0]
    for u in range(0, 24 * 24, 7):
        x, y = u % 24, u // 24
        lst = []
        for i in vis:
            b = pr["box"][i]
            if not (b[0] <= x <= b[1] and b[2] <= y <= b[3]):
                continue
            dx, dy = pr["mean2d"][i, 0] - x, pr["mean2d"][i, 1] - y
            A, B, Cc = pr["conic"][i]
            a = pr["opacity"][i] * math.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
            if a >= 1 / 255:
                lst.append((pr["depth"][i], i, min(a, 0.99)))
        lst.sort()
        T, best, dom = 1.0, -1.0, -1
        for _, i, a in lst:
            if T * (1 - a) < 1e-4:
                break
            if T * a > best:
                best, dom = T * a, i
            T *= 1 - a
        assert rd["dominant"][u] == dom


def test_tile_lists_by_definition(orc):
    """Instances per tile = Gaussians whose tile rectangle covers the tile,
    ordered by (float32 depth, id) (brute force in Python)."""
    sc = scenes.scene_box(21, 200, 0)
    cam = scenes.camera_origin_forward(64, 48)
    pr = orc.project(orc.theta_of(sc), 0, cam)
    d32 = pr["depth"].astype(np.float32)
    d32[5] = d32[6]  # force a depth tie: resolved by id
    start, inst = orc.tile_lists(d32, pr["rect"], pr["tiles"], 4, 3)
    for t in range(12):
        tx, ty = t % 4, t // 4
        ids = [i for i in range(200) if pr["tiles"][i] > 0 and pr["rect"][i, 0] <= tx <= pr["rect"][i, 1]
               and pr["rect"][i, 2] <= ty <= pr["rect"][i, 3]]
        ids.sort(key=lambda i: (d32[i], i))
        assert list(inst[start[t]:start[t + 1]]) == ids
