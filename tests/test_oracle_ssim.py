"""Pins of the oracle's D-SSIM loss term: identity, the closed form for constant
images, symmetry, the window, and the gradient against central differences of the
oracle's own loss."""
import numpy as np

import oracle as O

C1, C2 = 0.01 ** 2, 0.03 ** 2


def test_window():
    w = O.ssim_window()
    assert w.shape == (11,) and abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w, w[::-1])
    np.testing.assert_allclose(w[4] / w[5], np.exp(-1.0 / (2 * 1.5 ** 2)))


def test_identity_and_symmetry():
    rng = np.random.default_rng(0)
    x, y = rng.random(23 * 17 * 3), rng.random(23 * 17 * 3)
    l1, s, g = O.dssim_loss_grad(x, x, 17, 23)
    assert l1 == 0.0 and abs(s - 1.0) < 1e-12
    _, s_xy, _ = O.dssim_loss_grad(x, y, 17, 23)
    _, s_yx, _ = O.dssim_loss_grad(y, x, 17, 23)
    assert abs(s_xy - s_yx) < 1e-12 and s_xy < 1.0


def test_constant_images_closed_form_away_from_the_border():
    a, b = 0.7, 0.2
    x, y = np.full((30, 40), a), np.full((30, 40), b)
    S = O.ssim_channel(x, y)[0]
    want = (2 * a * b + C1) / (a * a + b * b + C1)  # no variance, no covariance
    np.testing.assert_allclose(S[5:-5, 5:-5], want, rtol=1e-12)
    assert abs(S[0, 0] - want) > 1e-3  # the zero padding changes the border


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    W, H = 14, 12
    x, y = rng.random(W * H * 3), rng.random(W * H * 3)
    lam = 0.2
    _, _, g = O.dssim_loss_grad(x, y, W, H, lam)

    def loss(xx):
        l1, s, _ = O.dssim_loss_grad(xx, y, W, H, lam)
        return (1 - lam) * l1 + lam * (1 - s)

    h = 1e-6
    for idx in rng.choice(x.size, 40, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(xp) - loss(xm)) / (2 * h)
        assert abs(fd - g.reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (idx, fd)
