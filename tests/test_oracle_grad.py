"""Pins of the oracle's gradient (complex-step derivative of the forward) against
central finite differences of the FP64 forward, and of its Adam step against the
closed form for a constant gradient."""
import numpy as np

import scenes


def _target(orc, seed, cam):
    sc, _ = scenes.subscene_for_gradients(seed, n=48, width=int(cam["width"]), height=int(cam["height"]))
    pr = orc.project(orc.theta_of(sc), 3, cam)
    rd = orc.render(pr, cam)
    return rd["rgb"].astype(np.float32).reshape(int(cam["height"]), int(cam["width"]), 3)


def test_gradient_matches_central_differences(orc):
    """All 59 parameters of several Gaussians of the 64-Gaussian, 32x32 scene:
    the oracle gradient agrees with central differences (h = 1e-6, FP64)."""
    sc, cam = scenes.subscene_for_gradients(0)
    tgt = _target(orc, 1, cam)
    theta = orc.theta_of(sc)
    sel = np.array([0, 5, 17, 33, 63], np.int32)
    g = orc.grad(theta, 3, cam, tgt, sel)
    h = 1e-6
    worst = 0.0
    for r, i in enumerate(sel):
        for p in range(theta.shape[1]):
            tp, tm = theta.copy(), theta.copy()
            tp[i, p] += h
            tm[i, p] -= h
            fd = (orc.l1_loss(tp, 3, cam, tgt) - orc.l1_loss(tm, 3, cam, tgt)) / (2 * h)
            err = abs(fd - g[r, p]) / (abs(g[r, p]) + 1e-6 * np.abs(g[r]).max() + 1e-12)
            worst = max(worst, err)
            assert err < 1e-4, (i, p, fd, g[r, p])
    assert np.abs(g).max() > 0


def test_gradient_zero_for_invisible_and_directional(orc):
    """A Gaussian behind the camera gets a zero gradient; a random direction over
    every parameter of the scene matches a central difference of the loss."""
    sc, cam = scenes.subscene_for_gradients(2)
    sc["mean"][3] = [0, 0, -1]
    tgt = _target(orc, 3, cam)
    theta = orc.theta_of(sc)
    g = orc.grad(theta, 3, cam, tgt)
    assert not g[3].any()
    rng = np.random.default_rng(0)
    d = rng.normal(size=theta.shape)
    h = 1e-7
    fd = (orc.l1_loss(theta + h * d, 3, cam, tgt) - orc.l1_loss(theta - h * d, 3, cam, tgt)) / (2 * h)
    assert abs(fd - (g * d).sum()) < 1e-5 * abs(fd)


def test_adam_constant_gradient_closed_form(orc):
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2, so every step moves theta by lr g / (|g| + eps)."""
    n, P = 3, 59
    rng = np.random.default_rng(1)
    theta = rng.normal(size=(n, P))
    g = rng.normal(size=(n, P))
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    t0 = theta.copy()
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    grp = np.array([0] * 3 + [1] + [2] * 3 + [3] * 4 + [4] * 3 + [5] * 45)
    for step in range(1, 6):
        orc.adam(theta, g, m, v, step, lr=lr, eps=1e-8)
    ref = t0 - 5 * lr[grp][None, :] * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(theta, ref, rtol=1e-9, atol=1e-12)
