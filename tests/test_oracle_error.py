"""Pins of the oracle's error stage: error map (Eq. 6), mask and bands, erosion,
per-Gaussian attribution, top-k choice, error regions (Eqs. 7-8) and region
statistics. Each test checks against a library routine, numpy or brute force."""
import numpy as np
import pytest

import scenes

ndi = pytest.importorskip("scipy.ndimage")


def test_error_map_normalisation_and_invariance(orc):
    img, tgt, _ = scenes.error_stage_inputs(1, 40, 30, 50)
    em = orc.error_map(img, tgt, 0.1, 3)
    raw = np.abs(img.astype(np.float64) - tgt).sum(-1).reshape(-1)
    np.testing.assert_allclose(em["raw"], raw, rtol=1e-6)
    assert em["minmax"][0] == em["raw"].min() and em["minmax"][1] == em["raw"].max()
    assert em["E"].min() == 0.0 and em["E"].max() == 1.0
    np.testing.assert_allclose(em["E"], (raw - raw.min()) / (raw.max() - raw.min()), atol=1e-6)
    # scaling both images by a power of two is exact in float32 and leaves E unchanged
    em2 = orc.error_map(img * np.float32(0.5), tgt * np.float32(0.5), 0.1, 3)
    assert np.array_equal(em["E"], em2["E"]) and np.array_equal(em["B"], em2["B"])


def test_error_map_threshold_is_strict_and_bands(orc):
    # raw errors 0, 0.1, 0.4, 0.7, 1.0 (red channel only): E equals raw exactly
    vals = np.array([0.0, 0.1, 0.4, 0.7, 1.0, 0.7000001, 0.3999999], np.float32)
    img = np.zeros((1, len(vals), 3), np.float32)
    tgt = img.copy()
    tgt[0, :, 0] = vals
    em = orc.error_map(img, tgt, 0.1, 3)
    assert list(em["M"]) == [0, 0, 1, 1, 1, 1, 1]  # E = 0.1 is not > 0.1
    # bands split [0.1, 1] into thirds at 0.4 and 0.7
    assert list(em["B"]) == [0, 0, 1, 2, 2, 2, 0]
    flat = orc.error_map(img, img, 0.1, 3)
    assert not flat["M"].any() and not flat["E"].any()


def test_bands_partition_the_interval(orc):
    img, tgt, _ = scenes.error_stage_inputs(4, 64, 64, 30)
    for L in (1, 2, 3, 5):
        em = orc.error_map(img, tgt, 0.1, L)
        E = em["E"].astype(np.float64)
        m = em["M"].astype(bool)
        lo = 0.1 + em["B"][m] * 0.9 / L
        hi = lo + 0.9 / L
        assert np.all(E[m] >= lo - 1e-6) and np.all(E[m] <= hi + 1e-6)
        assert np.all(em["B"][~m] == 0)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_erosion_matches_scipy(orc, r):
    rng = np.random.default_rng(r)
    M = (rng.uniform(size=(37, 53)) < 0.8).astype(np.uint8)
    out = orc.erode(M.reshape(-1), 53, 37, r)
    if r == 0:
        ref = M
    else:
        ref = ndi.binary_erosion(M, structure=np.ones((2 * r + 1, 2 * r + 1)), border_value=1)
    assert np.array_equal(out.reshape(37, 53), ref.astype(np.uint8))


def test_gauss_stats_and_topk(orc):
    img, tgt, D = scenes.error_stage_inputs(7, 80, 60, 40)
    em = orc.error_map(img, tgt, 0.1, 3)
    count, mass = orc.gauss_stats(em["M"], D.reshape(-1), em["E"], 40)
    sel = (em["M"] == 1) & (D.reshape(-1) >= 0)
    ref_c = np.bincount(D.reshape(-1)[sel], minlength=40)
    ref_m = np.bincount(D.reshape(-1)[sel], weights=em["E"][sel].astype(np.float64), minlength=40)
    assert np.array_equal(count, ref_c)
    np.testing.assert_allclose(mass, ref_m, rtol=1e-15)
    mass2 = mass.copy()
    mass2[3] = mass2[7]  # a tie: the lower id wins
    for k in (0, 1, 7, 40):
        ids = orc.topk_mass(mass2, k)
        order = np.lexsort((np.arange(40), -mass2))[:k]
        assert list(ids) == sorted(order.tolist())


def _regions_by_scipy(Mero, B, D, cand_flag, W, H, m_min):
    """Components of each (dominant, band) class with scipy's 8-connected label."""
    valid = (Mero == 1) & (D >= 0) & cand_flag[np.maximum(D, 0)].astype(bool)
    out = []
    labels = np.full(W * H, -1, np.int64)
    for d, b in set(zip(D[valid].tolist(), B[valid].tolist())):
        mask = (valid & (D == d) & (B == b)).reshape(H, W)
        lab, nl = ndi.label(mask, structure=np.ones((3, 3)))
        for k in range(1, nl + 1):
            pix = np.flatnonzero(lab.reshape(-1) == k)
            labels[pix] = pix.min()
            if len(pix) >= m_min:
                out.append((int(pix.min()), d, b, pix))
    out.sort()
    return out, labels


def test_regions_match_scipy_label_and_numpy_moments(orc):
    img, tgt, D = scenes.error_stage_inputs(2, 96, 72, 25, n_cells=30)
    W, H = 96, 72
    em = orc.error_map(img, tgt, 0.1, 3)
    Mero = orc.erode(em["M"], W, H, 1)
    Df = D.reshape(-1)
    flag = np.zeros(25, np.uint8)
    flag[::2] = 1
    rg = orc.regions(3, W, H, Mero, em["B"], Df, 25, flag, tgt, m_min=5)
    ref, ref_labels = _regions_by_scipy(Mero, em["B"], Df, flag, W, H, 5)
    assert np.array_equal(rg["labels"], ref_labels)
    assert len(ref) == rg["label"].shape[0] > 5
    for k, (lab, d, b, pix) in enumerate(ref):
        assert rg["label"][k] == lab and rg["parent"][k] == d and rg["band"][k] == b
        assert rg["view"][k] == 3
        x, y = (pix % W).astype(np.int64), (pix // W).astype(np.int64)
        mom = [len(pix), x.sum(), y.sum(), (x * x).sum(), (x * y).sum(), (y * y).sum()]
        assert list(rg["moments"][k]) == mom
        st = rg["stats"][k]
        xy = np.stack([x, y], 0).astype(np.float64)
        cov = np.cov(xy, bias=True)
        np.testing.assert_allclose(st[0:2], xy.mean(1), rtol=1e-14)
        np.testing.assert_allclose(st[2:5], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-9, atol=1e-12)
        lam, vec = np.linalg.eigh(cov)
        np.testing.assert_allclose(st[7:9], np.sqrt(np.maximum(lam[::-1], 0)), rtol=1e-9, atol=1e-9)
        if lam[1] - lam[0] > 1e-9:
            e1 = vec[:, 1] * np.sign(vec[0, 1] if vec[0, 1] != 0 else vec[1, 1])
            np.testing.assert_allclose(st[5:7], e1, atol=1e-9)
        assert st[5] > 0 or (st[5] == 0 and st[6] > 0)
        xi = int(np.clip(np.floor(st[0] + 0.5), 0, W - 1))
        yi = int(np.clip(np.floor(st[1] + 0.5), 0, H - 1))
        np.testing.assert_array_equal(st[9:12], tgt[yi, xi].astype(np.float64))


def test_regions_small_cases_brute_force(orc):
    """Hand cases: a diagonal chain is one 8-connected region; a change of band
    or of dominant Gaussian splits it; areas below m_min are dropped."""
    W, H = 6, 5
    M = np.zeros((H, W), np.uint8)
    D = np.full((H, W), -1, np.int32)
    B = np.zeros((H, W), np.uint8)
    for k in range(5):  # diagonal chain of 5 pixels owned by Gaussian 2
        M[k, k] = 1
        D[k, k] = 2
    M[0, 5] = M[1, 5] = 1
    D[0, 5] = D[1, 5] = 2
    B[1, 5] = 1  # same owner, different band: two regions of area 1
    flag = np.array([0, 0, 1], np.uint8)
    tgt = np.zeros((H, W, 3), np.float32)
    rg = orc.regions(0, W, H, M.reshape(-1), B.reshape(-1), D.reshape(-1), 3, flag, tgt, m_min=1)
    assert list(rg["label"]) == [0, 5, 11]
    assert list(rg["moments"][:, 0]) == [5, 1, 1]
    rg5 = orc.regions(0, W, H, M.reshape(-1), B.reshape(-1), D.reshape(-1), 3, flag, tgt, m_min=5)
    assert list(rg5["label"]) == [0]
    flag0 = np.array([0, 0, 0], np.uint8)
    rg0 = orc.regions(0, W, H, M.reshape(-1), B.reshape(-1), D.reshape(-1), 3, flag0, tgt, m_min=1)
    assert rg0["label"].shape[0] == 0 and np.all(rg0["labels"] == -1)
