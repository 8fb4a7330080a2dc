"""GPU parity of the error statistics against the FP64 oracle.

The error map, mask and bands are decided in float32 with correctly rounded
operations on both sides, so given the same image they are bit-exact; the
per-Gaussian mass is an exact sum on both sides; labels, moments and top-k ids are
integers and must match exactly; region statistics are FP64 on both sides.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, np_
from paper_2605_06876_b300 import _abi, ops

pytestmark = pytest.mark.gpu


def _cams(sizes):
    return [scenes.camera_origin_forward(w, h) for (w, h) in sizes]


def _inputs(sizes, n_gauss, seed):
    imgs, tgts, doms = [], [], []
    for k, (w, h) in enumerate(sizes):
        i, t, d = scenes.error_stage_inputs(seed + k, w, h, n_gauss)
        imgs.append(i.reshape(-1, 3))
        tgts.append(t.reshape(-1, 3))
        doms.append(d.reshape(-1))
    cat = lambda a: np.ascontiguousarray(np.concatenate(a))
    return cat(imgs), cat(tgts), cat(doms)


@pytest.mark.parametrize("sizes,n_gauss", [([(97, 61)], 40), ([(1280, 832)], 5000),
                                           ([(200, 120), (64, 48), (131, 77)], 300)])
def test_error_stats_bit_exact(sizes, n_gauss):
    img, tgt, dom = _inputs(sizes, n_gauss, 11)
    cams = _cams(sizes)
    t = lambda a: torch.as_tensor(a, device=DEV)
    maps, count, mass = ops.error_stats(t(img), t(tgt), t(dom), n_gauss, cams)
    torch.cuda.synchronize()
    off = 0
    c_ref = np.zeros(n_gauss, np.int32)
    m_ref = np.zeros(n_gauss)
    for v, (w, h) in enumerate(sizes):
        P = w * h
        em = O.error_map(img[off:off + P].reshape(h, w, 3), tgt[off:off + P].reshape(h, w, 3), 0.1, 3)
        assert np.array_equal(np_(maps.E[off:off + P]), em["E"])
        mask = np_(maps.mask[off:off + P])
        assert np.array_equal(mask & 1, em["M"])
        assert np.array_equal(mask >> 4, em["B"])
        assert np.array_equal(np_(maps.minmax[v]), em["minmax"])
        O.gauss_stats(em["M"], dom[off:off + P], em["E"], n_gauss, c_ref, m_ref)
        off += P
    assert np.array_equal(np_(count), c_ref)
    assert np.array_equal(np_(mass), m_ref)  # exact sums of float32 values in (0.1, 1]


def test_select_topk_bit_exact():
    rng = np.random.default_rng(2)
    n = 300_000
    mass = np.floor(rng.exponential(3.0, n) * 8) / 8  # many exact ties
    mass[rng.uniform(size=n) < 0.3] = 0.0
    t = torch.as_tensor(mass, device=DEV)
    for k in (0, 1, 17, 1000, 29_999, n - 1, n):
        got = np_(ops.select_topk(t, n, k))
        assert np.array_equal(got, O.topk_mass(mass, k)), k


@pytest.mark.parametrize("sizes,n_gauss,r", [([(150, 110)], 30, 1), ([(1280, 832)], 3000, 2),
                                             ([(160, 100), (90, 70)], 200, 0)])
def test_regions_bit_exact(sizes, n_gauss, r):
    img, tgt, dom = _inputs(sizes, n_gauss, 23)
    cams = _cams(sizes)
    prm = _abi.default_params(r_erode=r)
    t = lambda a: torch.as_tensor(a, device=DEV)
    maps, count, mass = ops.error_stats(t(img), t(tgt), t(dom), n_gauss, cams, prm)
    cand = np.arange(0, n_gauss, 3, dtype=np.int32)
    regs = ops.error_regions(maps, t(dom), t(tgt), n_gauss, cams, t(cand), prm, labels=True)
    torch.cuda.synchronize()
    flag = np.zeros(n_gauss, np.uint8)
    flag[cand] = 1
    parts = []
    off = 0
    mask = np_(maps.mask)
    labels = np_(regs.labels)
    for v, (w, h) in enumerate(sizes):
        P = w * h
        em = O.error_map(img[off:off + P].reshape(h, w, 3), tgt[off:off + P].reshape(h, w, 3), 0.1, 3)
        Mero = O.erode(em["M"], w, h, r)
        assert np.array_equal((mask[off:off + P] >> 1) & 1, Mero)
        rg = O.regions(v, w, h, Mero, em["B"], dom[off:off + P], n_gauss, flag,
                       tgt[off:off + P].reshape(h, w, 3), 5)
        assert np.array_equal(labels[off:off + P], rg["labels"])
        parts.append(rg)
        off += P
    ref = O.concat_regions(parts)
    got = regs.to_numpy()
    assert len(ref["view"]) > 3
    for k in ("view", "parent", "label", "band", "moments"):
        assert np.array_equal(got[k], ref[k]), k
    np.testing.assert_allclose(got["stats"], ref["stats"], rtol=1e-12, atol=1e-12)
    # without per-pixel labels (no flatten pass: the moments pass finds the roots)
    nolab = ops.error_regions(maps, t(dom), t(tgt), n_gauss, cams, t(cand), prm).to_numpy()
    for k in ("view", "parent", "label", "band", "moments"):
        assert np.array_equal(nolab[k], ref[k]), k
    np.testing.assert_allclose(nolab["stats"], ref["stats"], rtol=1e-12, atol=1e-12)


def test_regions_capacity_overflow_reports_count():
    img, tgt, dom = _inputs([(200, 150)], 50, 31)
    cams = _cams([(200, 150)])
    t = lambda a: torch.as_tensor(a, device=DEV)
    maps, _, _ = ops.error_stats(t(img), t(tgt), t(dom), 50, cams)
    cand = t(np.arange(50, dtype=np.int32))
    full = ops.error_regions(maps, t(dom), t(tgt), 50, cams, cand)
    R = int(full.count.item())
    assert R > 4
    small = ops.error_regions(maps, t(dom), t(tgt), 50, cams, cand, capacity=R // 2, grow=False)
    assert int(small.count.item()) == R
    got = small.to_numpy()
    ref = full.to_numpy()
    assert np.array_equal(got["label"], ref["label"][:R // 2])
