"""Gradients with a row mask: the backward writes only the rows of Gaussians that
some view renders (and the mask), the Adam entry points read only those rows.
Both must give the same results as the dense gradient, whose other rows are
zero."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import DEV, small_cluster_inputs
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.pipeline import PlainStep

pytestmark = pytest.mark.gpu


def _masked_grad_like(g, fill):
    gm = ops.Gaussians(g.n, g.sh_degree, DEV, zero=False, row_mask=True)
    for t in gm.tensors():
        t.fill_(fill)
    gm.rows.fill_(7)
    return gm


def test_masked_backward_writes_rendered_rows_only():
    sc, cams = small_cluster_inputs(6000, 160, 112, views=2, seed=31)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams)
    tgt = torch.rand((img.rgb.shape[0], 3), device=DEV, generator=torch.Generator(DEV).manual_seed(2))
    dense = ops.render_backward(g, pr, bins, img, cams, target=tgt)
    masked = _masked_grad_like(g, 7.0)
    ops.render_backward(g, pr, bins, img, cams, target=tgt, grad=masked)
    torch.cuda.synchronize()
    seen = (pr.tiles.view(len(cams), g.n) > 0).any(0)
    assert torch.equal(masked.rows != 0, seen)
    assert 0 < int(seen.sum()) < g.n
    for a, b in zip(dense.tensors(), masked.tensors()):
        if a.dim() == 3:
            a_on, b_on, b_off, a_off = a[:, seen], b[:, seen], b[:, ~seen], a[:, ~seen]
        else:
            a_on, b_on, b_off, a_off = a[seen], b[seen], b[~seen], a[~seen]
        # float atomics sum in any order: equal up to the last bits
        scale = a_on.abs().max().item() + 1e-30
        assert (a_on - b_on).abs().max().item() <= 1e-5 * scale
        assert not a_off.any()               # the dense gradient zeroes those rows
        assert bool((b_off == 7.0).all())    # the masked one never touches them


def _random_state(g, seed):
    gen = torch.Generator(DEV).manual_seed(seed)
    grad, m, v = g.zeros_like(), g.zeros_like(), g.zeros_like()
    for t in grad.tensors():
        t.normal_(0.0, 1e-2, generator=gen)
    for t in m.tensors():
        t.normal_(0.0, 1e-3, generator=gen)
    for t in v.tensors():
        t.uniform_(0.0, 1e-4, generator=gen)
    keep = torch.rand(g.n, device=DEV, generator=gen) < 0.3
    return grad, m, v, keep


def _dense_and_masked(grad, keep):
    """The dense gradient (rows outside keep zeroed) and the same gradient with a
    row mask whose masked-out rows hold NaN (they must never be read)."""
    dense = grad.clone()
    masked = ops.Gaussians(grad.n, grad.sh_degree, DEV, zero=False, row_mask=True)
    for d, mk, s in zip(dense.tensors(), masked.tensors(), grad.tensors()):
        mk.copy_(s)
        if d.dim() == 3:
            d[:, ~keep] = 0.0
            mk[:, ~keep] = float("nan")
        else:
            d[~keep] = 0.0
            mk[~keep] = float("nan")
    masked.rows.copy_(keep.to(torch.uint8))
    return dense, masked


def test_masked_adam_step_equals_dense():
    sc, _ = small_cluster_inputs(5000, 64, 64, seed=33)
    g0 = ops.Gaussians.from_scene(sc, DEV)
    grad, m0, v0, keep = _random_state(g0, 4)
    dense, masked = _dense_and_masked(grad, keep)
    out = []
    for gr in (dense, masked):
        g, m, v = g0.clone(), m0.clone(), v0.clone()
        ops.adam_step(g, gr, m, v, 3)
        rows = torch.arange(0, g.n, 7, dtype=torch.int32, device=DEV)
        ops.adam_step_rows(g, gr, m, v, rows, 4)
        torch.cuda.synchronize()
        out.append(g.tensors() + m.tensors() + v.tensors())
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_masked_fused_adam_compaction_equals_dense():
    sc, cams = small_cluster_inputs(8000, 160, 112, seed=35)
    tg = scenes.scene_clusters(36, 12000, 3)
    gt = ops.Gaussians.from_scene(tg, DEV)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    st = PlainStep(ops.Gaussians.from_scene(sc, DEV), cams, target, 0.1)
    noise = torch.as_tensor(scenes.fallback_noise(9, st.k), device=DEV)
    st.step(noise)
    torch.cuda.synchronize()
    grad, m0, v0, keep = _random_state(st.g, 6)
    dense, masked = _dense_and_masked(grad, keep)
    res = []
    for gr in (dense, masked):
        g, m, v = st.g.clone(), m0.clone(), v0.clone()
        d_step = torch.full((1,), 2, dtype=torch.int32, device=DEV)
        out = [ops.Gaussians(st.out_capacity, g.sh_degree, DEV, zero=True) for _ in range(3)]
        ops.adam_step_rows(g, gr, m, v, st.cand, d_step, st.lr)
        plan = ops.split_plan(g, st.cams, st.regions, st.cand, st.count, st.params, sync=False)
        ops.split_apply_adam(g, gr, m, v, plan, st.regions, st.cand, noise, d_step, out[0], out[1],
                             out[2], st.params, st.lr)
        torch.cuda.synchronize()
        res.append((int(plan.d_new_n.item()), out))
    (n1, o1), (n2, o2) = res
    assert n1 == n2 > st.g.n
    for a, b in zip(sum((x.tensors() for x in o1), []), sum((x.tensors() for x in o2), [])):
        if a.dim() == 3:
            assert torch.equal(a[:, :n1], b[:, :n1])
        else:
            assert torch.equal(a[:n1], b[:n1])
