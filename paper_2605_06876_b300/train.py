"""A small densification loop on synthetic scenes: the adaptive density control of
Sec. 3 with AdpSplit as its split operator, against the vanilla N = 2 split.

A coarse model is fitted to renders of a seeded ground-truth scene. Every
iteration renders one training view, takes the L1 loss backward (accumulating the
image-space statistic of Eq. 2) and one Adam step. Every `interval` iterations until
`densify_until`, Eq. 2 picks the split and clone candidates from the statistic of
the interval. The split candidates are then split either by AdpSplit, with the error
regions of `n_sampled` training views rendered in one batched launch, or by the
vanilla split (every candidate gets two children, Eqs. 3-4). The clones are
appended after the split. The loss (L1 only) and the optimizer are those of the
single step. Pruning, opacity resets and the other baseline-specific rules are not
part of the comparison. Quality is the PSNR of held-out views at the end.

Every step runs in this library's kernels; the loop itself only reads the new
population size back after each densification (to size the next buffers).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _abi as A
from . import ops


def _target_views(gt: ops.Gaussians, cams):
    """Renders of the ground truth, one image per camera (batched launches of at most
    ADP_MAX_VIEWS views)."""
    out = []
    for c0 in range(0, len(cams), A.ADP_MAX_VIEWS):
        part = cams[c0:c0 + A.ADP_MAX_VIEWS]
        pr = ops.project(gt, part)
        bins = ops.bin_sort(gt.n, pr, part)
        img = ops.render(gt.n, pr, bins, part)
        off = 0
        for c in part:
            P = int(c["width"]) * int(c["height"])
            out.append(img.rgb[off:off + P].clone())
            off += P
    return out


def psnr(model: ops.Gaussians, cams, targets):
    """Mean PSNR over views (images in [0, 1], MSE over pixels and channels)."""
    vals = []
    for c, t in zip(cams, targets):
        pr = ops.project(model, [c])
        img = ops.render(model.n, pr, ops.bin_sort(model.n, pr, [c]), [c])
        mse = float(((img.rgb.clamp(0.0, 1.0) - t) ** 2).mean())
        vals.append(10.0 * math.log10(1.0 / max(mse, 1e-12)))
    return float(np.mean(vals))


def _rows(g: ops.Gaussians, n):
    """The first n rows of a (capacity) population as a population of n."""
    out = ops.Gaussians(n, g.sh_degree, g.mean_logit.device, zero=False)
    for d, s in zip(out.tensors(), g.tensors()):
        if d.dim() == 3:
            d.copy_(s[:, :n])
        else:
            d.copy_(s[:n])
    return out


def train(model: ops.Gaussians, train_cams, train_targets, mode="adpsplit", iters=2000,
          interval=100, densify_from=100, densify_until=1000, n_sampled=10, tau_g=2e-4,
          tau_s=0.05, params=None, seed=0, lr=ops.ADAM_LR):
    """Fits model (modified in place through its returned replacement) and returns
    (final population, stats). mode: 'adpsplit' or 'vanilla'."""
    assert mode in ("adpsplit", "vanilla")
    params = params or A.default_params()
    dev = model.mean_logit.device
    rng = np.random.default_rng(seed)
    g = model
    m, v = g.zeros_like(), g.zeros_like()
    grad = ops.Gaussians(g.n, g.sh_degree, dev, zero=False, row_mask=True)
    accum = torch.zeros(g.n, dtype=torch.float32, device=dev)
    visits = torch.zeros(g.n, dtype=torch.int32, device=dev)
    step_t = torch.ones(1, dtype=torch.int32, device=dev)
    V = len(train_cams)
    counts = []
    split_total = clone_total = 0
    statuses = {"adaptive": 0, "fallback": 0, "reset": 0, "children": 0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(1, iters + 1):
        vi = int(rng.integers(V))
        cam = [train_cams[vi]]
        pr = ops.project(g, cam, params)
        bins = ops.bin_sort(g.n, pr, cam, params)
        img = ops.render(g.n, pr, bins, cam, params=params)
        ops.render_backward(g, pr, bins, img, cam, target=train_targets[vi], params=params,
                            grad=grad, grad2d_accum=accum, grad2d_visits=visits)
        ops.adam_step(g, grad, m, v, step_t, lr)
        if densify_from <= it <= densify_until and it % interval == 0:
            g, m, v, ns, nc, st = _densify(g, m, v, accum, visits, train_cams, train_targets,
                                           mode, n_sampled, tau_g, tau_s, params, rng)
            for k_ in statuses:
                statuses[k_] += st[k_]
            split_total += ns
            clone_total += nc
            grad = ops.Gaussians(g.n, g.sh_degree, dev, zero=False, row_mask=True)
            accum = torch.zeros(g.n, dtype=torch.float32, device=dev)
            visits = torch.zeros(g.n, dtype=torch.int32, device=dev)
            counts.append(g.n)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return g, {"mode": mode, "iterations": iters, "seconds": round(seconds, 3),
               "final_gaussians": g.n, "population_after_each_densification": counts,
               "split_candidates": split_total, "clones": clone_total, "split_status": statuses}


def _densify(g, m, v, accum, visits, cams, targets, mode, n_sampled, tau_g, tau_s, params, rng):
    dev = g.mean_logit.device
    n = g.n
    sets = ops.densify_select(accum, visits, g, tau_g, tau_s)
    cand = sets.split  # the whole list (-1 past the count)
    idx = rng.choice(len(cams), size=min(n_sampled, len(cams)), replace=False)
    views = [cams[i] for i in idx]
    tgt = torch.cat([targets[i] for i in idx])
    pr = ops.project(g, views, params)
    bins = ops.bin_sort(n, pr, views, params)
    img = ops.render(n, pr, bins, views, params=params)
    maps, count, mass = ops.error_stats(img.rgb, tgt, img.dominant, n, views, params)
    if mode == "vanilla":
        count = torch.zeros_like(count)  # no attributed error pixel: every candidate splits in two
        regions = ops.Regions.alloc(1, None, dev)
        regions.count.zero_()
    else:
        regions = ops.error_regions(maps, img.dominant, tgt, n, views, cand, params)
    plan = ops.split_plan(g, views, regions, cand, count, params)
    ns, nc = (int(x) for x in sets.counts.cpu())
    cap = plan.new_n + nc
    noise = torch.as_tensor(rng.standard_normal((n, 2, 3)), dtype=torch.float32, device=dev)
    out = ops.Gaussians(cap, g.sh_degree, dev, zero=False)
    m_out = ops.Gaussians(cap, g.sh_degree, dev, zero=False)
    v_out = ops.Gaussians(cap, g.sh_degree, dev, zero=False)
    ops.split_apply(g, plan, regions, cand, noise, params, m_in=m, v_in=v, out=out, m_out=m_out,
                    v_out=v_out)
    d_new = ops.split_clone(g, plan, regions, cand, sets.clone, sets.counts[1:], n, out, m_out,
                            v_out)
    new_n = int(d_new.item())
    assert new_n <= cap
    status = plan.status[:ns].long()
    st = {"adaptive": int((status == A.ADP_ADAPTIVE).sum()),
          "fallback": int((status == A.ADP_FALLBACK).sum()),
          "reset": int((status == A.ADP_RESET).sum()),
          "children": int(plan.n_children[:ns].sum())}
    return _rows(out, new_n), _rows(m_out, new_n), _rows(v_out, new_n), ns, nc, st


def compare(gt: ops.Gaussians, init: ops.Gaussians, train_cams, test_cams, **kw):
    """Trains copies of init with both split operators; returns their statistics with
    the test-view PSNR of each."""
    train_t = _target_views(gt, train_cams)
    test_t = _target_views(gt, test_cams)
    res = {"initial_psnr": round(psnr(init, test_cams, test_t), 3)}
    for mode in ("vanilla", "adpsplit"):
        g, st = train(init.clone(), train_cams, train_t, mode=mode, **kw)
        st["test_psnr"] = round(psnr(g, test_cams, test_t), 3)
        st["train_psnr"] = round(psnr(g, train_cams, train_t), 3)
        res[mode] = st
    return res
