"""GPU parity of the AdpSplit operator and compaction, the backward and Adam
against the FP64 oracle.

The split stage runs in FP64 on both sides, so statuses and child counts must be
identical; the new population is compared value by value (children through their
covariance R diag(s^2) R^T, which is invariant to the sign and order freedom of the
axes). Gradients are compared with the oracle's complex-step derivative.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, c0_inputs, np_, small_cluster_inputs
from paper_2605_06876_b300 import ops

pytestmark = pytest.mark.gpu


def _sigma(ls, q):
    R = O.quat_to_rot(q)
    s = np.exp(np.asarray(ls, np.float64))
    return np.einsum("nij,nj,nkj->nik", R, s * s, R)


def _oracle_case(sc, cams, targets, k):
    out = O.plain_step(sc, cams, targets, k_cand=k,
                       noise=scenes.fallback_noise(7, k).astype(np.float64))
    return out


def _gpu_split(sc, cams, orc, noise):
    g = ops.Gaussians.from_scene(sc, DEV)
    rg = orc["regions"]
    regs = ops.Regions.from_arrays(rg["view"], rg["parent"], rg["label"], rg["stats"], rg["band"],
                                   rg["moments"], DEV)
    cand = torch.as_tensor(orc["cand"], device=DEV)
    count = torch.as_tensor(orc["count"], device=DEV)
    rng = np.random.default_rng(3)
    m_in = ops.Gaussians.from_scene({**sc, **{k: rng.normal(size=sc[k].shape).astype(np.float32)
                                              for k in ("mean", "logit", "logscale", "quat", "sh")}}, DEV)
    v_in = m_in.clone()
    plan = ops.split_plan(g, cams, regs, cand, count)
    out, m_out, v_out = ops.split_apply(g, plan, regs, cand, torch.as_tensor(noise, device=DEV),
                                        m_in=m_in, v_in=v_in)
    torch.cuda.synchronize()
    return g, plan, out, m_in, m_out


def _compare_split(sc, orc, plan, out, m_in, m_out):
    sp = orc["split"]
    assert np.array_equal(np_(plan.status), sp["status"])
    assert np.array_equal(np_(plan.n_children), sp["n_children"])
    assert plan.new_n == sp["new_n"] == out.n
    got = O.theta_of(out.to_scene())
    ref = sp["theta"]
    n = sc["mean"].shape[0]
    cand = set(orc["cand"].tolist())
    keep = [i for i in range(n) if i not in cand or sp["status"][list(orc["cand"]).index(i)] == O.RESET]
    nk = len(keep)
    assert np.array_equal(got[:nk], ref[:nk])  # kept Gaussians copied bit for bit
    mk = O.theta_of(m_out.to_scene())
    assert np.array_equal(mk[:nk], O.theta_of(m_in.to_scene())[keep])
    assert not mk[nk:].any()
    # appended Gaussians: centres, opacities, colours, covariances
    np.testing.assert_allclose(got[nk:, :3], ref[nk:, :3], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(got[nk:, 3], ref[nk:, 3], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(got[nk:, 11:], ref[nk:, 11:], rtol=1e-5, atol=1e-5)
    Sg = _sigma(got[nk:, 4:7], got[nk:, 7:11])
    Sr = _sigma(ref[nk:, 4:7], ref[nk:, 7:11])
    scale = np.abs(Sr).reshape(len(Sr), -1).max(1)[:, None, None]
    assert np.all(np.abs(Sg - Sr) <= 1e-5 * scale + 1e-12)


def test_split_c0_matches_oracle():
    sc, cam, target = c0_inputs()
    k = 200
    orc = _oracle_case(sc, [cam], [target], k)
    noise = scenes.fallback_noise(7, k)
    g, plan, out, m_in, m_out = _gpu_split(sc, [cam], orc, noise)
    st = orc["split"]["status"]
    assert (st == O.ADAPTIVE).sum() > 50
    _compare_split(sc, orc, plan, out, m_in, m_out)


def test_split_multiview_with_merges():
    """Several views of a cluster scene: proposals from different views of one
    parent merge (Eqs. 11-12) and the cap binds for some parents."""
    sc, cams = small_cluster_inputs(6000, 240, 160, views=4, seed=12)
    tg = scenes.scene_clusters(99, 9000, 3)
    targets = []
    for cam in cams:
        r = O.render(O.project(O.theta_of(tg), 3, cam), cam)
        targets.append(r["rgb"].astype(np.float32).reshape(cam["height"], cam["width"], 3))
    k = 600
    orc = O.plain_step(sc, cams, targets, k_cand=k, sp=O.SplitParams(n_max=4),
                       noise=scenes.fallback_noise(8, k).astype(np.float64))
    from paper_2605_06876_b300 import _abi
    prm = _abi.default_params(n_max=4)
    g = ops.Gaussians.from_scene(sc, DEV)
    rg = orc["regions"]
    regs = ops.Regions.from_arrays(rg["view"], rg["parent"], rg["label"], rg["stats"], rg["band"],
                                   rg["moments"], DEV)
    cand = torch.as_tensor(orc["cand"], device=DEV)
    plan = ops.split_plan(g, cams, regs, cand, torch.as_tensor(orc["count"], device=DEV), prm)
    out, _, _ = ops.split_apply(g, plan, regs, cand,
                                torch.as_tensor(scenes.fallback_noise(8, k), device=DEV), prm,
                                with_state=False)
    torch.cuda.synchronize()
    sp = orc["split"]
    assert np.array_equal(np_(plan.status), sp["status"])
    assert np.array_equal(np_(plan.n_children), sp["n_children"])
    assert (sp["n_children"] == 4).sum() > 0
    # at least one parent had more regions than children (merge or cap)
    per_parent = np.bincount(rg["parent"], minlength=sc["mean"].shape[0])[orc["cand"]]
    assert np.any(per_parent > sp["n_children"])
    got = O.theta_of(out.to_scene())
    ref = sp["theta"]
    np.testing.assert_allclose(got[:, :4], ref[:, :4], rtol=1e-5, atol=1e-5)
    Sg, Sr = _sigma(got[:, 4:7], got[:, 7:11]), _sigma(ref[:, 4:7], ref[:, 7:11])
    scale = np.abs(Sr).reshape(len(Sr), -1).max(1)[:, None, None]
    assert np.all(np.abs(Sg - Sr) <= 1e-5 * scale + 1e-12)


def test_backward_matches_oracle_gradient():
    """64 Gaussians at 32x32, SH degree 3: the GPU gradient of the mean L1 loss
    equals the oracle's complex-step derivative of its FP64 forward."""
    sc, cam = scenes.subscene_for_gradients(0)
    tsc, _ = scenes.subscene_for_gradients(1, n=48)
    tr = O.render(O.project(O.theta_of(tsc), 3, cam), cam)
    target = tr["rgb"].astype(np.float32).reshape(32, 32, 3)
    g, pr, bins, img = __import__("gpu_util").gpu_forward(sc, [cam])
    tgt = torch.as_tensor(target.reshape(-1, 3), device=DEV)
    grad = ops.render_backward(g, pr, bins, img, [cam], target=tgt)
    torch.cuda.synchronize()
    got = O.theta_of(grad.to_scene())
    ref = O.grad(O.theta_of(sc), 3, cam, target)
    groups = {"mean": slice(0, 3), "logit": slice(3, 4), "logscale": slice(4, 7),
              "quat": slice(7, 11), "sh": slice(11, 59)}
    for name, sl in groups.items():
        a, b = got[:, sl], ref[:, sl]
        tol = 2e-3 * np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() <= tol, (name, np.abs(a - b).max(), tol)
    assert np.abs(ref).max() > 0


def test_backward_upstream_gradient_and_views_sum():
    """With an explicit dL/dI the gradient is linear in it; two identical views
    give twice the gradient of one."""
    sc, cams = small_cluster_inputs(3000, 128, 96, seed=21)
    cam = cams[0]
    g = ops.Gaussians.from_scene(sc, DEV)
    pr1 = ops.project(g, [cam]); b1 = ops.bin_sort(g.n, pr1, [cam]); i1 = ops.render(g.n, pr1, b1, [cam])
    up = torch.randn((cam["width"] * cam["height"], 3), device=DEV)
    ga = ops.render_backward(g, pr1, b1, i1, [cam], dL_drgb=up)
    gb = ops.render_backward(g, pr1, b1, i1, [cam], dL_drgb=2 * up)
    pr2 = ops.project(g, [cam, cam]); b2 = ops.bin_sort(g.n, pr2, [cam, cam])
    i2 = ops.render(g.n, pr2, b2, [cam, cam])
    gc = ops.render_backward(g, pr2, b2, i2, [cam, cam], dL_drgb=torch.cat([up, up]))
    torch.cuda.synchronize()
    for a, b, c in zip(ga.tensors(), gb.tensors(), gc.tensors()):
        sc_ = a.abs().max().item() + 1e-30
        assert (2 * a - b).abs().max().item() <= 1e-5 * sc_
        assert (2 * a - c).abs().max().item() <= 1e-4 * sc_


def test_adam_matches_oracle():
    rng = np.random.default_rng(4)
    n, deg = 1000, 3
    mk = lambda: {"mean": rng.normal(size=(n, 3)).astype(np.float32),
                  "logit": rng.normal(size=n).astype(np.float32),
                  "logscale": rng.normal(size=(n, 3)).astype(np.float32),
                  "quat": rng.normal(size=(n, 4)).astype(np.float32),
                  "sh": rng.normal(size=(n, 16, 3)).astype(np.float32), "sh_degree": deg}
    p, gr, m = mk(), mk(), mk()
    v = {k: (np.abs(x) if k != "sh_degree" else x) for k, x in mk().items()}
    G = [ops.Gaussians.from_scene(d, DEV) for d in (p, gr, m, v)]
    for step in (1, 2, 3):
        ops.adam_step(G[0], G[1], G[2], G[3], step)
    torch.cuda.synchronize()
    th, g_, m_, v_ = (O.theta_of(d) for d in (p, gr, m, v))
    for step in (1, 2, 3):
        O.adam(th, g_, m_, v_, step)
    np.testing.assert_allclose(O.theta_of(G[0].to_scene()), th, rtol=2e-5, atol=2e-6)
    np.testing.assert_allclose(O.theta_of(G[2].to_scene()), m_, rtol=2e-5, atol=1e-6)


def test_split_apply_into_capacity_buffers_without_sync():
    """Planning without reading the size back and applying into buffers sized for
    the largest possible result gives the same population in the first new_n
    entries; a capacity below the planned size leaves the buffers untouched."""
    sc, cam, target = c0_inputs()
    k = 200
    orc = _oracle_case(sc, [cam], [target], k)
    g = ops.Gaussians.from_scene(sc, DEV)
    rg = orc["regions"]
    regs = ops.Regions.from_arrays(rg["view"], rg["parent"], rg["label"], rg["stats"], rg["band"],
                                   rg["moments"], DEV)
    cand = torch.as_tensor(orc["cand"], device=DEV)
    count = torch.as_tensor(orc["count"], device=DEV)
    noise = torch.as_tensor(scenes.fallback_noise(7, k), device=DEV)
    plan = ops.split_plan(g, [cam], regs, cand, count, sync=False)
    assert plan.new_n is None
    cap = g.n + k * 20
    big = ops.Gaussians(cap, 0, DEV, zero=True)
    ops.split_apply(g, plan, regs, cand, noise, with_state=False, out=big)
    exact, _, _ = ops.split_apply(g, plan, regs, cand, noise, with_state=False)
    torch.cuda.synchronize()
    new_n = int(plan.d_new_n.item())
    assert new_n == orc["split"]["new_n"] == exact.n
    for a, b in zip(big.tensors(), exact.tensors()):
        sl = (slice(None), slice(0, new_n)) if a.dim() == 3 else (slice(0, new_n),)
        assert torch.equal(a[sl], b)
    small = ops.Gaussians(new_n - 1, 0, DEV, zero=True)
    ops.split_apply(g, plan, regs, cand, noise, with_state=False, out=small)
    torch.cuda.synchronize()
    assert all(int(t.abs().sum().item()) == 0 for t in small.tensors())


def test_overlapped_split_equals_two_call_split():
    """The overlapped plan and compaction (proposals and merges on the library's
    auxiliary stream while the kept rows stream) give, bit for bit, what the
    two-call plan and fused compaction give: statuses, child counts, new size,
    population and moments. So does the overlapped plan made in two calls, its
    first part on a side stream beside the candidates' Adam step. Three capacities: the worst case (kept rows written
    against the bound on the new size), exactly the new size (merges remove
    children here, so the bound exceeds the capacity and the kept rows are
    written after the join), and one row less (nothing written)."""
    sc, cams = small_cluster_inputs(6000, 240, 160, views=4, seed=12)
    tg = scenes.scene_clusters(99, 9000, 3)
    targets = []
    for cam in cams:
        r = O.render(O.project(O.theta_of(tg), 3, cam), cam)
        targets.append(r["rgb"].astype(np.float32).reshape(cam["height"], cam["width"], 3))
    k, n_max = 600, 4
    orc = O.plain_step(sc, cams, targets, k_cand=k, sp=O.SplitParams(n_max=n_max),
                       noise=scenes.fallback_noise(8, k).astype(np.float64))
    from paper_2605_06876_b300 import _abi
    prm = _abi.default_params(n_max=n_max)
    g0 = ops.Gaussians.from_scene(sc, DEV)
    rg = orc["regions"]
    regs = ops.Regions.from_arrays(rg["view"], rg["parent"], rg["label"], rg["stats"], rg["band"],
                                   rg["moments"], DEV)
    cand = torch.as_tensor(orc["cand"], device=DEV)
    count = torch.as_tensor(orc["count"], device=DEV)
    noise = torch.as_tensor(scenes.fallback_noise(8, k), device=DEV)
    gen = torch.Generator(DEV).manual_seed(9)
    grad, m0, v0 = g0.zeros_like(), g0.zeros_like(), g0.zeros_like()
    for t in grad.tensors():
        t.normal_(0.0, 1e-2, generator=gen)
    for t in m0.tensors():
        t.normal_(0.0, 1e-3, generator=gen)
    for t in v0.tensors():
        t.uniform_(0.0, 1e-4, generator=gen)
    n = g0.n
    worst = n + k * (n_max + 1)

    def run(mode, cap):
        g, m, v = g0.clone(), m0.clone(), v0.clone()
        d_step = torch.full((1,), 3, dtype=torch.int32, device=DEV)
        out = [ops.Gaussians(cap, g.sh_degree, DEV, zero=True) for _ in range(3)]
        if mode == "two_call":
            # the first part on a side stream, beside the candidates' Adam step
            main, side = torch.cuda.current_stream(), torch.cuda.Stream()
            side.wait_stream(main)
            with torch.cuda.stream(side):
                plan = ops.split_plan_overlapped(g, cams, regs, cand, count, prm,
                                                 part="statuses")
            ops.adam_step_rows(g, grad, m, v, cand, d_step, ops.ADAM_LR)
            main.wait_stream(side)
            plan = ops.split_plan_overlapped(g, cams, regs, cand, count, prm, part="proposals",
                                             plan=plan)
        else:
            ops.adam_step_rows(g, grad, m, v, cand, d_step, ops.ADAM_LR)
            if mode == "overlapped":
                plan = ops.split_plan_overlapped(g, cams, regs, cand, count, prm)
            else:
                plan = ops.split_plan(g, cams, regs, cand, count, prm, sync=False)
        ops.split_apply_adam(g, grad, m, v, plan, regs, cand, noise, d_step, out[0], out[1],
                             out[2], prm, ops.ADAM_LR, overlapped=mode != "plain")
        torch.cuda.synchronize()
        return plan, out, int(d_step.item())

    ref_plan, ref_out, ref_step = run("plain", worst)
    n_new = int(ref_plan.d_new_n.item())
    st = np_(ref_plan.status)
    per_parent = np.bincount(rg["parent"], minlength=n)[orc["cand"]]
    bound = n + int(np.minimum(per_parent[st == 1], n_max).sum()) + int((st == 2).sum())
    assert n < n_new < bound <= worst

    def rows(gs, upto):
        return [t[:, :upto] if t.dim() == 3 else t[:upto] for x in gs for t in x.tensors()]

    for mode, cap in itertools.product(("overlapped", "two_call"), (worst, n_new, n_new - 1)):
        plan, out, step = run(mode, cap)
        assert torch.equal(plan.status, ref_plan.status)
        assert torch.equal(plan.n_children, ref_plan.n_children)
        assert int(plan.d_new_n.item()) == n_new and step == ref_step == 4
        if cap >= n_new:
            for a, b in zip(rows(out, n_new), rows(ref_out, n_new)):
                assert torch.equal(a, b)
        else:
            assert all(int(torch.count_nonzero(t)) == 0 for x in out for t in x.tensors())
