"""GPU parity of the adaptive density control pieces (Sec. 3, Eq. 2): the image-space
statistic accumulated by the backward, the split/clone selection, and the clone
append after the AdpSplit compaction."""
import numpy as np
import pytest
import torch

import oracle as O
import scenes
from gpu_util import DEV, np_, small_cluster_inputs
from paper_2605_06876_b300 import ops

pytestmark = pytest.mark.gpu


def test_backward_accumulates_the_ndc_gradient_statistic():
    sc, cams = small_cluster_inputs(1500, 96, 64, views=2, seed=41)
    theta = O.theta_of(sc)
    targets = [O.render(O.project(O.theta_of(scenes.scene_clusters(42 + v, 1000, 3)), 3, c), c)
               ["rgb"].astype(np.float32) for v, c in enumerate(cams)]
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams)
    tgt = torch.as_tensor(np.concatenate([t.reshape(-1, 3) for t in targets]), device=DEV)
    accum = torch.full((g.n,), 0.25, dtype=torch.float32, device=DEV)  # adds to what is there
    visits = torch.full((g.n,), 3, dtype=torch.int32, device=DEV)
    ops.render_backward(g, pr, bins, img, cams, target=tgt, grad2d_accum=accum,
                        grad2d_visits=visits)
    torch.cuda.synchronize()
    want = np.full(g.n, 0.25)
    want_v = np.full(g.n, 3)
    allid = np.arange(g.n, dtype=np.int32)
    for cam, t in zip(cams, targets):
        # the loss of a multi-view launch is the sum of each view's mean L1 error
        _, m2 = O.grad(theta, 3, cam, t, sel=allid, return_mean2d=True)
        seen = O.project(theta, 3, cam)["tiles"] > 0
        want += np.where(seen, O.densify_stat_ndc(m2, cam["width"], cam["height"]), 0.0)
        want_v += seen
    got = np_(accum).astype(np.float64)
    assert np.array_equal(np_(visits), want_v)
    rel = np.abs(got - want).max() / (np.abs(want - 0.25).max() + 1e-30)
    assert rel <= 2e-3, rel
    assert (want - 0.25).max() > 0


def test_selection_matches_the_oracle_bit_for_bit():
    rng = np.random.default_rng(5)
    n = 50_000
    sc = scenes.scene_clusters(43, n, 0)
    accum = rng.exponential(3e-4, n).astype(np.float32)
    visits = rng.integers(0, 6, n).astype(np.int32)
    # many exact ties at the gradient threshold and at the scale threshold
    tau_g, tau_s = np.float32(2e-4), 0.06
    accum[::97] = np.float32(4e-4)
    visits[::97] = 2
    ls = sc["logscale"].copy()
    ls[::89, 0] = np.float32(np.log(tau_s))
    sc["logscale"] = ls
    g = ops.Gaussians.from_scene(sc, DEV)
    out = ops.densify_select(torch.as_tensor(accum, device=DEV), torch.as_tensor(visits, device=DEV),
                             g, float(tau_g), tau_s)
    torch.cuda.synchronize()
    ns, ncl = (int(x) for x in np_(out.counts))
    split, clone = O.densify_select(accum, visits, ls, tau_g, tau_s)
    assert ns == len(split) and ncl == len(clone) and ns > 100 and ncl > 100
    assert np.array_equal(np_(out.split[:ns]), split)
    assert np.array_equal(np_(out.clone[:ncl]), clone)


def test_clone_append_after_the_split_compaction():
    from test_gpu_split import _oracle_case  # the oracle-side split of the tiny workload
    from gpu_util import c0_inputs

    sc, cam, target = c0_inputs()
    k = 200
    orc = _oracle_case(sc, [cam], [target], k)
    sp = orc["split"]
    n = sc["mean"].shape[0]
    cand = set(orc["cand"].tolist())
    rng = np.random.default_rng(7)
    clone_ids = np.sort(rng.choice([i for i in range(n) if i not in cand], 37, replace=False))
    clone_ids = clone_ids.astype(np.int32)
    g = ops.Gaussians.from_scene(sc, DEV)
    rg = orc["regions"]
    regs = ops.Regions.from_arrays(rg["view"], rg["parent"], rg["label"], rg["stats"], rg["band"],
                                   rg["moments"], DEV)
    cand_t = torch.as_tensor(orc["cand"], device=DEV)
    plan = ops.split_plan(g, [cam], regs, cand_t, torch.as_tensor(orc["count"], device=DEV))
    cap = plan.new_n + len(clone_ids) + 5
    out = ops.Gaussians(cap, g.sh_degree, DEV, zero=True)
    m_out = ops.Gaussians(cap, g.sh_degree, DEV, zero=False)
    v_out = ops.Gaussians(cap, g.sh_degree, DEV, zero=False)
    for t in m_out.tensors() + v_out.tensors():
        t.fill_(9.0)
    noise = torch.as_tensor(scenes.fallback_noise(7, k), device=DEV)
    m_in, v_in = g.zeros_like(), g.zeros_like()
    ops.split_apply(g, plan, regs, cand_t, noise, m_in=m_in, v_in=v_in, out=out, m_out=m_out,
                    v_out=v_out)
    ids_t = torch.as_tensor(clone_ids, device=DEV)
    cnt = torch.tensor([len(clone_ids)], dtype=torch.int64, device=DEV)
    d_new_n = ops.split_clone(g, plan, regs, cand_t, ids_t, cnt, len(clone_ids), out, m_out, v_out)
    torch.cuda.synchronize()
    new_n = int(d_new_n.item())
    assert new_n == plan.new_n + len(clone_ids)
    ref = O.clone_rows(sp["theta"], n, sp["status"], orc["cand"], clone_ids)
    got = O.theta_of(out.to_scene())
    # the clones copy the kept rows bit for bit (kept rows equal the oracle's exactly)
    np.testing.assert_array_equal(got[plan.new_n:new_n], ref[plan.new_n:new_n])
    for t in m_out.tensors() + v_out.tensors():
        part = t[:, plan.new_n:new_n] if t.dim() == 3 else t[plan.new_n:new_n]
        assert not bool(part.any())
    # too small a capacity: nothing written, the required size reported
    small = ops.Gaussians(plan.new_n + 3, g.sh_degree, DEV, zero=True)
    ops.split_apply(g, plan, regs, cand_t, noise, out=small)
    before = small.mean_logit.clone()
    d2 = ops.split_clone(g, plan, regs, cand_t, ids_t, cnt, len(clone_ids), small)
    torch.cuda.synchronize()
    assert int(d2.item()) == new_n
    assert torch.equal(small.mean_logit, before)


def test_eq2_step_invariants_and_graph_replay():
    from paper_2605_06876_b300 import _abi as A
    from paper_2605_06876_b300.pipeline import DensifyStep

    sc, cams = small_cluster_inputs(20000, 320, 208, seed=44)
    tg = ops.Gaussians.from_scene(scenes.scene_clusters(45, 30000, 3), DEV)
    prt = ops.project(tg, cams)
    target = ops.render(tg.n, prt, ops.bin_sort(tg.n, prt, cams), cams).rgb.clone()
    g = ops.Gaussians.from_scene(sc, DEV)
    st = DensifyStep(g, cams, target, tau_g=2e-4, tau_s=0.05)
    n = g.n
    noise = torch.as_tensor(scenes.fallback_noise(46, n), device=DEV)
    g0 = st.g.clone()
    out, m_out, v_out, plan = st.step(noise)
    torch.cuda.synchronize()
    assert st.check_capacity(plan)
    ns, ncl = (int(x) for x in np_(st.sets.counts))
    split, clone = np_(st.sets.split), np_(st.sets.clone)
    assert ns > 0 and ncl > 0
    assert np.all(np.diff(split[:ns]) > 0) and np.all(split[ns:] == -1)
    assert np.all(np.diff(clone[:ncl]) > 0) and np.all(clone[ncl:] == -1)
    assert not set(split[:ns]) & set(clone[:ncl])
    status, nch = np_(plan.status).astype(np.int64), np_(plan.n_children).astype(np.int64)
    assert np.all(status[ns:] == A.ADP_KEEP) and not nch[ns:].any()
    planned = int(plan.d_new_n.item())
    assert planned == (n + (status == A.ADP_FALLBACK).sum() +
                       nch[status == A.ADP_ADAPTIVE].sum())
    new_n = int(st.d_new_n.item())
    assert new_n == planned + ncl
    # each clone copies its parent's kept row (non-candidates keep their id order)
    keep = np.ones(n, bool)
    keep[split[:ns]] = status[:ns] == A.ADP_RESET
    rows = (np.cumsum(keep) - 1)[clone[:ncl]]
    th = O.theta_of(out.to_scene())
    np.testing.assert_array_equal(th[planned:new_n], th[rows])
    # a captured step replays to the same decisions as the eager one (from the same
    # input): the lists, statuses and sizes (values differ in the last bits, since the
    # backward's float atomics sum in any order)
    lists = (split.copy(), clone.copy(), status.copy())
    st.capture(noise)
    for d, s_ in zip(st.g.tensors(), g0.tensors()):
        d.copy_(s_)
    for t in st.m.tensors() + st.v.tensors():
        t.zero_()
    st.adam_t.fill_(1)
    _, _, _, plan2 = st.replay()
    torch.cuda.synchronize()
    assert int(st.d_new_n.item()) == new_n
    assert np.array_equal(np_(st.sets.split), lists[0])
    assert np.array_equal(np_(st.sets.clone), lists[1])
    assert np.array_equal(np_(plan2.status).astype(np.int64), lists[2])
