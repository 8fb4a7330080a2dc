"""The whole plain step: a step replayed from a captured CUDA graph equals the same
step launched eagerly, and Adam's device-side step counter equals host-side steps."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, small_cluster_inputs
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.pipeline import PlainStep

import scenes

pytestmark = pytest.mark.gpu


def test_adam_device_step_counter_matches_host_steps():
    rng = np.random.default_rng(0)
    n = 5000
    mk = lambda: {"mean": rng.normal(size=(n, 3)).astype(np.float32),
                  "logit": rng.normal(size=n).astype(np.float32),
                  "logscale": rng.normal(size=(n, 3)).astype(np.float32),
                  "quat": rng.normal(size=(n, 4)).astype(np.float32),
                  "sh": rng.normal(size=(n, 16, 3)).astype(np.float32), "sh_degree": 3}
    p, g = mk(), mk()
    A = [ops.Gaussians.from_scene(p, DEV), ops.Gaussians.from_scene(g, DEV)]
    B = [ops.Gaussians.from_scene(p, DEV), ops.Gaussians.from_scene(g, DEV)]
    ma, va = A[0].zeros_like(), A[0].zeros_like()
    mb, vb = B[0].zeros_like(), B[0].zeros_like()
    d_step = torch.ones(1, dtype=torch.int32, device=DEV)
    for t in (1, 2, 3):
        ops.adam_step(A[0], A[1], ma, va, t)
        ops.adam_step(B[0], B[1], mb, vb, d_step)
    torch.cuda.synchronize()
    assert int(d_step.item()) == 4
    for x, y in zip(A[0].tensors() + ma.tensors(), B[0].tensors() + mb.tensors()):
        torch.testing.assert_close(x, y, rtol=1e-6, atol=1e-9)


def _stepper(seed=31):
    sc, cams = small_cluster_inputs(30000, 320, 208, seed=seed)
    tg = scenes.scene_clusters(seed + 100, 40000, 3)
    gt = ops.Gaussians.from_scene(tg, DEV)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    g = ops.Gaussians.from_scene(sc, DEV)
    st = PlainStep(g, cams, target, 0.1)
    noise = torch.as_tensor(scenes.fallback_noise(3, st.k), device=DEV)
    return st, noise


def test_graph_replay_matches_eager_step():
    eager, noise = _stepper()
    out_e = eager.step(noise)
    torch.cuda.synchronize()
    graphed, noise_g = _stepper()
    init = [t.clone() for t in graphed.g.tensors()]
    graphed.capture(noise_g)  # runs one step eagerly on a side stream, then captures
    torch.cuda.synchronize()
    for t, s in zip(graphed.g.tensors(), init):  # back to the initial state
        t.copy_(s)
    for t in graphed.m.tensors() + graphed.v.tensors():
        t.zero_()
    graphed.adam_t.fill_(1)
    out_g = graphed.replay()
    torch.cuda.synchronize()
    pe, pg = out_e[3], out_g[3]
    assert torch.equal(pe.status, pg.status) and torch.equal(pe.n_children, pg.n_children)
    n_new = int(pe.d_new_n.item())
    assert n_new == int(pg.d_new_n.item()) and n_new > eager.g.n
    assert torch.equal(eager.cand, graphed.cand)
    assert torch.equal(eager.img.dominant, graphed.img.dominant)
    # float atomics in the backward make the last bits order-dependent
    for a, b in zip(eager.g.tensors(), graphed.g.tensors()):
        torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6)
    for a, b in zip(out_e[0].tensors(), out_g[0].tensors()):
        sl = (slice(None), slice(0, n_new)) if a.dim() == 3 else (slice(0, n_new),)
        torch.testing.assert_close(a[sl], b[sl], rtol=1e-4, atol=1e-5)
    assert int(graphed.adam_t.item()) == 2


def test_autotuner_picks_a_legal_shape_and_batch_with_identical_results():
    """The tuner times the fused batched step under every tile shape and per-block
    Gaussian batch and keeps the fastest; the tuned step gives the same image,
    error statistics and gradient as the default one."""
    from paper_2605_06876_b300.autotune import BATCHES, SHAPES, tune
    from paper_2605_06876_b300.pipeline import BatchedStep

    sc, cams = small_cluster_inputs(20000, 320, 208, views=2, seed=41)
    g = ops.Gaussians.from_scene(sc, DEV)
    P = sum(c["width"] * c["height"] for c in cams)
    target = torch.rand((P, 3), device=DEV)
    params, times = tune(g, cams, target, reps=2)
    best = (params.tile_w, params.tile_h, params.batch)
    assert best[:2] in SHAPES and best[2] in BATCHES
    assert len(times) == len(SHAPES) * len(BATCHES) and times[best] == min(times.values())
    ref = BatchedStep(g, cams, target)
    ref.run()
    got = BatchedStep(g, cams, target, params=params)
    got.run()
    torch.cuda.synchronize()
    assert torch.equal(ref.img.rgb, got.img.rgb) and torch.equal(ref.img.dominant, got.img.dominant)
    assert torch.equal(ref.count, got.count) and torch.equal(ref.mass, got.mass)
    for a, b in zip(ref.grad.dense().tensors(), got.grad.dense().tensors()):
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()))


def test_fused_adam_compaction_equals_adam_then_apply():
    """Adam on the candidate rows, the plan, then the compaction that applies the
    step to every other row while copying gives, bit for bit, the population and
    moments of a full Adam step followed by the plain compaction (same gradient:
    the backward's float atomics would otherwise differ in the last bits)."""
    st, noise = _stepper(seed=37)
    st.step(noise)  # fills the regions, candidates and counts of a real step
    torch.cuda.synchronize()
    gen = torch.Generator(DEV).manual_seed(5)
    grad = st.g.zeros_like()
    for t in grad.tensors():
        t.normal_(0.0, 1e-2, generator=gen)
    m0, v0 = st.g.zeros_like(), st.g.zeros_like()
    for t in m0.tensors():
        t.normal_(0.0, 1e-3, generator=gen)
    for t in v0.tensors():
        t.uniform_(0.0, 1e-4, generator=gen)
    cap = st.out_capacity
    res = []
    for fused in (False, True):
        g, m, v = st.g.clone(), m0.clone(), v0.clone()
        d_step = torch.full((1,), 3, dtype=torch.int32, device=DEV)
        out = [ops.Gaussians(cap, g.sh_degree, DEV, zero=True) for _ in range(3)]
        if fused:
            ops.adam_step_rows(g, grad, m, v, st.cand, d_step, st.lr)
        else:
            ops.adam_step(g, grad, m, v, d_step, st.lr)
        plan = ops.split_plan(g, st.cams, st.regions, st.cand, st.count, st.params, sync=False)
        if fused:
            ops.split_apply_adam(g, grad, m, v, plan, st.regions, st.cand, noise, d_step, out[0],
                                 out[1], out[2], st.params, st.lr)
        else:
            ops.split_apply(g, plan, st.regions, st.cand, noise, st.params, m_in=m, v_in=v,
                            out=out[0], m_out=out[1], v_out=out[2])
        torch.cuda.synchronize()
        res.append((plan, out, int(d_step.item())))
    (pp, op, sp), (pf, of, sf) = res
    n_new = int(pp.d_new_n.item())
    assert n_new == int(pf.d_new_n.item()) and n_new > st.g.n
    assert torch.equal(pp.status, pf.status) and torch.equal(pp.n_children, pf.n_children)
    assert sp == sf == 4
    for a, b in zip(sum((x.tensors() for x in op), []), sum((x.tensors() for x in of), [])):
        if a.dim() == 3:  # SH planes [planes][capacity][4]
            assert torch.equal(a[:, :n_new], b[:, :n_new])
        else:
            assert torch.equal(a[:n_new], b[:n_new])
