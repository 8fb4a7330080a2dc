"""Failure detection of the bounded device waits, without faulting or hanging
the GPU: a tiny poll bound (adp_set_spin_limit) makes the top-k's grid barrier
and the prefix sums' look-back give up. The kernels then return normally, the
caller's status word holds ADP_ERR_TIMEOUT, and the context stays usable: calls
at the default bound afterwards give exact results."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import DEV, np_, small_cluster_inputs
from paper_2605_06876_b300 import _abi as A
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.pipeline import PlainStep

pytestmark = pytest.mark.gpu

TIMEOUT = 4  # ADP_ERR_TIMEOUT


class tiny_spin_limit:
    def __enter__(self):
        A.lib().adp_set_spin_limit(1)

    def __exit__(self, *exc):
        A.lib().adp_set_spin_limit(0)  # back to the default bound
        return False


def test_topk_barrier_timeout_is_reported():
    """Every block of the cooperative top-k counts itself in at a grid barrier and
    then waits for the others; with a bound of one poll the first blocks to arrive
    give up (their flag is never set in time)."""
    n, k = 1_000_000, 100_000
    rng = np.random.default_rng(1)
    mass = np.floor(rng.exponential(2.0, n) * 16) / 16
    m = torch.as_tensor(mass, device=DEV)
    status = ops.status_word(DEV)
    with tiny_spin_limit():
        out = ops.select_topk(m, n, k, status=status)
        torch.cuda.synchronize()
    assert int(status.item()) == TIMEOUT
    ids = np_(out)
    assert np.all((ids == -1) | ((ids >= 0) & (ids < n)))
    assert len(set(ids[ids >= 0].tolist())) == int((ids >= 0).sum())  # distinct ids
    with pytest.raises(RuntimeError, match="ADP_ERR_TIMEOUT"):
        ops.check_status(status)
    # the context is usable and the default bound gives the exact selection
    ok = ops.status_word(DEV)
    out = ops.select_topk(m, n, k, status=ok)
    torch.cuda.synchronize()
    assert int(ok.item()) == 0
    want = np.sort(np.lexsort((np.arange(n), -mass))[:k]).astype(np.int32)
    assert np.array_equal(np_(out), want)


def test_scan_lookback_timeout_is_reported_and_nothing_is_binned_past_capacity():
    """The binning's two prefix sums (visible records, instance offsets) over many
    scan tiles: with a bound of one poll a look-back finds a predecessor that has
    not published yet and gives up. The instance lists stay inside the capacity and
    a later call at the default bound reproduces the reference binning."""
    sc, cams = small_cluster_inputs(300_000, 640, 416, views=2, seed=21)
    g = ops.Gaussians.from_scene(sc, DEV)
    pr = ops.project(g, cams)
    ref = ops.bin_sort(g.n, pr, cams)
    torch.cuda.synchronize()
    cap = ref.capacity
    bins = ops.Bins.alloc(cap, ops.n_tiles(cams), DEV)
    seen = False
    for _ in range(4):  # a timeout is all but certain on the first call
        status = ops.status_word(DEV)
        with tiny_spin_limit():
            ops.bin_sort(g.n, pr, cams, bins=bins, grow=False, status=status)
            torch.cuda.synchronize()
        r = np_(bins.ranges)
        assert r.min() >= 0 and r.max() <= cap
        if int(status.item()) == TIMEOUT:
            seen = True
            break
        assert int(status.item()) == 0
    assert seen, "no look-back gave up at a bound of one poll"
    status = ops.status_word(DEV)
    ops.bin_sort(g.n, pr, cams, bins=bins, grow=False, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert int(bins.n_inst.item()) == int(ref.n_inst.item())
    assert torch.equal(bins.ranges, ref.ranges)
    assert torch.equal(bins.inst[:int(ref.n_inst.item())], ref.inst[:int(ref.n_inst.item())])


def test_plain_step_reports_a_timeout_and_recovers():
    """A whole step (binning, top-k, regions, split plan and compaction) with every
    wait bounded to one poll: it runs to the end, check_status raises with the
    timeout, and the next step at the default bound matches a step of an
    untouched stepper."""
    sc, cams = small_cluster_inputs(60_000, 320, 208, seed=22)
    tg = ops.Gaussians.from_scene(scenes.scene_clusters(23, 90_000, 3), DEV)
    prt = ops.project(tg, cams)
    target = ops.render(tg.n, prt, ops.bin_sort(tg.n, prt, cams), cams).rgb.clone()
    noise = torch.as_tensor(scenes.fallback_noise(5, 6000), device=DEV)
    a = PlainStep(ops.Gaussians.from_scene(sc, DEV), cams, target, 0.1)
    b = PlainStep(ops.Gaussians.from_scene(sc, DEV), cams, target, 0.1)
    with tiny_spin_limit():
        a.step(noise)
        torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="ADP_ERR_TIMEOUT"):
        a.check_status()
    # restore a's inputs (its Adam step ran on undefined gradients) and step both
    for d, s in zip(a.g.tensors(), b.g.tensors()):
        d.copy_(s)
    for t in a.m.tensors() + a.v.tensors():
        t.zero_()
    a.adam_t.fill_(1)
    a.status.zero_()
    out_a = a.step(noise)
    out_b = b.step(noise)
    torch.cuda.synchronize()
    a.check_status()
    b.check_status()
    # the forward and the error statistics are deterministic; the gradients are
    # summed by float atomics, so the updated population agrees to rounding
    assert torch.equal(a.img.rgb, b.img.rgb) and torch.equal(a.img.dominant, b.img.dominant)
    assert torch.equal(a.count, b.count) and torch.equal(a.mass, b.mass)
    assert torch.equal(a.cand, b.cand)
    assert torch.equal(out_a[3].status, out_b[3].status)
    n_new = int(out_b[3].d_new_n.item())
    assert int(out_a[3].d_new_n.item()) == n_new
    for x, y in zip(out_a[0].tensors(), out_b[0].tensors()):
        xs = x[:, :n_new] if x.dim() == 3 else x[:n_new]
        ys = y[:, :n_new] if y.dim() == 3 else y[:n_new]
        torch.testing.assert_close(xs, ys, rtol=1e-4, atol=1e-5)
