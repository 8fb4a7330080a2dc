"""The view-sharded exchange of paper_2605_06876_b300.parallel on CPU, with
world-size-2 gloo process groups.

Each rank processes its share of four views. The per-view computation that the
GPU does in the product (projection, compositing, error map, per-Gaussian error
statistics, erosion, regions) is done here by the oracle; the exchange between
ranks is the product's own code: the all-reduce of the per-Gaussian counts and
masses, and the all-gather of the variable-length region tables into the global
(view, label) order. The split of the gathered regions must then equal the
oracle's single-process step over all four views, on both ranks: the same
candidates, the same region table, the same statuses, child counts and new
population. The gradient sum over ranks is checked on per-view partial sums.
"""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_VIEWS, K = 4, 150


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    import oracle as O
    import scenes

    sc = scenes.scene_box(0, 1500, 0)
    tg = scenes.scene_box(1, 3000, 0)
    cams = [scenes.camera_look_at(p, (0.0, 0.0, 4.0), 96, 72)
            for p in ((0, 0, 0), (0.6, 0, 0.2), (-0.5, -0.3, 0.1), (0.2, 0.5, -0.2))]
    targets = [O.render(O.project(O.theta_of(tg), 0, c), c)["rgb"].astype(np.float32)
               .reshape(c["height"], c["width"], 3) for c in cams]
    noise = scenes.fallback_noise(3, K).astype(np.float64)
    return sc, cams, targets, noise


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2605_06876_b300.parallel import allgather_regions, allreduce_sums, shard_views

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cams, targets, noise = _inputs()
        theta = O.theta_of(sc)
        n = theta.shape[0]
        sp = O.SplitParams()
        views = shard_views(N_VIEWS, rank, world)
        count, mass = np.zeros(n, np.int32), np.zeros(n, np.float64)
        grad = np.zeros(n)
        local = []
        for v in views:  # the rank's views (the GPU's part in the product)
            cam = cams[v]
            rd = O.render(O.project(theta, 0, cam), cam)
            em = O.error_map(rd["rgb"].astype(np.float32).reshape(cam["height"], cam["width"], 3),
                             targets[v], sp.tau_l1, sp.n_levels)
            O.gauss_stats(em["M"], rd["dominant"], em["E"], n, count, mass)
            grad += v + 1.0  # a per-view partial sum whose total is known: 1 + 2 + 3 + 4
            local.append((v, cam, rd, em))
        t_count, t_mass, t_grad = (torch.as_tensor(a) for a in (count, mass, grad))
        allreduce_sums([t_count, t_mass, t_grad])
        cand = O.topk_mass(t_mass.numpy(), K)
        flag = np.zeros(n, np.uint8)
        flag[cand] = 1
        parts = []
        for lv, (v, cam, rd, em) in enumerate(local):
            W, H = cam["width"], cam["height"]
            Me = O.erode(em["M"], W, H, sp.r_erode)
            parts.append(O.regions(lv, W, H, Me, em["B"], rd["dominant"], n, flag, targets[v],
                                   sp.m_min))
        regs = O.concat_regions(parts)
        gathered = allgather_regions(regs, views)
        g = {k: t.numpy() for k, t in gathered.items()}
        res = O.split(theta, 0, cams, g, cand, t_count.numpy(), noise, sp)
        out.put((rank, t_count.numpy(), t_mass.numpy(), t_grad.numpy(), cand, g, res))
    finally:
        dist.destroy_process_group()


def test_view_sharded_exchange_equals_one_process():
    import oracle as O

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r[0], r[1:]) for r in (out.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, cams, targets, noise = _inputs()
    ref = O.plain_step(sc, cams, targets, k_cand=K, noise=noise)
    n = O.theta_of(sc).shape[0]
    for rank in (0, 1):
        count, mass, grad, cand, regs, res = got[rank]
        assert np.array_equal(count, ref["count"]) and np.array_equal(mass, ref["mass"])
        np.testing.assert_array_equal(grad, np.full(n, 10.0))
        assert np.array_equal(cand, ref["cand"])
        assert len(regs["view"]) == len(ref["regions"]["view"]) > 0
        assert set(regs["view"].tolist()) == set(range(N_VIEWS))
        for key in ("view", "parent", "label", "band", "moments", "stats"):
            assert np.array_equal(regs[key], ref["regions"][key]), key
        sp = ref["split"]
        assert np.array_equal(res["status"], sp["status"])
        assert np.array_equal(res["n_children"], sp["n_children"])
        assert res["new_n"] == sp["new_n"]
        assert np.array_equal(res["theta"], sp["theta"])
    assert (ref["split"]["status"] == O.ADAPTIVE).sum() > 0


def _masked_rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2605_06876_b300.parallel import allreduce_masked_gradient

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 40
        rng = np.random.default_rng(7)  # the same draws on both ranks
        dense = [rng.standard_normal((2, n, 4)).astype(np.float32) for _ in range(2)]  # [rank]
        sh = [rng.standard_normal((2, 3, n, 4)).astype(np.float32) for _ in range(2)]
        marks = rng.random((2, n)) < 0.4
        rows = torch.as_tensor(marks[rank].astype(np.uint8))
        planes = [torch.as_tensor(dense[0][rank].copy()), torch.as_tensor(dense[1][rank].copy()),
                  torch.as_tensor(sh[0][rank].copy())]
        # rows this rank did not write hold no defined values
        for t in planes:
            if t.dim() == 3:
                t[:, ~torch.as_tensor(marks[rank])] = float("nan")
            else:
                t[~torch.as_tensor(marks[rank])] = float("nan")
        allreduce_masked_gradient(planes, rows)
        out.put((rank, [t.numpy() for t in planes], rows.numpy(), dense, sh, marks))
    finally:
        dist.destroy_process_group()


def test_masked_gradient_allreduce_ignores_unwritten_rows():
    """Each rank's row-masked gradient leaves the rows it did not render undefined
    (NaN here); the exchange must give on every rank the sum of the ranks' written
    rows (zero where no rank wrote) and the union of the masks."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_masked_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, planes, rows, dense, sh, marks in got:
        m = marks.astype(np.float32)
        want = [sum(dense[0][r] * m[r][:, None] for r in range(2)),
                sum(dense[1][r] * m[r][:, None] for r in range(2)),
                sum(sh[0][r] * m[r][None, :, None] for r in range(2))]
        for a, b in zip(planes, want):
            assert np.isfinite(a).all()
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-6)
        np.testing.assert_array_equal(rows, (marks[0] | marks[1]).astype(np.uint8))
