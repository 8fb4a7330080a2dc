"""The view-sharded densification step (paper_2605_06876_b300.parallel) on the GPU.

Every run has one GPU, so the sharded step runs here as a single NCCL rank: the
exchanges are then identities, and the step must give exactly what the direct
calls give (the batched call over all views, the top-k, the regions, the split),
which checks the wiring of the GPU path (buffers, devices, dtypes, the region
table's round trip through the all-gather). The exchanges themselves are checked
over two gloo ranks in test_parallel.py.
"""
import socket

import pytest
import torch
import torch.distributed as dist

import scenes
from gpu_util import DEV, small_cluster_inputs
from paper_2605_06876_b300 import ops
from paper_2605_06876_b300.parallel import ViewShardedStep

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_view_sharded_step_one_rank_equals_the_direct_calls():
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0,
                            world_size=1)
    try:
        sc, _ = small_cluster_inputs(20000, 8, 8, seed=50)
        cams = [scenes.camera_look_at((0.0, -0.3, -4.0), (0, 0, 0), 160, 112),
                scenes.camera_look_at((2.5, 0.2, -3.0), (0, 0, 0), 97, 131),
                scenes.camera_look_at((-2.0, -1.0, -3.2), (0, 0, 0), 144, 96)]
        tg = ops.Gaussians.from_scene(scenes.scene_clusters(51, 30000, 3), DEV)
        prt = ops.project(tg, cams)
        full = ops.render(tg.n, prt, ops.bin_sort(tg.n, prt, cams), cams).rgb.clone()
        targets, off = [], 0
        for c in cams:
            P = c["width"] * c["height"]
            targets.append(full[off:off + P].contiguous())
            off += P
        g = ops.Gaussians.from_scene(sc, DEV)
        vs = ViewShardedStep(g, cams, targets, cand_frac=0.1)
        noise = torch.as_tensor(scenes.fallback_noise(52, vs.k), device=DEV)
        (out, _, _), plan = vs.step(noise)
        torch.cuda.synchronize()
        ops.check_status(vs.local.status)

        _, _, img, maps, count, mass, grad = ops.train_step_batched(g, cams, full)
        cand = ops.select_topk(mass, g.n, vs.k)
        regs = ops.error_regions(maps, img.dominant, full, g.n, cams, cand)
        plan2 = ops.split_plan(g, cams, regs, cand, count)
        out2, _, _ = ops.split_apply(g, plan2, regs, cand, noise, with_state=False)
        torch.cuda.synchronize()

        assert torch.equal(vs.local.count, count) and torch.equal(vs.local.mass, mass)
        assert torch.equal(vs.local.grad.rows, grad.rows)
        assert torch.equal(vs.cand, cand)
        assert int(regs.count.item()) > 0
        assert torch.equal(plan.status, plan2.status)
        assert torch.equal(plan.n_children, plan2.n_children)
        assert out.n == out2.n
        for a, b in zip(out.tensors(), out2.tensors()):
            assert torch.equal(a, b)
    finally:
        dist.destroy_process_group()
