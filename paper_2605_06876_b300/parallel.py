"""View-sharded data parallelism of the densification step (the V views sampled
per step, Sec. 4.1, split across ranks).

Every rank holds a replica of the Gaussians and processes its share of the views:
the forward, the L1 error statistics, the backward and the error regions of those
views. Two exchanges make every rank's result that of one process doing all views:

- the per-Gaussian sums over views -- the gradient, the error-pixel counts and the
  error masses -- are summed over ranks (all-reduce; the gradient's rows that a
  rank did not render are zeroed first, and its row mask becomes the union). The
  masses are sums of float32 E values above the threshold, which are exact in
  float64, so their sum over ranks does not depend on the order; the gradient
  agrees to float rounding;
- the error regions of each rank's views are gathered by every rank (the tables
  have different lengths) and put in the global (view, label) order before the
  per-parent merge of Eqs. 11-12, which then sees every view's proposals.

The exchange functions below take torch tensors on any device, so they run over
NCCL on GPUs and over gloo on CPU tensors alike. ViewShardedStep drives the GPU
path (one process per GPU, launched by torchrun).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

REGION_INT_FIELDS = ("view", "parent", "label", "band")


def shard_views(n_views, rank, world):
    """The global indices of the views rank processes (round robin)."""
    return list(range(rank, n_views, world))


def allreduce_sums(tensors, group=None):
    """Sums every tensor over the ranks, in place (float gradients, int32 counts,
    float64 masses)."""
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def allreduce_masked_gradient(planes, rows, group=None):
    """Sums a row-masked gradient over the ranks, in place.

    planes: the gradient's float planes ([n, 4] tensors, or [P, n, 4] for the SH
    planes); rows: uint8 [n], 1 where this rank wrote the row. Rows with rows == 0
    hold no defined values (the backward never writes them), so they are zeroed
    before the sum; the mask becomes the union over ranks."""
    unset = rows == 0
    for t in planes:
        if t.dim() == 3:
            t.masked_fill_(unset[None, :, None], 0.0)
        else:
            t.masked_fill_(unset[:, None], 0.0)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(rows, op=dist.ReduceOp.MAX, group=group)
    return planes, rows


def _gather_rows(t, group=None):
    """All-gather of a [R, ...] tensor whose R differs between ranks."""
    world = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)
    pad = torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def allgather_regions(regions, local_views, group=None):
    """Gathers the region tables of every rank in the global (view, label) order.

    regions: dict with view (int32 [R], the LOCAL view index within the rank's
    share), parent, label, band (int32 [R]), moments (int64 [R, 6]) and stats
    (float64 [R, 12]), as torch tensors or numpy arrays, ordered by (local view,
    label); local_views: the global index of each local view. Returns the same
    fields for all ranks' regions with global view indices, as torch tensors on
    the device of the inputs."""
    dev = regions["stats"].device if torch.is_tensor(regions["stats"]) else torch.device("cpu")
    t = {k: torch.as_tensor(np.asarray(v) if not torch.is_tensor(v) else v).to(dev)
         for k, v in regions.items() if k in REGION_INT_FIELDS + ("moments", "stats")}
    gmap = torch.as_tensor(np.asarray(local_views, np.int64), device=dev)
    ints = torch.stack([gmap[t["view"].long()]] + [t[k].long() for k in REGION_INT_FIELDS[1:]], 1)
    ints = torch.cat([ints, t["moments"].long()], 1)  # [R, 4 + 6] int64
    all_ints = _gather_rows(ints, group)
    all_stats = _gather_rows(t["stats"].double(), group)
    # the global order: by view, then label (each label is unique within its view)
    key = all_ints[:, 0] * (1 << 32) + all_ints[:, 2]
    order = torch.argsort(key, stable=True)
    all_ints, all_stats = all_ints[order], all_stats[order]
    out = {k: all_ints[:, i].to(torch.int32) for i, k in enumerate(REGION_INT_FIELDS)}
    out["moments"] = all_ints[:, 4:].contiguous()
    out["stats"] = all_stats.contiguous()
    return out


class ViewShardedStep:
    """One densification step over n_views views sharded across the ranks of the
    default process group (one GPU each): the fused batched step on the rank's
    views, the all-reduce of gradient, counts and masses, the top-k candidates
    (identical on every rank), the regions of the rank's views, their all-gather,
    and the split plan and compaction on the gathered regions, so every rank ends
    with the same new population."""

    def __init__(self, g, cams, targets, cand_frac=0.1, params=None, group=None):
        from . import _abi as A
        from . import ops
        from .pipeline import BatchedStep

        self.ops, self.group = ops, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.views = shard_views(len(cams), self.rank, self.world)
        self.cams = [cams[v] for v in self.views]
        self.all_cams = list(cams)
        self.params = params or A.default_params()
        self.g = g
        target = torch.cat([targets[v] for v in self.views])
        self.local = BatchedStep(g, self.cams, target, params=self.params)
        self.target = target
        self.k = max(1, int(round(cand_frac * g.n)))
        self.cand = torch.empty(self.k, dtype=torch.int32, device=g.mean_logit.device)

    def step(self, noise):
        ops = self.ops
        st = self.local
        st.run()
        allreduce_masked_gradient(st.grad.tensors(), st.grad.rows, self.group)
        allreduce_sums([st.count, st.mass], self.group)
        ops.select_topk(st.mass, self.g.n, self.k, self.cand, status=st.status)
        regs = ops.error_regions(st.maps, st.img.dominant, self.target, self.g.n, self.cams,
                                 self.cand, self.params, status=st.status)
        local = regs.to_numpy()
        gathered = allgather_regions({k: torch.as_tensor(v, device=st.count.device)
                                      for k, v in local.items() if k != "labels"},
                                     self.views, self.group)
        regions = ops.Regions.from_arrays(gathered["view"].cpu().numpy(),
                                          gathered["parent"].cpu().numpy(),
                                          gathered["label"].cpu().numpy(),
                                          gathered["stats"].cpu().numpy(),
                                          gathered["band"].cpu().numpy(),
                                          gathered["moments"].cpu().numpy(),
                                          device=st.count.device)
        plan = ops.split_plan(self.g, self.all_cams, regions, self.cand, st.count, self.params,
                              status_word=st.status)
        out = ops.split_apply(self.g, plan, regions, self.cand, noise, self.params,
                              with_state=False)
        return out, plan
