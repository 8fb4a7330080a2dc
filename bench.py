"""Benchmark of the plain AdpSplit training step (one view, 1M Gaussians, SH degree 3,
1280x832): projection, binning, compositing with the dominant map, error
statistics, top-k candidates, error regions, render backward, Adam and the
AdpSplit operator with compaction of parameters and Adam moments.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent
replica on its own GPU (the step has no cross-GPU exchange); the job value is the
sum of steps over ranks divided by the slowest rank's time.

The reference arm (--impl reference) times the FP64 CPU oracle on this host's
cores on a bounded sample of the same workload (there is no released reference
implementation of the paper to run).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+error-stats iters/s, 1M Gaussians @1280x832"
UNIT = "iters/s"
WORKLOAD = dict(workload="single-view plain step: 1,000,000 Gaussians (64 clusters + 20% "
                "background), SH degree 3, one 1280x832 camera on a radius-4 ring; target "
                "rendered from a 1.5M-Gaussian scene; 10% candidates by error mass",
                n_gaussians=1_000_000, width=1280, height=832, sh_degree=3, views=1,
                cand_frac=0.10, l2="flushed between steps (256 MiB write)")


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "split_apply_traffic.json")


def _measured_traffic(stage, kernel=None):
    """DRAM bytes per launch of one kernel of a stage from the committed ncu capture,
    if the capture covers this stage and every source it was taken from is
    unchanged (sha1 of the files); otherwise None."""
    import hashlib

    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("stage") != stage:
        return None
    for rel, digest in rec.get("sources_sha1", {}).items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha1(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    per_kernel = rec.get("dram_bytes_per_launch")
    return per_kernel.get(kernel) if kernel and isinstance(per_kernel, dict) else None


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the default process group (x itself without
    one): the whole job takes as long as its slowest replica."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time
    (weak scaling: every rank processes the same units)."""
    return world * units_per_rank / max_seconds


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured", d
    return 6400.0, "fallback", {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, timestamped, every 20 ms; the
    summary keeps the samples inside the timed window [t0, t1]."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (kept after the run for inspection); set BENCH_CLOCKS_DIR
        # to keep them elsewhere than the system's temporary directory
        import tempfile

        folder = os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(folder, f"clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t0, t1):
        import datetime as dt

        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = dt.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]),
                             [nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 <= r[0] <= t1]
        note = "inside the timed region"
        if not inside and rows:  # a very short timed region: nearest samples
            rows.sort(key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))
            inside = rows[:3]
            note = "nearest samples to a timed region shorter than the sampling period"
        sm = [r[1] for r in inside]
        reasons = sorted({x for r in inside for x in r[3]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(r[2] for r in inside)) if inside else None,
                "reasons": reasons, "samples": len(inside), "window": note}


# --------------------------------------------------------------------------- algorithmic bytes

# FP32 operations (an FMA counts 2) of the compositing inner loops: evaluating
# alpha at one pixel for one Gaussian, blending it in the forward, and the
# contribution of one blended pair to the 2D gradients in the backward.
FLOP_EVAL = 16
FLOP_BLEND_FWD = 12
FLOP_BLEND_BWD = 56


def stage_bytes(n, n_vis, K, P, n_tiles, sh_planes, regions, k, kept, appended):
    """Algorithmic DRAM bytes of each stage for one step: each input read once and each
    output written once, from the per-unit figures below (bytes per Gaussian, visible
    record, tile instance, pixel, region and candidate)."""
    gbytes = 16 * (3 + sh_planes)  # one Gaussian's parameters (float4 planes)
    return {
        "project": n * gbytes + n * (3 * 16 + 16 + 4),
        "bin_sort": n * 8 + n_vis * 8 * 2 * 4 + K * (8 + 2 * 16) + n_tiles * 8,
        "render": n_tiles * 8 + K * 4 + n_vis * 48 + P * 28,
        "error_stats": P * (12 + 12 + 4 + 4 + 4 + 1) + n * 12,
        # the keys read once and the ids written: the radix select's extra passes over
        # the keys still in play are the kernel's own cost, not algorithmic bytes
        "select_topk": n * 8 + k * 4,
        "error_regions": P * (1 + 4 + 1 + 4 + 4 + 4 + 4) + regions * 160,
        # the gradient has a row mask: parameters read and gradients written for the
        # rendered Gaussians only, plus the mask byte and the tile counts of all
        "render_backward": (n_tiles * 8 + K * 4 + n_vis * 48 + P * (12 + 12 + 4 + 4) +
                            n_vis * 48 * 2 + n_vis * gbytes * 2 + n * (1 + 4)),
        # Adam: read parameter, m, v (and the gradient of rendered rows); write
        # parameter, m, v
        "adam": n * gbytes * 6 + n_vis * gbytes + n,
        "adam_rows": k * gbytes * 6 + min(k, n_vis) * gbytes + k * 5,
        # the plan's first part (candidate slots, kept-row destinations, statuses),
        # which the step runs on the side stream beside the backward
        "split_statuses": n * 12 + k * 16,
        # its second part (proposals and merges per region); in the step it runs on
        # the library's auxiliary stream beside the kept rows, and the main stream's
        # split_plan stage is only the fork
        "split_plan": regions * 300,
        # compaction with the fused Adam step (apply_keep_kernel): kept rows as in
        # Adam (gradients of rendered rows only), one destination word and one mask
        # byte per row
        "split_apply": kept * gbytes * 6 + min(kept, n_vis) * gbytes + n * (4 + 1),
        # appended rows (apply_append_kernel): the parents read, the new rows
        # written with zero moments
        "split_append": k * gbytes + appended * gbytes * 3,
    }


# --------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch

    import scenes
    from __graft_entry__ import build
    from paper_2605_06876_b300 import ops
    from paper_2605_06876_b300.pipeline import PlainStep, StageTimer

    build()
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    cfg = dict(scenes.CONFIGS[1])
    if args.gaussians:  # a smaller scene of the same recipe, for profiler captures
        cfg["n"], cfg["n_target"] = args.gaussians, args.gaussians * 3 // 2
    sc = scenes.scene_clusters(2, cfg["n"], cfg["sh_degree"])
    tg = scenes.scene_clusters(3, cfg["n_target"], cfg["sh_degree"])
    cams = scenes.ring_cameras(3, 1, cfg["ring_radius"], cfg["width"], cfg["height"])
    # target image: a render of the second scene (setup, outside any timing)
    gt = ops.Gaussians.from_scene(tg, dev)
    prt = ops.project(gt, cams)
    bt = ops.bin_sort(gt.n, prt, cams)
    target = ops.render(gt.n, prt, bt, cams).rgb.clone()
    del gt, prt, bt
    g = ops.Gaussians.from_scene(sc, dev)
    stepper = PlainStep(g, cams, target, cfg["cand_frac"])
    noise = torch.as_tensor(scenes.fallback_noise(5, stepper.k), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    sampler = ClockSampler(local_rank)
    sampler.start()
    for _ in range(args.warmup):
        stepper.step(noise)
    torch.cuda.synchronize()
    if not stepper.check_capacity():
        raise RuntimeError("instance or region capacity exceeded during warm-up")
    use_graph = not args.no_graph
    timer = StageTimer()
    if use_graph:
        # two captures of the same step: one with the stage events (replayed after
        # the timed region for the per-stage times) and the timed one, without them
        stepper.capture(noise, timer)
        staged_graph = stepper.graph
        stepper.capture(noise)
        for _ in range(args.warmup):
            staged_graph.replay()
            stepper.replay()
        torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    step_ms = []
    last_plan = None
    stage_ms = {}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.random_(0, 255)  # evict L2 between steps (not timed)
        ev0.record(stream)
        if use_graph:
            out = stepper.replay()
        else:
            timer = StageTimer()
            out = stepper.step(noise, timer)
        ev1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        if not use_graph:
            for kname, val in timer.durations().items():  # stages of this step
                stage_ms[kname] = stage_ms.get(kname, 0.0) + val
        last_plan = out[3]
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop(t_wall0, time.time())
    stage_steps = args.steps
    staged_ms = None
    if use_graph:  # the per-stage times, from the same number of instrumented replays
        staged = []
        for _ in range(args.steps):
            flush.random_(0, 255)
            ev0.record(stream)
            staged_graph.replay()  # re-records the captured stage events
            ev1.record(stream)
            torch.cuda.synchronize()
            staged.append(ev0.elapsed_time(ev1))
            for kname, val in timer.durations().items():
                stage_ms[kname] = stage_ms.get(kname, 0.0) + val
        staged_ms = sum(staged) / len(staged) if staged else None
    if not stepper.check_capacity(last_plan):
        raise RuntimeError("instance, region or population capacity exceeded in the timed region")
    new_n = int(last_plan.d_new_n.item())
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(args.steps, world, total_ms / 1e3)

    # end to end through the public API: every step's inputs (the Gaussian parameters,
    # the target, the fallback noise) come from pinned host memory and the split
    # decisions are read back and waited for. The inputs are double-buffered: step
    # k + 1's host-to-device copy runs on copy streams into a device staging buffer
    # while step k computes, and a device-to-device copy moves them into the step's
    # buffers before it starts
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
              (stepper.g.mean_logit.cpu().numpy(), stepper.g.logscale.cpu().numpy(),
               stepper.g.quat.cpu().numpy(), stepper.g.sh.cpu().numpy(),
               target.cpu().numpy(), noise.cpu().numpy())]
    dsts = stepper.g.tensors() + [target, noise]
    staging = [[torch.empty_like(d) for d in dsts] for _ in range(2)]
    st_h = torch.empty(stepper.k, dtype=torch.uint8).pin_memory()
    nc_h = torch.empty(stepper.k, dtype=torch.int32).pin_memory()
    e2e_steps = max(2, args.steps)  # the same K steps as the device-timed value
    h2d = sum(p.numel() * p.element_size() for p in pinned)
    d2h = stepper.k * (1 + 4)
    # the host link takes more in flight: each step's bytes go in pieces of about
    # 16 MB, spread over four copy streams (one stream carried 45 GB/s, four 50 GB/s)
    copy_streams = [torch.cuda.Stream(device=dev) for _ in range(4)]
    loaded = [[torch.cuda.Event() for _ in copy_streams] for _ in range(2)]  # buffer filled
    consumed = [torch.cuda.Event() for _ in range(2)]  # staging buffer copied out
    for ev in consumed:
        ev.record(stream)
    piece = 16 << 20

    def pieces(buf):
        for s_, src in zip(staging[buf], pinned):
            d8 = s_.view(-1).view(torch.uint8)
            h8 = src.view(-1).view(torch.uint8)
            for o in range(0, d8.numel(), piece):
                yield d8[o:o + piece], h8[o:o + piece]

    def h2d_into(buf):
        for cs in copy_streams:
            cs.wait_event(consumed[buf])
        for j, (dst, src) in enumerate(pieces(buf)):
            with torch.cuda.stream(copy_streams[j % len(copy_streams)]):
                dst.copy_(src, non_blocking=True)
        for cs, ev in zip(copy_streams, loaded[buf]):
            ev.record(cs)

    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d_into(0)
    for k_ in range(e2e_steps):
        buf = k_ % 2
        if k_ + 1 < e2e_steps:
            h2d_into(1 - buf)  # the next step's inputs, beside this step
        for ev in loaded[buf]:
            stream.wait_event(ev)
        for d_, s_ in zip(dsts, staging[buf]):
            d_.copy_(s_, non_blocking=True)
        consumed[buf].record(stream)
        out = stepper.replay() if use_graph else stepper.step(noise)
        st_h.copy_(out[3].status, non_blocking=True)
        nc_h.copy_(out[3].n_children, non_blocking=True)
        stream.synchronize()  # the host has the step's decisions
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dev)
    del staging

    # roofline of the dominant stage
    n = g.n
    n_vis = int((stepper.pr.tiles > 0).sum().item())
    K = int(stepper.bins.n_inst.item())
    R = int(stepper.regions.count.item())
    st_ = last_plan.status.long()
    appended = int(((st_ == 1) * (1 + last_plan.n_children.long()) + (st_ == 2) * 2).sum().item())
    sb = stage_bytes(n, n_vis, K, stepper.P, stepper.bins.ranges.shape[0], ops.sh_planes(3), R,
                     stepper.k, new_n - appended, appended)
    per_stage = {k: v / stage_steps for k, v in stage_ms.items()}
    # the roofline is reported for the step's top kernel in the ncu launch list,
    # apply_keep_kernel (the compaction of the kept rows with the fused Adam step,
    # HBM-bound), alone in its stage: the plan's proposals and merges run beside it
    # on the library's auxiliary stream, the appended rows follow in their own
    # stage. render_backward takes about as long, but it shares the SMs with the
    # concurrent error-statistics stream, so its stage time is not its own
    dom = "split_apply"
    peak, peak_kind, peaks = _peaks()
    ach = sb[dom] / (per_stage[dom] * 1e-3) / 1e9
    roof = {"kernel": "apply_keep_kernel", "stage": dom, "bound": "hbm",
            "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4),
            "traffic": _measured_traffic(dom, "apply_keep_kernel<1>"),
            "algorithmic_bytes": int(sb[dom]), "peak_source": peak_kind}
    # the compositing stages are bound by the FP32 pipes: exact per-pixel work of the
    # last step (list positions evaluated up to the last blended Gaussian, blended
    # pairs) over the stage time
    n_eval = int(stepper.img.last.sum().item())
    n_blend = int(stepper.img.n_contrib.sum().item())
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    alu_peak = sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12  # TFLOP/s, FP32 FMA = 2
    flops = {"render": n_eval * FLOP_EVAL + n_blend * FLOP_BLEND_FWD,
             "render_backward": n_eval * FLOP_EVAL + n_blend * FLOP_BLEND_BWD}
    roof_alu = {k: {"achieved": round(f / (per_stage[k] * 1e-3) / 1e12, 2), "peak": round(alu_peak, 1),
                    "unit": "TFLOP/s", "frac": round(f / (per_stage[k] * 1e-3) / 1e12 / alu_peak, 4),
                    "flops": int(f)} for k, f in flops.items() if k in per_stage}
    roof_alu["peak_source"] = f"{sm_count} SMs x 128 FP32 lanes x 2 x {clock_mhz:.0f} MHz"
    step_bytes = sum(v for k, v in sb.items() if k in per_stage)
    launches = None if args.no_launch_count else count_launches(stepper, noise) * args.steps
    dssim = dssim_kernels(stepper.img.rgb, target, cams, flush, dev)
    eq2 = None
    if not args.no_eq2:
        eq2 = eq2_step(g, cams, target, dev, flush, max(3, min(args.steps, 10)))
    batched = batched_c3 = None
    if args.batch_views > 1:
        cfg1 = scenes.CONFIGS[1]
        del stepper.out, stepper.m_out, stepper.v_out
        torch.cuda.empty_cache()
        reps = max(3, min(args.steps, 10))
        batched = batched_vs_plain(g, tg, dev, args.batch_views, reps, flush, cfg1["width"],
                                   cfg1["height"], cfg1["ring_radius"],
                                   autotune=not args.no_autotune, peak=peak, alu_peak=alu_peak)
        if not args.no_c3:
            cfg3 = scenes.CONFIGS[3]
            g3 = ops.Gaussians.from_scene(scenes.scene_clusters(6, cfg3["n"], 3), dev)
            tg3 = scenes.scene_clusters(7, cfg3["n"] * 3 // 2, 3)
            res3 = scenes.uneven_resolutions(7, cfg3["views"])
            batched_c3 = batched_vs_plain(g3, tg3, dev, cfg3["views"], reps, flush, None, None,
                                          cfg3["hemisphere_radius"], seed=7, resolutions=res3,
                                          autotune=not args.no_autotune, peak=peak,
                                          alu_peak=alu_peak)
            del g3, tg3
            torch.cuda.empty_cache()
    c2 = densify = None
    if not args.no_workloads:
        reps = max(3, min(args.steps, 10))
        c2 = backward_c2(dev, flush, reps, alu_peak)
        cfg4 = scenes.CONFIGS[4]
        densify = {
            "c4_5m_8views": densify_step(dev, flush, reps, cfg4["n"], cfg4["views"], 19,
                                         cfg4["cand_frac"], 8, "5M Gaussians, 8 views, 20%"),
            "indoor_1m_20views": densify_step(dev, flush, reps, cfg["n"], 20, 19, 0.1, 2,
                                              "1M Gaussians, V = 20, N_max = 19"),
            "outdoor_1m_10views": densify_step(dev, flush, reps, cfg["n"], 10, 9, 0.1, 2,
                                               "1M Gaussians, V = 10, N_max = 9"),
        }
    loop = None
    if not args.no_train:
        loop = densify_loop(dev)
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded cluster scene; random-init Gaussians, no dataset)",
        "config": dict(WORKLOAD, parallelism=f"replicas{world}" if world > 1 else "single",
                       **({"n_gaussians": g.n, "note": "reduced scene for profiling"}
                          if args.gaussians else {})),
        "e2e": {"value": round(job_rate(1, world, e2e_ms / 1e3), 3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "roofline": roof,
        "roofline_alu": roof_alu,
        # the stages this step ran (the unfused "adam" entry of stage_bytes only
        # applies to a step without the fused compaction)
        "step_hbm": {"algorithmic_bytes": int(step_bytes),
                     "frac": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4),
                     "stages": sorted(k for k in sb if k in per_stage)},
        "graph": use_graph,
        "stages_ms": {k: round(v, 4) for k, v in per_stage.items()},
        # the step time of the instrumented graph the stage times come from (its
        # stage events are graph nodes between the kernels)
        "staged_ms_per_step": round(staged_ms, 4) if staged_ms else None,
        "batched_vs_plain": batched,
        "batched_c3": batched_c3,
        "backward_c2": c2,
        "densify_steps": densify,
        "dssim": dssim,
        "eq2_step": eq2,
        "densify_loop": loop,
        "stage_gbs": {k: round(sb[k] / (per_stage[k] * 1e-3) / 1e9, 1) for k in per_stage
                      if k in sb and per_stage[k] > 0.005},
        "workload_counts": {"visible": n_vis, "instances": K, "regions": R,
                            "pixel_evaluations": n_eval, "blended_pairs": n_blend,
                            "candidates": stepper.k, "new_population": new_n},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    return result


def dssim_kernels(img, target, cams, flush, dev, reps=10):
    """The D-SSIM loss-term kernels (forward maps, then the image gradient) on the
    step's render, timed by CUDA events with L2 flushed before each call, against the
    HBM roofline: per pixel 24 B read and 36 B written by the forward, 36 + 24 B read
    and 12 B written by the backward."""
    import torch

    from paper_2605_06876_b300 import ops

    dL = torch.empty_like(img)
    loss = torch.zeros((len(cams), 2), dtype=torch.float64, device=dev)
    need = ops.A.lib().adp_dssim_workspace_size(len(cams), ops.A.cameras(cams))
    ws = ops.workspace(need, dev)
    ops.dssim_loss_grad(img, target, cams, 0.2, dL=dL, loss=loss, ws=ws)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ops.dssim_loss_grad(img, target, cams, 0.2, dL=dL, loss=loss, ws=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    P = img.shape[0]
    nbytes = P * (24 + 36 + 36 + 24 + 12)
    peak, kind, _ = _peaks()
    return {"ms": round(ms, 4), "algorithmic_bytes": int(nbytes),
            "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
            "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4), "peak_source": kind,
            "ssim": round(float(loss[0, 1]), 6), "l1": round(float(loss[0, 0]), 6)}


def densify_loop(dev):
    """The small-scale analogue of the paper's training-time comparison: a coarse
    model (5% of a 200,000-Gaussian cluster scene's points) fitted to 48 ring views
    at 480x320 for 6,000 iterations, densified every 100 iterations until 3,000 with
    Eq. 2 candidates split by AdpSplit (errors of 10 sampled views) or by the
    vanilla split; PSNR on 4 held-out views."""
    import scenes
    from paper_2605_06876_b300 import ops, train

    gt_sc = scenes.scene_clusters(70, 200_000, 3)
    gt = ops.Gaussians.from_scene(gt_sc, dev)
    init = ops.Gaussians.from_scene(scenes.scene_initial_points(gt_sc, 0.05, 71), dev)
    tr = scenes.ring_cameras(72, 48, 14.0, 480, 320)
    te = scenes.ring_cameras(73, 4, 14.0, 480, 320)
    res = train.compare(gt, init, tr, te, iters=6000, densify_until=3000)
    res["config"] = ("200k-Gaussian cluster scene, 5% initial points, 48 training and 4 test "
                     "ring views at 480x320, 6000 iterations, densification every 100 until 3000")
    return res


def eq2_step(g, cams, target, dev, flush, steps):
    """The same step with the paper's own candidate choice (Eq. 2 on the image-space
    statistic of this step, clones appended after the split), as a CUDA graph, L2
    flushed before each replay. Returns its time and what it selected."""
    import torch

    import scenes
    from paper_2605_06876_b300.pipeline import DensifyStep

    st = DensifyStep(g, cams, target)
    noise = torch.as_tensor(scenes.fallback_noise(6, g.n), device=dev)
    saved = [t.clone() for t in st.g.tensors()]
    st.capture(noise)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        st.replay()
    ts = []
    for _ in range(steps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = st.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    if not st.check_capacity(out[3]):
        raise RuntimeError("capacity exceeded in the Eq. 2 step")
    ns, ncl = (int(x) for x in st.sets.counts.cpu())
    res = {"ms_per_step": round(float(np.mean(ts)), 4), "tau_g": st.tau_g, "tau_s": st.tau_s,
           "split_candidates": ns, "clones": ncl, "new_population": int(st.d_new_n.item()),
           "note": "statistic of this step only; candidates split by AdpSplit, clones appended"}
    for d, s_ in zip(st.g.tensors(), saved):  # the replays stepped Adam on the shared scene
        d.copy_(s_)
    del st
    torch.cuda.empty_cache()
    return res


# Algorithmic DRAM bytes of one forward + backward + error-statistics pass over
# V views, per unit: per Gaussian the parameters read for the forward (240 B), its
# projected record written (48) and read back by the backward (48), the parameters
# read by the backward (240) and the gradient written (236); per visible (view,
# Gaussian) record 52 B; per tile instance the pair written (12), one read and
# write by the sort (24) and the id and record read by the forward and the
# backward (2 x 52); per pixel the target (12), the image written (12) and read
# back (12), T, the count and the dominant id (12) and the error statistics (4).
BYTES_PER_GAUSSIAN = 240 + 48 + 48 + 240 + 236
BYTES_PER_RECORD = 52
BYTES_PER_INSTANCE = 12 + 24 + 2 * 52
BYTES_PER_PIXEL = 12 + 12 + 12 + 12 + 4


def fwd_bwd_stats_bytes(n, records, instances, pixels):
    return (n * BYTES_PER_GAUSSIAN + records * BYTES_PER_RECORD +
            instances * BYTES_PER_INSTANCE + pixels * BYTES_PER_PIXEL)


def _graph_ms(graph, steps, flush):
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(3):
        graph.replay()
    ts = []
    for _ in range(steps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))


def batched_vs_plain(g, tg, dev, n_views, steps, flush, width, height, radius, seed=11,
                     resolutions=None, autotune=True, peak=None, alu_peak=None):
    """fwd + bwd + error statistics for n_views views three ways, each a CUDA graph
    with L2 flushed before every repetition: the fused batched step
    (adp_train_step_batched: one persistent per-tile forward + error + backward
    kernel over all views), one launch per stage over all views, and n_views
    one-view launch sequences (the plain path). With autotune the tile shape and
    Gaussian batch of all three come from the autotuner."""
    import torch

    import scenes
    from paper_2605_06876_b300 import ops
    from paper_2605_06876_b300.pipeline import BatchedStep, ViewStages, capture_graph

    if resolutions is None:
        cams = scenes.ring_cameras(seed, n_views, radius, width, height)
    else:
        cams = scenes.hemisphere_cameras(seed, n_views, radius, resolutions)
    gt = ops.Gaussians.from_scene(tg, dev)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    del gt, prt
    torch.cuda.empty_cache()
    params, tune_ms = None, None
    if autotune:
        from paper_2605_06876_b300.autotune import tune

        params, tune_ms = tune(g, cams, target, reps=3)
        torch.cuda.empty_cache()
    res = {}
    fused = BatchedStep(g, cams, target, params=params)
    res["fused"] = _graph_ms(fused.capture(), steps, flush)
    if not fused.fits():
        raise RuntimeError("instance capacity exceeded in the fused batched step")
    n_vis = int((fused.pr.tiles > 0).sum().item())
    K = int(fused.bins.n_inst.item())
    P = fused.P
    n_eval = int(fused.img.last.sum().item())
    n_blend = int(fused.img.n_contrib.sum().item())
    tw, th, batch = fused.params.tile_w, fused.params.tile_h, fused.params.batch
    del fused
    torch.cuda.empty_cache()
    stages = ViewStages(g, cams, target, params=params)
    res["stages"] = _graph_ms(capture_graph(stages.run), steps, flush)
    ok = stages.fits()
    del stages
    torch.cuda.empty_cache()
    offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    grad = ops.Gaussians(g.n, g.sh_degree, dev, zero=False, row_mask=True)
    plain = [ViewStages(g, [c], target[offs[v]:offs[v + 1]], params=params, grad=grad)
             for v, c in enumerate(cams)]
    res["plain"] = _graph_ms(capture_graph(lambda: [p.run() for p in plain]), steps, flush)
    ok = ok and all(p.fits() for p in plain)
    del plain
    torch.cuda.empty_cache()
    if not ok:
        raise RuntimeError("instance capacity exceeded in the batched/plain comparison")
    nbytes = fwd_bwd_stats_bytes(g.n, n_vis, K, P)
    flops = n_eval * 2 * FLOP_EVAL + n_blend * (FLOP_BLEND_FWD + FLOP_BLEND_BWD)
    fused_s = res["fused"] * 1e-3
    out = {"views": n_views, "gaussians": g.n,
           "resolution": (f"{width}x{height}" if resolutions is None
                          else "uneven 640x416..1600x1056"),
           "batched_ms": round(res["fused"], 4), "stages_ms": round(res["stages"], 4),
           "plain_ms": round(res["plain"], 4),
           "speedup": round(res["plain"] / res["fused"], 3),
           "speedup_stages": round(res["plain"] / res["stages"], 3),
           "views_per_s_batched": round(n_views / fused_s, 1),
           "views_per_s_plain": round(1e3 * n_views / res["plain"], 1),
           "tile": [tw, th], "batch": batch,
           "counts": {"visible_records": n_vis, "instances": K, "pixels": P,
                      "pixel_evaluations": n_eval, "blended_pairs": n_blend},
           "hbm": {"algorithmic_bytes": int(nbytes),
                   "achieved_gbs": round(nbytes / fused_s / 1e9, 1),
                   "frac": round(nbytes / fused_s / 1e9 / peak, 4) if peak else None},
           "fp32": {"flops": int(flops), "achieved_tflops": round(flops / fused_s / 1e12, 2),
                    "frac": round(flops / fused_s / 1e12 / alu_peak, 4) if alu_peak else None},
           "autotune_ms": None if tune_ms is None else {f"{k[0]}x{k[1]}/{k[2]}": round(v, 4)
                                                        for k, v in tune_ms.items()}}
    return out


def backward_c2(dev, flush, steps, alu_peak):
    """The hand backward at 2,000,000 Gaussians, one 1280x832 view: adp_render_backward
    (per-pixel walk and per-Gaussian chain rule) of the L1 loss, as a CUDA graph."""
    import torch

    import scenes
    from paper_2605_06876_b300 import ops
    from paper_2605_06876_b300.pipeline import capture_graph

    cfg = scenes.CONFIGS[2]
    cams = scenes.ring_cameras(5, 1, cfg["ring_radius"], cfg["width"], cfg["height"])
    g = ops.Gaussians.from_scene(scenes.scene_clusters(4, cfg["n"], 3), dev)
    gt = ops.Gaussians.from_scene(scenes.scene_clusters(5, cfg["n"] * 3 // 2, 3), dev)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    del gt, prt
    pr = ops.project(g, cams)
    bins = ops.bin_sort(g.n, pr, cams)
    img = ops.render(g.n, pr, bins, cams)
    grad = ops.Gaussians(g.n, 3, dev, zero=False, row_mask=True)
    ws = ops.workspace(__import__("paper_2605_06876_b300._abi", fromlist=["lib"]).lib()
                       .adp_render_backward_workspace_size(g.n, 1), dev)
    graph = capture_graph(lambda: ops.render_backward(g, pr, bins, img, cams, target=target,
                                                      grad=grad, ws=ws))
    ms = _graph_ms(graph, steps, flush)
    n_eval = int(img.last.sum().item())
    n_blend = int(img.n_contrib.sum().item())
    flops = n_eval * FLOP_EVAL + n_blend * FLOP_BLEND_BWD
    out = {"gaussians": g.n, "resolution": f"{cfg['width']}x{cfg['height']}", "ms": round(ms, 4),
           "visible": int((pr.tiles > 0).sum().item()), "pixel_evaluations": n_eval,
           "blended_pairs": n_blend,
           "fp32": {"achieved_tflops": round(flops / (ms * 1e-3) / 1e12, 2),
                    "frac": round(flops / (ms * 1e-3) / 1e12 / alu_peak, 4)}}
    del g, pr, bins, img, grad, ws, graph
    torch.cuda.empty_cache()
    return out


def densify_step(dev, flush, steps, n, views, n_max, cand_frac, scene_seed, label):
    """One densification step over `views` sampled views (the fused batched call,
    top-k candidates, regions, AdpSplit and the compaction with the Adam step), as a
    CUDA graph; returns its time, the population it grows to, and the time of one
    training step (fused batched fwd + bwd + error statistics and Adam) on that
    grown population."""
    import torch

    import scenes
    from paper_2605_06876_b300 import _abi as A
    from paper_2605_06876_b300 import ops
    from paper_2605_06876_b300.pipeline import BatchedStep, PlainStep, capture_graph

    cams = scenes.ring_cameras(scene_seed + 1, views, 4.0, 1280, 832)
    gt = ops.Gaussians.from_scene(scenes.scene_clusters(scene_seed + 1, n * 3 // 2, 3), dev)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    del gt, prt
    torch.cuda.empty_cache()
    g = ops.Gaussians.from_scene(scenes.scene_clusters(scene_seed, n, 3), dev)
    prm = A.default_params(n_max=n_max)
    st = PlainStep(g, cams, target, cand_frac, params=prm, fused_views=True)
    noise = torch.as_tensor(scenes.fallback_noise(scene_seed, st.k), device=dev)
    st.capture(noise)
    ms = _graph_ms(st.graph, steps, flush)
    out_g, _, _, plan = st.graph_out
    if not st.check_capacity(plan):
        raise RuntimeError(f"capacity exceeded in the {label} densification step")
    new_n = int(plan.d_new_n.item())
    status = plan.status.long()
    res = {"workload": label, "gaussians": n, "views": views, "n_max": n_max,
           "candidates": st.k, "step_ms": round(ms, 4), "new_population": new_n,
           "adaptive": int((status == A.ADP_ADAPTIVE).sum().item()),
           "fallback": int((status == A.ADP_FALLBACK).sum().item()),
           "reset": int((status == A.ADP_RESET).sum().item())}
    grown = ops.Gaussians(new_n, 3, dev, zero=False)
    for d, s_ in zip(grown.tensors(), out_g.tensors()):
        d.copy_(s_[:, :new_n] if s_.dim() == 3 else s_[:new_n])
    del st, out_g, plan
    torch.cuda.empty_cache()
    bs = BatchedStep(grown, cams, target, params=prm)
    m, v = grown.zeros_like(), grown.zeros_like()
    t = torch.ones(1, dtype=torch.int32, device=dev)

    def train():
        bs.run()
        ops.adam_step(grown, bs.grad, m, v, t)

    res["grown_train_step_ms"] = round(_graph_ms(capture_graph(train), steps, flush), 4)
    if not bs.fits():
        raise RuntimeError(f"capacity exceeded in the {label} grown training step")
    del bs, grown, m, v
    torch.cuda.empty_cache()
    return res


def run_batched_only(args, local_rank):
    """Only the fused batched step (fwd + bwd + error statistics over --batch-views
    ring views of the single-view workload's scene, or --gaussians of it), as a
    CUDA graph: --warmup replays, then --steps timed ones with L2 flushed before
    each. For profiler captures of the batched kernels."""
    import torch

    import scenes
    from __graft_entry__ import build
    from paper_2605_06876_b300 import _abi as A
    from paper_2605_06876_b300 import ops
    from paper_2605_06876_b300.pipeline import BatchedStep

    build()
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    cfg = dict(scenes.CONFIGS[1])
    n = args.gaussians or cfg["n"]
    V = max(1, args.batch_views)
    cams = scenes.ring_cameras(11, V, cfg["ring_radius"], cfg["width"], cfg["height"])
    gt = ops.Gaussians.from_scene(scenes.scene_clusters(3, n * 3 // 2, 3), dev)
    prt = ops.project(gt, cams)
    target = ops.render(gt.n, prt, ops.bin_sort(gt.n, prt, cams), cams).rgb.clone()
    del gt, prt
    g = ops.Gaussians.from_scene(scenes.scene_clusters(2, n, 3), dev)
    st = BatchedStep(g, cams, target, params=A.default_params(batch=args.batch))
    graph = st.capture()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        graph.replay()
    ms = _graph_ms(graph, args.steps, flush) if args.steps > 0 else None
    if not st.fits():
        raise RuntimeError("instance capacity exceeded")
    return {"metric": "batched fwd+bwd+error-stats views/s", "views": V, "gaussians": n,
            "batch": st.params.batch, "ms": ms,
            "value": None if ms is None else round(1e3 * V / ms, 1), "unit": "views/s"}


def count_launches(stepper, noise):
    """Kernels of this library launched by one step (CUPTI trace of one extra step,
    outside the timed region)."""
    import torch
    from torch.profiler import ProfilerActivity, profile

    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        stepper.step(noise)
        torch.cuda.synchronize()
    names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    return sum(1 for nm in names if "adp::" in nm or "_ZN3adp" in nm)


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(budget_s=20.0):
    """Times the FP64 oracle, as it stands, on a bounded sample of the step and
    scales it to one full step. Returns (seconds per full step, description, cores)."""
    import oracle as O
    import scenes

    O.build()
    cfg = scenes.CONFIGS[1]
    sc = scenes.scene_clusters(2, cfg["n"], cfg["sh_degree"])
    cam = scenes.ring_cameras(3, 1, cfg["ring_radius"], cfg["width"], cfg["height"])[0]
    W, H = cam["width"], cam["height"]
    th = O.theta_of(sc)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    pr = O.project(th, 3, cam)
    t_proj = time.perf_counter() - t0
    # compositing: a band of rows through a cropped camera (same pixels, same Gaussians)
    rows = 16
    band = dict(cam, height=rows, py=np.float32(float(cam["py"]) - (H // 2)))
    t0 = time.perf_counter()
    prb = O.project(th, 3, band)
    rb = O.render(prb, band)
    t_band = time.perf_counter() - t0 - t_proj  # project cost counted once
    t_render = max(t_band, 1e-6) * (H / rows)
    # error statistics and regions at full size on generator inputs
    img, tgt, dom = scenes.error_stage_inputs(4, W, H, cfg["n"])
    t0 = time.perf_counter()
    em = O.error_map(img, tgt, 0.1, 3)
    cnt, mass = O.gauss_stats(em["M"], dom.reshape(-1), em["E"], cfg["n"])
    k = int(cfg["cand_frac"] * cfg["n"])
    cand = O.topk_mass(mass, k)
    flag = np.zeros(cfg["n"], np.uint8)
    flag[cand] = 1
    Me = O.erode(em["M"], W, H, 2)
    rg = O.regions(0, W, H, Me, em["B"], dom.reshape(-1), cfg["n"], flag, tgt, 5)
    sp = O.split(th, 3, [cam], rg, cand, cnt, np.zeros((k, 2, 3)))
    t_err = time.perf_counter() - t0
    # gradient: 8 visible Gaussians of median footprint, scaled by footprint area
    # (its cost grows with the pixels of the Gaussian's box) to all visible ones
    vis = np.nonzero(pr["tiles"] > 0)[0]
    b = pr["box"][vis]
    area = (b[:, 1] - b[:, 0] + 1).astype(np.float64) * (b[:, 3] - b[:, 2] + 1)
    order = vis[np.argsort(area)]
    mid = len(order) // 2
    sel = np.ascontiguousarray(order[max(0, mid - 4):mid + 4], np.int32)
    sel_area = area[np.searchsorted(vis, sel)].sum()
    t0 = time.perf_counter()
    O.grad(th, 3, cam, tgt, sel)
    t_grad = (time.perf_counter() - t0) * area.sum() / max(sel_area, 1.0)
    t0 = time.perf_counter()
    z = np.zeros_like(th)
    O.adam(th.copy(), z, z.copy(), z.copy(), 1)
    t_adam = time.perf_counter() - t0
    total = t_proj + t_render + t_err + t_grad + t_adam
    desc = (f"oracle FP64 on {cores} threads: projection of all 1M Gaussians ({t_proj:.2f}s), "
            f"compositing of a {rows}-row band scaled x{H / rows:.0f} ({t_band:.2f}s), full-size "
            f"error map/top-k/regions/split on generator maps ({t_err:.2f}s), gradient of "
            f"{len(sel)} median-footprint Gaussians scaled by box area to {len(vis)} visible "
            f"({t_grad:.1f}s est.), Adam "
            f"({t_adam:.2f}s)")
    return total, desc, cores


def run_reference(args, rank, world):
    if rank != 0:
        return None
    per_step, desc, cores = None, None, None
    times = []
    for _ in range(args.warmup and 1):
        oracle_sample()
    for _ in range(args.steps):
        per_step, desc, cores = oracle_sample()
        times.append(per_step)
    value = 1.0 / float(np.mean(times))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism="cpu"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shape and batch in the batched comparisons")
    ap.add_argument("--only-batched", action="store_true",
                    help="time only the fused batched step (--batch-views views; profiler use)")
    ap.add_argument("--batch", type=int, default=64,
                    help="Gaussians staged per compositing batch in --only-batched")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 2M backward and the densification-step workloads")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the 3M-Gaussian, 16 uneven views batched comparison")
    ap.add_argument("--batch-views", type=int, default=16,
                    help="views of the batched-vs-plain comparison (0 or 1: skip)")
    ap.add_argument("--no-train", action="store_true",
                    help="skip the densification-loop comparison (vanilla split vs AdpSplit)")
    ap.add_argument("--no-eq2", action="store_true",
                    help="skip the timing of the step with the Eq. 2 candidate choice")
    ap.add_argument("--no-launch-count", action="store_true",
                    help="skip the CUPTI kernel count (for runs under ncu)")
    ap.add_argument("--gaussians", type=int, default=0,
                    help="scene size override for small profiler captures (default: 1M)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if args.only_batched:
        print(json.dumps(run_batched_only(args, local_rank)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            per_step, desc, cores = oracle_sample()
            res["cpu_baseline"] = {"value": 1.0 / per_step, "unit": UNIT, "cores": cores,
                                   "kind": "oracle", "sample": desc}
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
