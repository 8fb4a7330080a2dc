"""One plain AdpSplit training step over preallocated device buffers.

A step runs the whole hot path: projection, binning and depth sort, compositing with
the dominant map, error statistics, top-k candidate choice by error mass, error
regions, the render backward of the L1 loss, one Adam step, and the AdpSplit operator
(plan and apply into buffers sized for the largest possible result, so no step
synchronises with the host). The error chain runs on a second stream beside the
backward, and the split's proposals and merges on the library's auxiliary stream
beside the compaction; every fork is joined within the step, so a step captures into
one CUDA graph. The new population (the first plan.d_new_n entries of the returned
buffers) is returned; the step's own population is updated only by Adam, so repeated
steps see the same workload.
"""
from __future__ import annotations

import torch

from . import _abi as A
from . import ops


class StageTimer:
    """CUDA timing events between stages, each recorded on the stream its stage
    runs on (the current stream at mark time). Inside a CUDA-graph capture they
    are recorded with cudaEventRecordExternal, so they become event-record nodes
    and every replay re-records them: the stage durations of the latest replay (or
    eager step) come from durations(), each from a mark to the next mark on the
    same stream (the last mark of a stream only ends the previous stage)."""

    def __init__(self):
        from cuda.bindings import runtime as rt

        self.rt = rt
        self.events = []

    def mark(self, name):
        rt = self.rt
        err, ev = rt.cudaEventCreateWithFlags(rt.cudaEventDefault)
        if err != rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaEventCreateWithFlags: {err}")
        st = torch.cuda.current_stream()
        # an external record (a node of the graph) inside a capture, a plain one outside
        err, cap = rt.cudaStreamIsCapturing(st.cuda_stream)
        if err != rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaStreamIsCapturing: {err}")
        active = cap == rt.cudaStreamCaptureStatus.cudaStreamCaptureStatusActive
        flags = rt.cudaEventRecordExternal if active else rt.cudaEventRecordDefault
        (err,) = rt.cudaEventRecordWithFlags(ev, st.cuda_stream, flags)
        if err != rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaEventRecordWithFlags: {err}")
        self.events.append((name, ev, st.cuda_stream))

    def durations(self):
        out = {}
        by_stream = {}
        for name, ev, sid in self.events:
            by_stream.setdefault(sid, []).append((name, ev))
        for evs in by_stream.values():
            for (name, a), (_, b) in zip(evs[:-1], evs[1:]):
                err, ms = self.rt.cudaEventElapsedTime(a, b)
                if err != self.rt.cudaError_t.cudaSuccess:
                    raise RuntimeError(f"cudaEventElapsedTime: {err}")
                out[name] = out.get(name, 0.0) + ms
        return out

    def __del__(self):
        try:
            for _, ev, _ in self.events:
                self.rt.cudaEventDestroy(ev)
        except Exception:
            pass


class PlainStep:
    def __init__(self, g: ops.Gaussians, cams, target, cand_frac=0.1, params=None,
                 bg=(0.0, 0.0, 0.0), lr=ops.ADAM_LR, bins_margin=1.15, region_margin=1.25,
                 fused_adam=True, out_capacity=None, dssim_lambda=0.0, overlap_split=True,
                 fused_views=False):
        self.g = g
        # fused_views: projection, binning, compositing, error statistics and the L1
        # backward of all views as one adp_train_step_batched call (its persistent
        # per-tile forward + error + backward kernel) instead of five calls with the
        # error statistics on the side stream; the top-k and regions then follow
        self.fused_views = bool(fused_views)
        if self.fused_views and dssim_lambda > 0:
            raise ValueError("the fused views step differentiates the L1 loss only")
        # fused_adam: the Adam step of the candidates runs before the plan and the
        # compaction applies it to every other row while copying (one pass over
        # parameters and moments instead of two; same result bit for bit)
        self.fused_adam = fused_adam
        # overlap_split (with fused_adam): the plan's proposals and merges run on the
        # library's auxiliary stream while the compaction streams the kept rows
        # (adp_split_plan_overlapped / adp_split_apply_adam_overlapped; same result)
        self.overlap_split = overlap_split
        # dssim_lambda > 0: the baselines' loss (1 - lambda) L1 + lambda (1 - SSIM),
        # its image gradient fed to the backward; 0 keeps the pure L1 loss
        self.dssim_lambda = float(dssim_lambda)
        self.cams = list(cams)
        self.V = len(self.cams)
        self.target = target
        self.params = params or A.default_params()
        self.bg = bg
        self.lr = lr
        self.dev = g.mean_logit.device
        n = g.n
        self.k = max(1, int(round(cand_frac * n)))
        self.P = ops.n_pixels(self.cams)
        self.m, self.v = g.zeros_like(), g.zeros_like()
        # the gradient carries a row mask: rows of Gaussians no view renders are
        # neither written by the backward nor read by Adam
        self.grad = ops.Gaussians(n, g.sh_degree, self.dev, zero=False, row_mask=True)
        self.pr = ops.Projected.alloc(self.V * n, self.dev)
        self.img = ops.Image.alloc(self.P, self.dev)
        self.maps = ops.ErrorMaps.alloc(self.P, self.V, self.dev)
        self.count = torch.empty(n, dtype=torch.int32, device=self.dev)
        self.mass = torch.empty(n, dtype=torch.float64, device=self.dev)
        self.cand = torch.empty(self.k, dtype=torch.int32, device=self.dev)
        self.adam_t = torch.ones(1, dtype=torch.int32, device=self.dev)  # Adam step, on device
        # device status word of the calls with bounded waits (scans, top-k barrier):
        # nonzero once one gave up; read at a sync point by check_status()
        self.status = ops.status_word(self.dev)
        self.graph = None
        # the error-statistics chain (error map, top-k, regions) runs on a second
        # stream, concurrently with the render backward: both need only the
        # forward image. The chain is a string of small latency-bound kernels, so
        # its stream has the higher priority: its blocks are scheduled ahead of
        # the backward's waiting ones instead of queueing behind them
        self.side = torch.cuda.Stream(device=self.dev, priority=-1)
        # size the instance and region buffers from one probing pass
        ops.project(g, self.cams, self.params, self.pr)
        probe = ops.bin_sort(n, self.pr, self.cams, self.params)
        k_inst = int(probe.n_inst.item())
        self.bins = ops.Bins.alloc(int(k_inst * bins_margin) + 1024,
                                   ops.n_tiles(self.cams, self.params.tile_w, self.params.tile_h),
                                   self.dev)
        self.ws_bins = ops.workspace(ops.bin_sort_workspace_size(n, self.V, self.bins.capacity), self.dev)
        ops.bin_sort(n, self.pr, self.cams, self.params, bins=self.bins, ws=self.ws_bins, grow=False)
        ops.render(n, self.pr, self.bins, self.cams, bg, self.params, self.img)
        ops.error_stats(self.img.rgb, target, self.img.dominant, n, self.cams, self.params,
                        self.maps, self.count, self.mass)
        ops.select_topk(self.mass, n, self.k, self.cand)
        probe_r = ops.error_regions(self.maps, self.img.dominant, target, n, self.cams, self.cand,
                                    self.params)
        cap = int(int(probe_r.count.item()) * region_margin) + 1024
        self.regions = ops.Regions.alloc(cap, None, self.dev)
        ca = A.cameras(self.cams)
        self.ws_regions = ops.workspace(A.lib().adp_error_regions_workspace_size(n, self.V, ca), self.dev)
        self.ws_topk = ops.workspace(A.lib().adp_select_topk_workspace_size(n), self.dev)
        self.ws_bwd = ops.workspace(A.lib().adp_render_backward_workspace_size(n, self.V), self.dev)
        if self.fused_views:
            import ctypes

            self.ws_views = ops.workspace(A.lib().adp_train_step_batched_workspace_size(
                n, self.V, ca, ctypes.byref(self.params), self.bins.capacity), self.dev)
        if self.dssim_lambda > 0:
            self.dL = torch.empty((self.P, 3), dtype=torch.float32, device=self.dev)
            self.loss = torch.zeros((self.V, 2), dtype=torch.float64, device=self.dev)
            self.ws_dssim = ops.workspace(A.lib().adp_dssim_workspace_size(self.V, ca), self.dev)
        self.ws_split = ops.workspace(ops.split_workspace_size(n, self.k, cap), self.dev)
        # the largest population a split can produce: no read-back inside a step
        self.out_capacity = (out_capacity if out_capacity is not None
                             else n + self.k * (self.params.n_max + 1))
        self.out = ops.Gaussians(self.out_capacity, g.sh_degree, self.dev, zero=False)
        self.m_out = ops.Gaussians(self.out_capacity, g.sh_degree, self.dev, zero=False)
        self.v_out = ops.Gaussians(self.out_capacity, g.sh_degree, self.dev, zero=False)
        torch.cuda.synchronize()

    def step(self, noise, timer: StageTimer = None):
        """One step; returns (new Gaussians, new m, new v, split plan)."""
        g, cams, prm, n = self.g, self.cams, self.params, self.g.n
        mark = timer.mark if timer else (lambda name: None)
        if self.fused_views:
            return self._step_fused_views(noise, mark)
        mark("project")
        ops.project(g, cams, prm, self.pr)
        mark("bin_sort")
        ops.bin_sort(n, self.pr, cams, prm, bins=self.bins, ws=self.ws_bins, grow=False,
                     status=self.status)
        mark("render")
        ops.render(n, self.pr, self.bins, cams, self.bg, prm, self.img)
        main = torch.cuda.current_stream()
        overlap = self.fused_adam and self.overlap_split
        self.side.wait_stream(main)  # fork after the forward
        with torch.cuda.stream(self.side):
            mark("error_stats")
            ops.error_stats(self.img.rgb, self.target, self.img.dominant, n, cams, prm, self.maps,
                            self.count, self.mass)
            mark("select_topk")
            ops.select_topk(self.mass, n, self.k, self.cand, ws=self.ws_topk, status=self.status)
            cand_ready = torch.cuda.Event()
            cand_ready.record(self.side)
            mark("error_regions")
            ops.error_regions(self.maps, self.img.dominant, self.target, n, cams, self.cand, prm,
                              regions=self.regions, ws=self.ws_regions, grow=False,
                              status=self.status)
            if overlap:
                # the plan's first part (statuses, kept rows, the bound) reads no
                # parameter, so it runs here, beside the backward
                mark("split_statuses")
                plan = ops.split_plan_overlapped(g, cams, self.regions, self.cand, self.count,
                                                 prm, ws=self.ws_split, status_word=self.status,
                                                 part="statuses")
            mark("error_end")
        if self.dssim_lambda > 0:
            mark("dssim")
            ops.dssim_loss_grad(self.img.rgb, self.target, cams, self.dssim_lambda, prm,
                                dL=self.dL, loss=self.loss, ws=self.ws_dssim)
        mark("render_backward")
        if self.dssim_lambda > 0:
            ops.render_backward(g, self.pr, self.bins, self.img, cams, dL_drgb=self.dL,
                                bg=self.bg, params=prm, grad=self.grad, ws=self.ws_bwd)
        else:
            ops.render_backward(g, self.pr, self.bins, self.img, cams, target=self.target,
                                bg=self.bg, params=prm, grad=self.grad, ws=self.ws_bwd)
        if self.fused_adam:
            # the candidates' Adam step needs only the gradient and the candidates, so
            # it runs beside the regions (the longer branch) instead of after them
            main.wait_event(cand_ready)
            mark("adam_rows")
            ops.adam_step_rows(g, self.grad, self.m, self.v, self.cand, self.adam_t, self.lr)
        mark("join")
        main.wait_stream(self.side)  # join before the split
        if not self.fused_adam:
            mark("adam")
            ops.adam_step(g, self.grad, self.m, self.v, self.adam_t, self.lr)
        mark("split_plan")
        if overlap:  # the proposals and merges, forked onto the library's auxiliary stream
            plan = ops.split_plan_overlapped(g, cams, self.regions, self.cand, self.count, prm,
                                             ws=self.ws_split, status_word=self.status,
                                             part="proposals", plan=plan)
        else:
            plan = ops.split_plan(g, cams, self.regions, self.cand, self.count, prm,
                                  ws=self.ws_split, sync=False, status_word=self.status)
        mark("split_apply")
        if overlap:  # the kept rows (the dominant kernel), then the join and the appended rows
            args = (g, self.grad, self.m, self.v, plan, self.regions, self.cand, noise, self.adam_t,
                    self.out, self.m_out, self.v_out, prm, self.lr)
            ops.split_apply_adam(*args, overlapped=True, part="keep")
            mark("split_append")
            ops.split_apply_adam(*args, overlapped=True, part="append")
        elif self.fused_adam:
            ops.split_apply_adam(g, self.grad, self.m, self.v, plan, self.regions, self.cand, noise,
                                 self.adam_t, self.out, self.m_out, self.v_out, prm, self.lr)
        else:
            ops.split_apply(g, plan, self.regions, self.cand, noise, prm, m_in=self.m, v_in=self.v,
                            out=self.out, m_out=self.m_out, v_out=self.v_out)
        mark("end")
        return self.out, self.m_out, self.v_out, plan

    def _step_fused_views(self, noise, mark):
        """The step with the view-dependent stages in one adp_train_step_batched call."""
        g, cams, prm, n = self.g, self.cams, self.params, self.g.n
        mark("views")
        ops.train_step_batched(g, cams, self.target, prm, self.bg, pr=self.pr, bins=self.bins,
                               img=self.img, maps=self.maps, count=self.count, mass=self.mass,
                               grad=self.grad, ws=self.ws_views, status=self.status)
        mark("select_topk")
        ops.select_topk(self.mass, n, self.k, self.cand, ws=self.ws_topk, status=self.status)
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):  # the regions beside the candidates' Adam step
            mark("error_regions")
            ops.error_regions(self.maps, self.img.dominant, self.target, n, cams, self.cand, prm,
                              regions=self.regions, ws=self.ws_regions, grow=False,
                              status=self.status)
            mark("error_end")
        mark("adam_rows")
        ops.adam_step_rows(g, self.grad, self.m, self.v, self.cand, self.adam_t, self.lr)
        mark("join")
        main.wait_stream(self.side)
        mark("split_plan")
        plan = ops.split_plan_overlapped(g, cams, self.regions, self.cand, self.count, prm,
                                         ws=self.ws_split, status_word=self.status)
        mark("split_apply")
        args = (g, self.grad, self.m, self.v, plan, self.regions, self.cand, noise, self.adam_t,
                self.out, self.m_out, self.v_out, prm, self.lr)
        ops.split_apply_adam(*args, overlapped=True, part="keep")
        mark("split_append")
        ops.split_apply_adam(*args, overlapped=True, part="append")
        mark("end")
        return self.out, self.m_out, self.v_out, plan

    def capture(self, noise, timer: StageTimer = None):
        """Captures one step in a CUDA graph (no step synchronises with the host, and
        every buffer is preallocated, so the whole step replays as one launch). A
        timer's stage events are captured with it and re-recorded by each replay."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(noise)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.graph_out = self.step(noise, timer)
        return self.graph_out

    def replay(self):
        """One step from the captured graph; returns what the captured step returned."""
        self.graph.replay()
        return self.graph_out

    def check_status(self):
        """Raises if a bounded device wait of any step so far gave up (reads the
        status word: a synchronisation)."""
        ops.check_status(self.status, type(self).__name__)

    def check_capacity(self, plan=None):
        """True if the last step's instances, regions (and population) fit their buffers."""
        self.check_status()
        ok = (int(self.bins.n_inst.item()) <= self.bins.capacity and
              int(self.regions.count.item()) <= self.regions.capacity)
        if plan is not None:
            ok = ok and int(plan.d_new_n.item()) <= self.out_capacity
        return ok


class ViewStages:
    """The view-dependent stages of a step -- projection, binning, compositing,
    error statistics and the render backward -- for a set of views, each launched
    once over all of them. Used to compare one batched launch over V views with V
    one-view launches (pass a shared `grad` to the one-view instances)."""

    def __init__(self, g: ops.Gaussians, cams, target, params=None, bg=(0.0, 0.0, 0.0),
                 grad: ops.Gaussians = None, bins_margin=1.15):
        self.g, self.cams, self.target = g, list(cams), target
        self.params = params or A.default_params()
        self.bg = bg
        self.dev = g.mean_logit.device
        n, V = g.n, len(self.cams)
        self.P = ops.n_pixels(self.cams)
        self.pr = ops.Projected.alloc(V * n, self.dev)
        self.img = ops.Image.alloc(self.P, self.dev)
        self.maps = ops.ErrorMaps.alloc(self.P, V, self.dev)
        self.count = torch.empty(n, dtype=torch.int32, device=self.dev)
        self.mass = torch.empty(n, dtype=torch.float64, device=self.dev)
        self.grad = grad if grad is not None else ops.Gaussians(n, g.sh_degree, self.dev,
                                                                zero=False, row_mask=True)
        ops.project(g, self.cams, self.params, self.pr)
        probe = ops.bin_sort(n, self.pr, self.cams, self.params)
        cap = int(int(probe.n_inst.item()) * bins_margin) + 1024
        self.bins = ops.Bins.alloc(cap, ops.n_tiles(self.cams, self.params.tile_w,
                                                     self.params.tile_h), self.dev)
        self.ws_bins = ops.workspace(ops.bin_sort_workspace_size(n, V, cap), self.dev)
        self.ws_bwd = ops.workspace(A.lib().adp_render_backward_workspace_size(n, V), self.dev)
        self.side = torch.cuda.Stream(device=self.dev, priority=-1)
        torch.cuda.synchronize()

    def run(self):
        g, cams, prm, n = self.g, self.cams, self.params, self.g.n
        ops.project(g, cams, prm, self.pr)
        ops.bin_sort(n, self.pr, cams, prm, bins=self.bins, ws=self.ws_bins, grow=False)
        ops.render(n, self.pr, self.bins, cams, self.bg, prm, self.img)
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)  # error statistics beside the backward, as in PlainStep
        with torch.cuda.stream(self.side):
            ops.error_stats(self.img.rgb, self.target, self.img.dominant, n, cams, prm, self.maps,
                            self.count, self.mass)
        ops.render_backward(g, self.pr, self.bins, self.img, cams, target=self.target, bg=self.bg,
                            params=prm, grad=self.grad, ws=self.ws_bwd)
        main.wait_stream(self.side)

    def fits(self):
        return int(self.bins.n_inst.item()) <= self.bins.capacity


class BatchedStep:
    """The view-dependent part of a training step for many views in one call,
    adp_train_step_batched: projection and binning of all views, one persistent
    fused forward + L1-error + backward kernel over the (view, tile) work queue,
    the error statistics and the per-Gaussian gradient summed over views. All
    buffers are preallocated (the instance capacity from one probing pass), so
    run() never synchronises and capture() records it as one CUDA graph."""

    def __init__(self, g: ops.Gaussians, cams, target, params=None, bg=(0.0, 0.0, 0.0),
                 bins_margin=1.15, grad2d=False):
        self.g, self.cams, self.target = g, list(cams), target
        self.params = params or A.default_params()
        self.bg = bg
        self.dev = g.mean_logit.device
        n, V = g.n, len(self.cams)
        self.P = ops.n_pixels(self.cams)
        self.pr = ops.Projected.alloc(V * n, self.dev)
        ops.project(g, self.cams, self.params, self.pr)
        probe = ops.bin_sort(n, self.pr, self.cams, self.params)
        cap = int(int(probe.n_inst.item()) * bins_margin) + 1024
        del probe
        self.bins = ops.Bins.alloc(cap, ops.n_tiles(self.cams, self.params.tile_w,
                                                     self.params.tile_h), self.dev)
        self.img = ops.Image.alloc(self.P, self.dev)
        self.maps = ops.ErrorMaps.alloc(self.P, V, self.dev)
        self.count = torch.empty(max(n, 1), dtype=torch.int32, device=self.dev)
        self.mass = torch.empty(max(n, 1), dtype=torch.float64, device=self.dev)
        self.grad = ops.Gaussians(n, g.sh_degree, self.dev, zero=False, row_mask=True)
        self.accum = torch.zeros(n, dtype=torch.float32, device=self.dev) if grad2d else None
        self.visits = torch.zeros(n, dtype=torch.int32, device=self.dev) if grad2d else None
        import ctypes

        self.ws = ops.workspace(A.lib().adp_train_step_batched_workspace_size(
            n, V, A.cameras(self.cams), ctypes.byref(self.params), cap), self.dev)
        self.status = ops.status_word(self.dev)
        self.graph = None
        torch.cuda.synchronize()

    def run(self):
        ops.train_step_batched(self.g, self.cams, self.target, self.params, self.bg, pr=self.pr,
                               bins=self.bins, img=self.img, maps=self.maps, count=self.count,
                               mass=self.mass, grad=self.grad, grad2d_accum=self.accum,
                               grad2d_visits=self.visits, ws=self.ws, status=self.status)

    def capture(self):
        self.graph = capture_graph(self.run)
        return self.graph

    def replay(self):
        self.graph.replay()

    def fits(self):
        ops.check_status(self.status, "BatchedStep")
        return int(self.bins.n_inst.item()) <= self.bins.capacity


def capture_graph(fn):
    """A CUDA graph of fn() (run once eagerly on a side stream first)."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fn()
    return graph


class DensifyStep(PlainStep):
    """One step with the paper's own candidate choice instead of the top-k
    workload rule: the backward accumulates the image-space statistic of Sec. 3,
    Eq. 2 picks the split candidates (g_i >= tau_g, max s_i > tau_s) and the clone
    candidates (g_i >= tau_g, max s_i <= tau_s), AdpSplit splits the former and the
    latter are cloned after the compaction. The candidate lists are passed whole
    (n entries, -1 past the device-held counts), so nothing reads a count back.
    The statistic covers this step only (the accumulators are cleared first); the
    output population is sized from one probing step."""

    def __init__(self, g: ops.Gaussians, cams, target, tau_g=2e-4, tau_s=0.05, params=None,
                 bg=(0.0, 0.0, 0.0), lr=ops.ADAM_LR, out_margin=1.25):
        self.tau_g, self.tau_s = float(tau_g), float(tau_s)
        super().__init__(g, cams, target, cand_frac=1.0, params=params, bg=bg, lr=lr,
                         out_capacity=1)
        n = g.n
        self.accum = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.visits = torch.zeros(n, dtype=torch.int32, device=self.dev)
        self.sets = ops.densify_select(self.accum, self.visits, g, self.tau_g, self.tau_s)
        self.ws_densify = ops.workspace(A.lib().adp_densify_select_workspace_size(n), self.dev)
        self.d_new_n = torch.zeros(1, dtype=torch.int64, device=self.dev)
        self.cand = self.sets.split  # the whole list: the first counts[0] entries are ids
        # probe: one step into a population as large as the worst case of this input
        probe_cap = n + n * (self.params.n_max + 1)
        self._alloc_out(1)
        noise = torch.zeros((n, 2, 3), dtype=torch.float32, device=self.dev)
        g0 = [t.clone() for t in g.tensors()]
        m0, v0, t0 = self.m.clone(), self.v.clone(), self.adam_t.clone()
        self._probe = True
        plan = self.step(noise)
        torch.cuda.synchronize()
        need = int(self.d_new_n.item())
        # the probe's Adam step is undone so the first real step starts from the input
        for d, s in zip(g.tensors(), g0):
            d.copy_(s)
        self.m, self.v = m0, v0
        self.adam_t.copy_(t0)
        self._probe = False
        self._alloc_out(min(probe_cap, int(need * out_margin) + 1024))
        torch.cuda.synchronize()
        del plan

    def _alloc_out(self, cap):
        self.out_capacity = cap
        self.out = ops.Gaussians(cap, self.g.sh_degree, self.dev, zero=False)
        self.m_out = ops.Gaussians(cap, self.g.sh_degree, self.dev, zero=False)
        self.v_out = ops.Gaussians(cap, self.g.sh_degree, self.dev, zero=False)

    def step(self, noise, timer: StageTimer = None):
        """One step; returns (new Gaussians, new m, new v, split plan); the new size
        (split and clones) is self.d_new_n."""
        g, cams, prm, n = self.g, self.cams, self.params, self.g.n
        mark = timer.mark if timer else (lambda name: None)
        mark("project")
        ops.project(g, cams, prm, self.pr)
        mark("bin_sort")
        ops.bin_sort(n, self.pr, cams, prm, bins=self.bins, ws=self.ws_bins, grow=False,
                     status=self.status)
        mark("render")
        ops.render(n, self.pr, self.bins, cams, self.bg, prm, self.img)
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            mark("error_stats")
            ops.error_stats(self.img.rgb, self.target, self.img.dominant, n, cams, prm, self.maps,
                            self.count, self.mass)
            mark("error_end")
        mark("render_backward")
        self.accum.zero_()
        self.visits.zero_()
        ops.render_backward(g, self.pr, self.bins, self.img, cams, target=self.target, bg=self.bg,
                            params=prm, grad=self.grad, ws=self.ws_bwd,
                            grad2d_accum=self.accum, grad2d_visits=self.visits)
        mark("densify_select")
        ops.densify_select(self.accum, self.visits, g, self.tau_g, self.tau_s, out=self.sets,
                           ws=self.ws_densify, status=self.status)
        # the regions of the selected candidates (beside the error map's stream) and
        # the candidates' Adam step run concurrently
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            mark("error_regions")
            ops.error_regions(self.maps, self.img.dominant, self.target, n, cams, self.cand, prm,
                              regions=self.regions, ws=self.ws_regions, grow=False,
                              status=self.status)
            mark("error_regions_end")
        mark("adam_rows")
        ops.adam_step_rows(g, self.grad, self.m, self.v, self.cand, self.adam_t, self.lr)
        mark("join")
        main.wait_stream(self.side)
        mark("split_plan")
        plan = ops.split_plan_overlapped(g, cams, self.regions, self.cand, self.count, prm,
                                         ws=self.ws_split, status_word=self.status)
        mark("split_apply")
        ops.split_apply_adam(g, self.grad, self.m, self.v, plan, self.regions, self.cand, noise,
                             self.adam_t, self.out, self.m_out, self.v_out, prm, self.lr,
                             overlapped=True)
        mark("clone")
        ops.split_clone(g, plan, self.regions, self.cand, self.sets.clone, self.sets.counts[1:],
                        n, self.out, self.m_out, self.v_out, d_new_n=self.d_new_n)
        mark("end")
        return self.out, self.m_out, self.v_out, plan

    def check_capacity(self, plan=None):
        self.check_status()
        ok = (int(self.bins.n_inst.item()) <= self.bins.capacity and
              int(self.regions.count.item()) <= self.regions.capacity)
        if plan is not None:
            ok = ok and int(self.d_new_n.item()) <= self.out_capacity
        return ok
