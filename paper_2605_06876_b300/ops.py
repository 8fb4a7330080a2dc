"""Thin torch-side binding of the C ABI: device buffers as torch tensors, one
Python function per entry point. Argument marshalling only -- every step of the
hot path runs in libadpsplit.so; there is no CPU or PyTorch fallback."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi as A

F32, I32, I64, U8, F64 = torch.float32, torch.int32, torch.int64, torch.uint8, torch.float64


def sh_coeffs(deg):
    return (deg + 1) ** 2


def sh_planes(deg):
    return (3 * sh_coeffs(deg) + 3) // 4


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def n_tiles(cams, tile_w=16, tile_h=16):
    return sum(((int(c["width"]) + tile_w - 1) // tile_w) * ((int(c["height"]) + tile_h - 1) // tile_h)
               for c in cams)


def n_pixels(cams):
    return sum(int(c["width"]) * int(c["height"]) for c in cams)


def workspace(nbytes, device="cuda"):
    return torch.empty(max(int(nbytes), 256), dtype=U8, device=device)


def status_word(device="cuda"):
    """A zeroed device status word for the calls with bounded device waits."""
    return torch.zeros(1, dtype=I32, device=device)


def check_status(word, what="step"):
    """Reads a device status word (a synchronisation) and raises if a call that
    was given it reported an error (ADP_ERR_TIMEOUT: a bounded wait gave up)."""
    v = int(word.item())
    if v != 0:
        raise RuntimeError(f"{what}: device status {A.STATUS_NAMES.get(v, v)}")


# --------------------------------------------------------------------------- Gaussians

class Gaussians:
    """Gaussian parameters (or gradients / Adam moments) as float4 planes."""

    def __init__(self, n, sh_degree, device="cuda", zero=True, row_mask=False):
        alloc = torch.zeros if zero else torch.empty
        self.n = int(n)
        self.sh_degree = int(sh_degree)
        self.mean_logit = alloc((self.n, 4), dtype=F32, device=device)
        self.logscale = alloc((self.n, 4), dtype=F32, device=device)
        self.quat = alloc((self.n, 4), dtype=F32, device=device)
        self.sh = alloc((sh_planes(sh_degree), self.n, 4), dtype=F32, device=device)
        # gradients only: rows with rows[i] == 0 are zero and never touched
        self.rows = (torch.zeros(self.n, dtype=torch.uint8, device=device) if row_mask
                     else None)

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        n = scene["mean"].shape[0]
        deg = int(scene["sh_degree"])
        g = cls(n, deg, device, zero=False)
        ml = np.concatenate([scene["mean"], scene["logit"][:, None]], 1)
        ls = np.concatenate([scene["logscale"], np.zeros((n, 1), np.float32)], 1)
        flat = scene["sh"].reshape(n, 3 * sh_coeffs(deg))
        pad = np.zeros((n, 4 * sh_planes(deg)), np.float32)
        pad[:, :flat.shape[1]] = flat
        sh = pad.reshape(n, sh_planes(deg), 4).transpose(1, 0, 2)
        g.mean_logit.copy_(torch.from_numpy(np.ascontiguousarray(ml, np.float32)))
        g.logscale.copy_(torch.from_numpy(np.ascontiguousarray(ls, np.float32)))
        g.quat.copy_(torch.from_numpy(np.ascontiguousarray(scene["quat"], np.float32)))
        g.sh.copy_(torch.from_numpy(np.ascontiguousarray(sh, np.float32)))
        return g

    def to_scene(self):
        n, deg = self.n, self.sh_degree
        K = sh_coeffs(deg)
        ml = self.mean_logit.cpu().numpy()
        sh = self.sh.cpu().numpy().transpose(1, 0, 2).reshape(n, 4 * sh_planes(deg))[:, :3 * K]
        return {"mean": ml[:, :3].copy(), "logit": ml[:, 3].copy(),
                "logscale": self.logscale.cpu().numpy()[:, :3].copy(),
                "quat": self.quat.cpu().numpy().copy(), "sh": sh.reshape(n, K, 3).copy(),
                "sh_degree": deg}

    def tensors(self):
        return [self.mean_logit, self.logscale, self.quat, self.sh]

    def zeros_like(self):
        return Gaussians(self.n, self.sh_degree, self.mean_logit.device)

    def clone(self):
        g = Gaussians(self.n, self.sh_degree, self.mean_logit.device, zero=False)
        for d, s in zip(g.tensors(), self.tensors()):
            d.copy_(s)
        return g

    def dense(self):
        """The gradient with every masked-out row written as zero (a copy)."""
        out = Gaussians(self.n, self.sh_degree, self.mean_logit.device, zero=False)
        keep = (self.rows != 0) if self.rows is not None else None
        for d, s in zip(out.tensors(), self.tensors()):
            d.copy_(s)
            if keep is not None:
                if d.dim() == 3:
                    d[:, ~keep] = 0
                else:
                    d[~keep] = 0
        return out

    def c(self):
        return A.AdpGaussians(self.n, self.sh_degree, 0, _p(self.mean_logit), _p(self.logscale),
                              _p(self.quat), _p(self.sh),
                              _p(self.rows) if self.rows is not None else None)


# --------------------------------------------------------------------------- buffers

@dataclass
class Projected:
    xyod: torch.Tensor
    conic: torch.Tensor
    rgb: torch.Tensor
    rect: torch.Tensor
    tiles: torch.Tensor

    @classmethod
    def alloc(cls, records, device="cuda"):
        return cls(torch.empty((records, 4), dtype=F32, device=device),
                   torch.empty((records, 4), dtype=F32, device=device),
                   torch.empty((records, 4), dtype=F32, device=device),
                   torch.empty((records, 4), dtype=I32, device=device),
                   torch.empty(records, dtype=I32, device=device))

    def c(self):
        return A.AdpProjected(_p(self.xyod), _p(self.conic), _p(self.rgb), _p(self.rect),
                              _p(self.tiles))


@dataclass
class Bins:
    inst: torch.Tensor
    ranges: torch.Tensor
    n_inst: torch.Tensor

    @classmethod
    def alloc(cls, capacity, tiles, device="cuda"):
        return cls(torch.empty(max(int(capacity), 1), dtype=I32, device=device),
                   torch.empty((tiles, 2), dtype=I32, device=device),
                   torch.zeros(1, dtype=I64, device=device))

    @property
    def capacity(self):
        return self.inst.numel()

    def c(self):
        return A.AdpBins(self.capacity, _p(self.inst), _p(self.ranges), _p(self.n_inst))


@dataclass
class Image:
    rgb: torch.Tensor
    T: torch.Tensor
    n_contrib: torch.Tensor
    last: torch.Tensor
    dominant: torch.Tensor

    @classmethod
    def alloc(cls, P, device="cuda"):
        return cls(torch.empty((P, 3), dtype=F32, device=device),
                   torch.empty(P, dtype=F32, device=device), torch.empty(P, dtype=I32, device=device),
                   torch.empty(P, dtype=I32, device=device), torch.empty(P, dtype=I32, device=device))

    def c(self):
        return A.AdpImage(_p(self.rgb), _p(self.T), _p(self.n_contrib), _p(self.last),
                          _p(self.dominant))


@dataclass
class ErrorMaps:
    E: torch.Tensor
    mask: torch.Tensor
    minmax: torch.Tensor

    @classmethod
    def alloc(cls, P, V, device="cuda"):
        return cls(torch.empty(P, dtype=F32, device=device), torch.empty(P, dtype=U8, device=device),
                   torch.empty((V, 2), dtype=F32, device=device))

    def c(self):
        return A.AdpErrorMaps(_p(self.E), _p(self.mask), _p(self.minmax))


@dataclass
class Regions:
    view: torch.Tensor
    parent: torch.Tensor
    label: torch.Tensor
    band: torch.Tensor
    moments: torch.Tensor
    stats: torch.Tensor
    count: torch.Tensor
    labels: torch.Tensor = None

    @classmethod
    def alloc(cls, capacity, P=None, device="cuda"):
        cap = max(int(capacity), 1)
        mk = lambda *s, dt: torch.empty(s, dtype=dt, device=device)
        return cls(mk(cap, dt=I32), mk(cap, dt=I32), mk(cap, dt=I32), mk(cap, dt=I32),
                   mk(cap, 6, dt=I64), mk(cap, 12, dt=F64), torch.zeros(1, dtype=I64, device=device),
                   None if P is None else mk(P, dt=I32))

    @classmethod
    def from_arrays(cls, view, parent, label, stats, band=None, moments=None, device="cuda"):
        """A region table given by the caller (e.g. from another implementation)."""
        R = len(view)
        r = cls.alloc(max(R, 1), None, device)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        if R:
            r.view[:R] = t(view, I32)
            r.parent[:R] = t(parent, I32)
            r.label[:R] = t(label, I32)
            r.stats[:R] = t(stats, F64)
            r.band[:R] = t(band if band is not None else np.zeros(R), I32)
            r.moments[:R] = t(moments if moments is not None else np.zeros((R, 6)), I64)
        r.count[0] = R
        return r

    @property
    def capacity(self):
        return self.view.numel()

    def c(self):
        return A.AdpRegions(self.capacity, _p(self.view), _p(self.parent), _p(self.label),
                            _p(self.band), _p(self.moments), _p(self.stats), _p(self.count),
                            _p(self.labels))

    def to_numpy(self):
        R = min(int(self.count.item()), self.capacity)
        return {"view": self.view[:R].cpu().numpy(), "parent": self.parent[:R].cpu().numpy(),
                "label": self.label[:R].cpu().numpy(), "band": self.band[:R].cpu().numpy(),
                "moments": self.moments[:R].cpu().numpy(), "stats": self.stats[:R].cpu().numpy()}


# --------------------------------------------------------------------------- entry points

def project(g: Gaussians, cams, params=None, out: Projected = None, stream=None):
    """adp_project: EWA projection into every view."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    out = out or Projected.alloc(len(cams) * g.n, g.mean_logit.device)
    gc, oc = g.c(), out.c()
    A.check(A.lib().adp_project(C.byref(gc), ca, len(cams), C.byref(params), C.byref(oc),
                                _stream(stream)), "adp_project")
    return out


def bin_sort_workspace_size(n, n_views, capacity):
    return A.lib().adp_bin_sort_workspace_size(n, n_views, capacity)


def bin_sort(n, pr: Projected, cams, params=None, capacity=None, bins: Bins = None, ws=None,
             stream=None, grow=True, status=None):
    """adp_bin_sort. With grow=True an overflowing capacity is enlarged and the call
    repeated (this reads the instance count back, a synchronisation)."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    V = len(cams)
    dev = pr.xyod.device
    if bins is None:
        if capacity is None:
            capacity = max(1024, int(pr.tiles.sum().item() * 1.0) + 1)
        bins = Bins.alloc(capacity, n_tiles(cams, params.tile_w, params.tile_h), dev)
    need = bin_sort_workspace_size(n, V, bins.capacity)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    pc, bc = pr.c(), bins.c()
    A.check(A.lib().adp_bin_sort(n, C.byref(pc), ca, V, C.byref(params), C.byref(bc), _p(ws),
                                 ws.numel(), _p(status), _stream(stream)), "adp_bin_sort")
    if grow:
        k = int(bins.n_inst.item())
        if k > bins.capacity:
            return bin_sort(n, pr, cams, params, capacity=int(k * 1.25) + 1, stream=stream,
                            status=status)
    return bins


def render(n, pr: Projected, bins: Bins, cams, bg=(0.0, 0.0, 0.0), params=None, out: Image = None,
           stream=None):
    """adp_render: compositing and dominant map."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    out = out or Image.alloc(n_pixels(cams), pr.xyod.device)
    bgc = (C.c_float * 3)(*[float(x) for x in bg])
    pc, bc, oc = pr.c(), bins.c(), out.c()
    A.check(A.lib().adp_render(n, C.byref(pc), C.byref(bc), ca, len(cams), bgc, C.byref(params),
                               C.byref(oc), _stream(stream)), "adp_render")
    return out


def error_stats(img, target, dominant, n, cams, params=None, maps: ErrorMaps = None, count=None,
                mass=None, stream=None):
    """adp_error_stats: E, M, bands, per-Gaussian count and mass."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    dev = img.device
    maps = maps or ErrorMaps.alloc(n_pixels(cams), len(cams), dev)
    count = count if count is not None else torch.empty(max(n, 1), dtype=I32, device=dev)
    mass = mass if mass is not None else torch.empty(max(n, 1), dtype=F64, device=dev)
    mc = maps.c()
    A.check(A.lib().adp_error_stats(_p(img), _p(target), _p(dominant), n, ca, len(cams),
                                    C.byref(params), C.byref(mc), _p(count), _p(mass),
                                    _stream(stream)), "adp_error_stats")
    return maps, count, mass


def select_topk(mass, n, k, out=None, ws=None, stream=None, status=None):
    """adp_select_topk: ids of the k largest masses, ascending."""
    k = min(int(k), int(n))
    out = out if out is not None else torch.empty(max(k, 1), dtype=I32, device=mass.device)
    need = A.lib().adp_select_topk_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, mass.device)
    A.check(A.lib().adp_select_topk(_p(mass), n, k, _p(out), _p(ws), ws.numel(), _p(status),
                                    _stream(stream)), "adp_select_topk")
    return out[:k]


def error_regions(maps: ErrorMaps, dominant, target, n, cams, candidates, params=None,
                  capacity=None, regions: Regions = None, ws=None, stream=None, labels=False,
                  grow=True, status=None):
    """adp_error_regions: erosion, 8-connected regions, area filter, statistics."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    V = len(cams)
    dev = maps.E.device
    P = n_pixels(cams)
    if regions is None:
        regions = Regions.alloc(capacity or max(1024, P // 64), P if labels else None, dev)
    need = A.lib().adp_error_regions_workspace_size(n, V, ca)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    nc = 0 if candidates is None else int(candidates.numel())
    mc, rc = maps.c(), regions.c()
    A.check(A.lib().adp_error_regions(C.byref(mc), _p(dominant), _p(target), n, ca, V,
                                      _p(candidates) if nc else None, nc, C.byref(params),
                                      C.byref(rc), _p(ws), ws.numel(), _p(status),
                                      _stream(stream)), "adp_error_regions")
    if grow:
        cnt = int(regions.count.item())
        if cnt > regions.capacity:
            return error_regions(maps, dominant, target, n, cams, candidates, params,
                                 int(cnt * 1.25) + 1, None, None, stream, labels, False, status)
    return regions


def split_workspace_size(n, n_cand, region_capacity):
    return A.lib().adp_split_workspace_size(n, n_cand, region_capacity)


@dataclass
class SplitPlan:
    status: torch.Tensor
    n_children: torch.Tensor
    new_n: int
    ws: torch.Tensor
    d_new_n: torch.Tensor
    # the whole status and child-count buffers (at least one entry), which the
    # second part of a two-call overlapped plan writes through again
    status_buf: torch.Tensor = None
    nch_buf: torch.Tensor = None


def split_plan(g: Gaussians, cams, regions: Regions, candidates, count, params=None, ws=None,
               stream=None, sync=True, status_word=None):
    """adp_split_plan: statuses and child counts. With sync=True the new size is read
    back (one synchronisation); otherwise it stays on the device (plan.d_new_n)."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    dev = g.mean_logit.device
    nc = int(candidates.numel())
    need = split_workspace_size(g.n, nc, regions.capacity)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    status = torch.empty(max(nc, 1), dtype=U8, device=dev)
    nch = torch.empty(max(nc, 1), dtype=I32, device=dev)
    d_new_n = torch.empty(1, dtype=I64, device=dev)
    h_new_n = C.c_int64(0)
    gc, rc = g.c(), regions.c()
    A.check(A.lib().adp_split_plan(C.byref(gc), ca, len(cams), C.byref(rc), _p(candidates), nc,
                                   _p(count), C.byref(params), _p(status), _p(nch), _p(d_new_n),
                                   C.byref(h_new_n) if sync else None, _p(ws), ws.numel(),
                                   _p(status_word), _stream(stream)), "adp_split_plan")
    return SplitPlan(status[:nc], nch[:nc], int(h_new_n.value) if sync else None, ws, d_new_n)


def split_plan_overlapped(g: Gaussians, cams, regions: Regions, candidates, count, params=None,
                          ws=None, stream=None, status_word=None, part="all", plan=None):
    """adp_split_plan_overlapped: the statuses and kept rows on the stream, the
    proposals and merges on the library's auxiliary stream; must be followed by
    split_apply_adam(..., overlapped=True), which joins them. part="statuses"
    enqueues only the first part (adp_split_plan_statuses) and returns the plan;
    part="proposals" takes that plan (same arguments, the same workspace) and
    enqueues the second (adp_split_plan_proposals_overlapped)."""
    fn = {"all": "adp_split_plan_overlapped", "statuses": "adp_split_plan_statuses",
          "proposals": "adp_split_plan_proposals_overlapped"}[part]
    params = params or A.default_params()
    ca = A.cameras(cams)
    dev = g.mean_logit.device
    nc = int(candidates.numel())
    if part == "proposals":
        if plan is None:
            raise ValueError("part='proposals' needs the plan of part='statuses'")
        ws = plan.ws
        status, nch, d_new_n = plan.status_buf, plan.nch_buf, plan.d_new_n
    else:
        need = split_workspace_size(g.n, nc, regions.capacity)
        if ws is None or ws.numel() < need:
            ws = workspace(need, dev)
        status = torch.empty(max(nc, 1), dtype=U8, device=dev)
        nch = torch.empty(max(nc, 1), dtype=I32, device=dev)
        d_new_n = torch.empty(1, dtype=I64, device=dev)
    gc, rc = g.c(), regions.c()
    A.check(getattr(A.lib(), fn)(C.byref(gc), ca, len(cams), C.byref(rc), _p(candidates), nc,
                                 _p(count), C.byref(params), _p(status), _p(nch), _p(d_new_n),
                                 _p(ws), ws.numel(), _p(status_word), _stream(stream)), fn)
    return SplitPlan(status[:nc], nch[:nc], None, ws, d_new_n, status, nch)


def split_apply(g: Gaussians, plan: SplitPlan, regions: Regions, candidates, noise, params=None,
                m_in: Gaussians = None, v_in: Gaussians = None, with_state=True, stream=None,
                out: Gaussians = None, m_out: Gaussians = None, v_out: Gaussians = None):
    """adp_split_apply: the new population (and Adam moments). Given out (and m_out,
    v_out) the population is written into those capacity buffers (entries
    [0, plan.d_new_n)); otherwise buffers of exactly the planned size are made."""
    params = params or A.default_params()
    dev = g.mean_logit.device
    if out is None:
        new_n = plan.new_n if plan.new_n is not None else int(plan.d_new_n.item())
        out = Gaussians(new_n, g.sh_degree, dev, zero=False)
        m_out = Gaussians(new_n, g.sh_degree, dev, zero=False) if with_state else None
        v_out = Gaussians(new_n, g.sh_degree, dev, zero=False) if with_state else None
    nc = int(candidates.numel())
    if noise is None:
        noise = torch.zeros((max(nc, 1), 2, 3), dtype=F32, device=dev)
    gc, oc, rc = g.c(), out.c(), regions.c()
    mic = m_in.c() if m_in is not None else None
    vic = v_in.c() if v_in is not None else None
    moc = m_out.c() if m_out is not None else None
    voc = v_out.c() if v_out is not None else None
    ref = lambda s: C.byref(s) if s is not None else None
    A.check(A.lib().adp_split_apply(C.byref(gc), ref(mic), ref(vic), C.byref(rc), _p(candidates), nc,
                                    _p(plan.status), _p(plan.n_children), _p(noise),
                                    C.byref(params), C.byref(oc), ref(moc), ref(voc), _p(plan.ws),
                                    plan.ws.numel(), _stream(stream)), "adp_split_apply")
    return out, m_out, v_out


def split_apply_adam(g: Gaussians, grad: Gaussians, m_in: Gaussians, v_in: Gaussians,
                     plan: SplitPlan, regions: Regions, candidates, noise, step, out: Gaussians,
                     m_out: Gaussians, v_out: Gaussians, params=None, lr=None, beta1=0.9,
                     beta2=0.999, eps=1e-15, stream=None, overlapped=False, part=None):
    """adp_split_apply_adam: the compaction with the Adam step applied to every kept
    non-candidate row on the way (candidates first via adam_step_rows). With
    overlapped=True it follows split_plan_overlapped: adp_split_keep_overlapped
    writes the kept rows while the merge finishes, then adp_split_append_overlapped
    joins and appends (part="keep" or "append" issues one of the two)."""
    params = params or A.default_params()
    lrc = (C.c_float * 6)(*[float(x) for x in (lr or ADAM_LR)])
    host_step, d_step = _step_arg(step)
    nc = int(candidates.numel())
    if noise is None:
        noise = torch.zeros((max(nc, 1), 2, 3), dtype=F32, device=g.mean_logit.device)
    gc, grc, mic, vic = g.c(), grad.c(), m_in.c(), v_in.c()
    oc, moc, voc, rc = out.c(), m_out.c(), v_out.c(), regions.c()
    if not overlapped:
        fns = ["adp_split_apply_adam"]
    else:
        fns = {None: ["adp_split_keep_overlapped", "adp_split_append_overlapped"],
               "keep": ["adp_split_keep_overlapped"],
               "append": ["adp_split_append_overlapped"]}[part]
    for fn in fns:
        A.check(getattr(A.lib(), fn)(
            C.byref(gc), C.byref(grc), C.byref(mic), C.byref(vic), C.byref(rc), _p(candidates), nc,
            _p(plan.status), _p(plan.n_children), _p(noise), C.byref(params), host_step, d_step,
            lrc, beta1, beta2, eps, C.byref(oc), C.byref(moc), C.byref(voc), _p(plan.ws),
            plan.ws.numel(), _stream(stream)), fn)
    return out, m_out, v_out


def train_step_batched(g: Gaussians, cams, target, params=None, bg=(0.0, 0.0, 0.0),
                       pr: Projected = None, bins: Bins = None, img: Image = None,
                       maps: ErrorMaps = None, count=None, mass=None, grad: Gaussians = None,
                       grad2d_accum=None, grad2d_visits=None, ws=None, status=None, stream=None):
    """adp_train_step_batched: projection, binning, the fused per-tile forward +
    L1 error + backward over all views, error statistics and the per-Gaussian
    gradient. Missing buffers are allocated (bins sized from the rectangle count,
    which reads it back). Returns (pr, bins, img, maps, count, mass, grad)."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    V, n = len(cams), g.n
    dev = g.mean_logit.device
    P = n_pixels(cams)
    pr = pr or Projected.alloc(V * n, dev)
    if bins is None:
        project(g, cams, params, pr, stream)
        bins = Bins.alloc(max(1024, int(pr.tiles.sum().item()) + 1),
                          n_tiles(cams, params.tile_w, params.tile_h), dev)
    img = img or Image.alloc(P, dev)
    maps = maps or ErrorMaps.alloc(P, V, dev)
    count = count if count is not None else torch.empty(max(n, 1), dtype=I32, device=dev)
    mass = mass if mass is not None else torch.empty(max(n, 1), dtype=F64, device=dev)
    grad = grad or Gaussians(n, g.sh_degree, dev, zero=False, row_mask=True)
    need = A.lib().adp_train_step_batched_workspace_size(n, V, ca, C.byref(params),
                                                         bins.capacity)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    bgc = (C.c_float * 3)(*[float(x) for x in bg])
    gc, pc, bc, ic, mc, grc = g.c(), pr.c(), bins.c(), img.c(), maps.c(), grad.c()
    A.check(A.lib().adp_train_step_batched(
        C.byref(gc), ca, V, _p(target), bgc, C.byref(params), C.byref(pc), C.byref(bc),
        C.byref(ic), C.byref(mc), _p(count), _p(mass), C.byref(grc), _p(grad2d_accum),
        _p(grad2d_visits), _p(ws), ws.numel(), _p(status), _stream(stream)),
        "adp_train_step_batched")
    return pr, bins, img, maps, count, mass, grad


@dataclass
class DensifySets:
    split: torch.Tensor   # int32 [n]: the first counts[0] entries are the split ids
    clone: torch.Tensor   # int32 [n]: the first counts[1] entries are the clone ids
    counts: torch.Tensor  # int64 [2] on the device


def densify_select(grad2d_accum, grad2d_visits, g: Gaussians, tau_g, tau_s, out: DensifySets = None,
                   ws=None, stream=None, status=None):
    """adp_densify_select: Eq. 2 split candidates and the clone candidates."""
    dev = g.mean_logit.device
    if out is None:
        n1 = max(g.n, 1)
        out = DensifySets(torch.empty(n1, dtype=I32, device=dev),
                          torch.empty(n1, dtype=I32, device=dev),
                          torch.zeros(2, dtype=I64, device=dev))
    need = A.lib().adp_densify_select_workspace_size(g.n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    gc = g.c()
    A.check(A.lib().adp_densify_select(_p(grad2d_accum), _p(grad2d_visits), C.byref(gc),
                                       float(tau_g), float(tau_s), _p(out.split), _p(out.clone),
                                       _p(out.counts), _p(ws), ws.numel(), _p(status),
                                       _stream(stream)), "adp_densify_select")
    return out


def split_clone(g: Gaussians, plan: SplitPlan, regions: Regions, candidates, clone_ids, d_n_clone,
                max_clone, out: Gaussians, m_out: Gaussians = None, v_out: Gaussians = None,
                d_new_n=None, stream=None):
    """adp_split_clone: copies of the clone ids appended after the split's rows (call
    after split_apply / split_apply_adam with the same plan). Returns the device
    new size."""
    d_new_n = d_new_n if d_new_n is not None else torch.zeros(1, dtype=I64, device=out.mean_logit.device)
    oc = out.c()
    mc = m_out.c() if m_out is not None else None
    vc = v_out.c() if v_out is not None else None
    A.check(A.lib().adp_split_clone(
        g.n, int(candidates.numel()), regions.capacity, _p(clone_ids), _p(d_n_clone),
        int(max_clone), C.byref(oc), C.byref(mc) if mc is not None else None,
        C.byref(vc) if vc is not None else None, _p(plan.ws), plan.ws.numel(), _p(d_new_n),
        _stream(stream)), "adp_split_clone")
    return d_new_n


def dssim_loss_grad(img, target, cams, lam=0.2, params=None, dL=None, loss=None, ws=None,
                    stream=None):
    """adp_dssim_loss_grad: dL/dI for L = (1 - lam) L1 + lam (1 - SSIM) per view, and
    (in loss, float64 [V][2]) each view's mean L1 and mean SSIM."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    V = len(cams)
    dev = img.device
    dL = dL if dL is not None else torch.empty_like(img)
    loss = loss if loss is not None else torch.empty((V, 2), dtype=F64, device=dev)
    need = A.lib().adp_dssim_workspace_size(V, ca)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    A.check(A.lib().adp_dssim_loss_grad(_p(img), _p(target), ca, V, float(lam), C.byref(params),
                                        _p(dL), _p(loss), _p(ws), ws.numel(), _stream(stream)),
            "adp_dssim_loss_grad")
    return dL, loss


def render_backward(g: Gaussians, pr: Projected, bins: Bins, fwd: Image, cams, target=None,
                    dL_drgb=None, bg=(0.0, 0.0, 0.0), params=None, grad: Gaussians = None, ws=None,
                    stream=None, grad2d_accum=None, grad2d_visits=None):
    """adp_render_backward: gradients of the L1 loss (or of dL_drgb) for every parameter.
    grad2d_accum (float32 [n]) and grad2d_visits (int32 [n]), if given, accumulate
    the densification statistic of Eq. 2 (see adpsplit.h)."""
    params = params or A.default_params()
    ca = A.cameras(cams)
    V = len(cams)
    dev = g.mean_logit.device
    grad = grad or Gaussians(g.n, g.sh_degree, dev, zero=False)
    need = A.lib().adp_render_backward_workspace_size(g.n, V)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    bgc = (C.c_float * 3)(*[float(x) for x in bg])
    gc, pc, bc, fc, grc = g.c(), pr.c(), bins.c(), fwd.c(), grad.c()
    A.check(A.lib().adp_render_backward(C.byref(gc), C.byref(pc), C.byref(bc), C.byref(fc),
                                        _p(target), _p(dL_drgb), ca, V, bgc, C.byref(params),
                                        C.byref(grc), _p(grad2d_accum), _p(grad2d_visits), _p(ws),
                                        ws.numel(), _stream(stream)),
            "adp_render_backward")
    return grad


ADAM_LR = (1.6e-4, 0.05, 0.005, 0.001, 0.0025, 0.0025 / 20.0)


def adam_step(param: Gaussians, grad: Gaussians, m: Gaussians, v: Gaussians, step, lr=ADAM_LR,
              beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """adp_adam_step: one in-place bias-corrected Adam step. `step` is an int, or a
    device int32 tensor of one element holding the step number (advanced by the call)."""
    lrc = (C.c_float * 6)(*[float(x) for x in lr])
    pc, gc, mc, vc = param.c(), grad.c(), m.c(), v.c()
    host_step, d_step = _step_arg(step)
    A.check(A.lib().adp_adam_step(C.byref(pc), C.byref(gc), C.byref(mc), C.byref(vc), host_step,
                                  d_step, lrc, beta1, beta2, eps, _stream(stream)),
            "adp_adam_step")


def adam_step_rows(param: Gaussians, grad: Gaussians, m: Gaussians, v: Gaussians, rows, step,
                   lr=ADAM_LR, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """adp_adam_step_rows: the Adam step on the listed rows only (a device step
    counter is read, not advanced)."""
    lrc = (C.c_float * 6)(*[float(x) for x in lr])
    pc, gc, mc, vc = param.c(), grad.c(), m.c(), v.c()
    host_step, d_step = _step_arg(step)
    A.check(A.lib().adp_adam_step_rows(C.byref(pc), C.byref(gc), C.byref(mc), C.byref(vc),
                                       _p(rows), int(rows.numel()), host_step, d_step, lrc, beta1,
                                       beta2, eps, _stream(stream)), "adp_adam_step_rows")


def _step_arg(step):
    """(host step, device step pointer) from an int or a one-element int32 tensor."""
    if isinstance(step, torch.Tensor):
        return 0, _p(step)
    return int(step), None
