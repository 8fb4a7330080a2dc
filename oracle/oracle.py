"""numpy front end of the FP64 oracle (adp_oracle.c).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline leg
of the benchmark are the only users. It shares no code with the CUDA path and never
reads anything the CUDA path produced.

Every function names the step of the paper it follows; the arithmetic lives in
adp_oracle.c, except the densification selection of Sec. 3 (Eq. 2) and the clone
bookkeeping at the end of this file, which are a few plain numpy lines. Inputs
come from the `scenes` module (float32), widened to float64.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KEEP, ADAPTIVE, FALLBACK, RESET = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compiles adp_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double),
                ("fy", C.c_double), ("px", C.c_double), ("py", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3)]


class OrcConfig(C.Structure):
    _fields_ = [("near_plane", C.c_double), ("low_pass", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_min", C.c_double),
                ("tie_alpha_min", C.c_double), ("tie_stop", C.c_double),
                ("tie_alpha_max", C.c_double), ("tie_margin", C.c_double),
                ("tie_capture", C.c_double), ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class OrcSplitConfig(C.Structure):
    _fields_ = [("gamma_d", C.c_double), ("gamma_c", C.c_double), ("eps_t", C.c_double),
                ("eta", C.c_double), ("scale_floor", C.c_double), ("n_max", C.c_int32),
                ("pad", C.c_int32)]


_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)
_u8 = C.POINTER(C.c_uint8)
_vp = C.c_void_p


def _declare(L):
    L.orc_sh_basis.argtypes = [C.c_int32, C.c_int64, _vp, _vp]
    L.orc_quat_to_rot.argtypes = [C.c_int64, _vp, _vp]
    L.orc_rot_to_quat.argtypes = [C.c_int64, _vp, _vp]
    L.orc_project.argtypes = [C.c_int64, C.c_int32, _vp, C.POINTER(OrcCamera),
                              C.POINTER(OrcConfig)] + [_vp] * 10
    L.orc_render.argtypes = [C.c_int64] + [_vp] * 7 + [C.c_int32, C.c_int32, _vp,
                                                       C.POINTER(OrcConfig), C.c_int64, _vp] + [_vp] * 7
    L.orc_tile_lists.argtypes = [C.c_int64, _vp, _vp, _vp, C.c_int32, C.c_int32, _vp,
                                 C.c_int64, _vp]
    L.orc_tile_lists.restype = C.c_int64
    L.orc_error_map.argtypes = [C.c_int32, C.c_int32, _vp, _vp, C.c_float, C.c_int32] + [_vp] * 5
    L.orc_erode.argtypes = [C.c_int32, C.c_int32, _vp, C.c_int32, _vp]
    L.orc_gauss_stats.argtypes = [C.c_int64, _vp, _vp, _vp, C.c_int64, _vp, _vp]
    L.orc_topk_mass.argtypes = [C.c_int64, _vp, C.c_int64, _vp]
    L.orc_regions.argtypes = [C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_int64, _vp,
                              _vp, C.c_int32, _vp, C.c_int64] + [_vp] * 6
    L.orc_regions.restype = C.c_int64
    L.orc_child_proposal.argtypes = [_vp, C.POINTER(OrcCamera), _vp, C.c_double, C.c_double,
                                     _vp, _vp, _vp, _vp, _vp]
    L.orc_merge.argtypes = [C.c_int32, _vp, _vp, _vp, _vp, C.c_double, C.c_double,
                            C.c_double] + [_vp] * 6
    L.orc_merge.restype = C.c_int32
    L.orc_split.argtypes = [C.c_int64, C.c_int32, _vp, _vp, _vp, _vp, C.c_int32, C.c_int64,
                            _vp, _vp, _vp, _vp, C.c_int64, _vp, _vp, _vp,
                            C.POINTER(OrcSplitConfig), _vp, _vp, C.c_int64, _vp, _vp, _vp]
    L.orc_split.restype = C.c_int64
    L.orc_grad.argtypes = [C.c_int64, C.c_int32, _vp, C.POINTER(OrcCamera), C.POINTER(OrcConfig),
                           _vp, _vp, C.c_double, C.c_int64, _vp, _vp, _vp]
    L.orc_adam.argtypes = [C.c_int64, C.c_int32, _vp, _vp, _vp, _vp, C.c_int32, _vp,
                           C.c_double, C.c_double, C.c_double]
    L.orc_version.restype = C.c_int32


def _p(a):
    """Pointer to a contiguous numpy array (None passes NULL)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# --------------------------------------------------------------------------- params

def n_params(deg: int) -> int:
    return 11 + 3 * (deg + 1) ** 2


def theta_of(scene) -> np.ndarray:
    """Flat FP64 parameter matrix [n, 11 + 3K]: mean, logit, log-scale, quat, SH."""
    n = scene["mean"].shape[0]
    return np.ascontiguousarray(np.concatenate([
        scene["mean"].astype(np.float64), scene["logit"].astype(np.float64)[:, None],
        scene["logscale"].astype(np.float64), scene["quat"].astype(np.float64),
        scene["sh"].astype(np.float64).reshape(n, -1)], axis=1))


def scene_of_theta(theta, deg):
    """Inverse of theta_of (values rounded to float32)."""
    n = theta.shape[0]
    K = (deg + 1) ** 2
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"mean": f(theta[:, 0:3]), "logit": f(theta[:, 3]), "logscale": f(theta[:, 4:7]),
            "quat": f(theta[:, 7:11]), "sh": f(theta[:, 11:].reshape(n, K, 3)),
            "sh_degree": int(deg)}


def camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.px, c.py = (float(cam[k]) for k in ("fx", "fy", "px", "py"))
    for i in range(9):
        c.R[i] = float(cam["R"][i])
    for i in range(3):
        c.t[i] = float(cam["t"][i])
    return c


@dataclass
class Config:
    """Forward conventions (3DGS defaults) and tie bands.

    A pixel is a tie when one of the discontinuous decisions of its compositing is
    within an absolute band of its threshold: some alpha_raw within tie_alpha_min of
    1/255 (bit 1), some stop test T (1 - alpha) within tie_stop of 1e-4 (bit 2),
    some alpha_raw within tie_alpha_max of the 0.99 clamp (bit 4), or the two
    largest weights T alpha closer than tie_margin (bit 8). The defaults are the
    stated tolerance's 1e-6 for every band. render() also returns each pixel's
    distances to the four thresholds, so a caller can apply other bands."""
    near_plane: float = 0.2
    low_pass: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    tie_alpha_min: float = 1e-6
    tie_stop: float = 1e-6
    tie_alpha_max: float = 1e-6
    tie_margin: float = 1e-6
    tie_capture: float = 1e-4  # misses this close below 1/255 report their distance
    tile_w: int = 16
    tile_h: int = 16

    def c(self) -> OrcConfig:
        return OrcConfig(self.near_plane, self.low_pass, self.alpha_min, self.alpha_max,
                         self.t_min, self.tie_alpha_min, self.tie_stop, self.tie_alpha_max,
                         self.tie_margin, self.tie_capture, self.tile_w, self.tile_h)


def tie_bits(dist, alpha_min=1e-6, stop=1e-6, alpha_max=1e-6, margin=1e-6):
    """Tie bits (as render() sets them) of per-pixel threshold distances [P, 4]
    under the given absolute bands."""
    d = np.asarray(dist)
    return ((d[:, 0] < alpha_min) * 1 + (d[:, 1] < stop) * 2 + (d[:, 2] < alpha_max) * 4 +
            (d[:, 3] < margin) * 8).astype(np.int32)


@dataclass
class SplitParams:
    """AdpSplit hyper-parameters (Sec. 5.1 defaults; eta from the 3DGS split)."""
    tau_l1: float = 0.1
    r_erode: int = 2
    m_min: int = 5
    n_levels: int = 3
    n_max: int = 19
    gamma_d: float = 2.0
    gamma_c: float = 0.15
    eps_t: float = 1e-8
    eta: float = 0.8
    scale_floor: float = 1e-7

    def c(self) -> OrcSplitConfig:
        return OrcSplitConfig(self.gamma_d, self.gamma_c, self.eps_t, self.eta,
                              self.scale_floor, self.n_max, 0)


# --------------------------------------------------------------------------- basics

def sh_basis(deg, dirs):
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    out = np.zeros((dirs.shape[0], K))
    lib().orc_sh_basis(deg, dirs.shape[0], _p(dirs), _p(out))
    return out


def quat_to_rot(q):
    q = _c(q, np.float64).reshape(-1, 4)
    R = np.zeros((q.shape[0], 9))
    lib().orc_quat_to_rot(q.shape[0], _p(q), _p(R))
    return R.reshape(-1, 3, 3)


def rot_to_quat(R):
    R = _c(R, np.float64).reshape(-1, 9)
    q = np.zeros((R.shape[0], 4))
    lib().orc_rot_to_quat(R.shape[0], _p(R), _p(q))
    return q


# --------------------------------------------------------------------------- forward

def project(theta, deg, cam, cfg: Config = Config()):
    """EWA projection of every Gaussian into one camera (Sec. 3)."""
    theta = _c(theta, np.float64)
    n = theta.shape[0]
    out = dict(mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)),
               depth=np.zeros(n), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               clamped=np.zeros((n, 3), np.int32), box=np.zeros((n, 4), np.int32),
               rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32))
    cc, cf = camera(cam), cfg.c()
    lib().orc_project(n, deg, _p(theta), C.byref(cc), C.byref(cf), _p(out["mean2d"]),
                      _p(out["cov2d"]), _p(out["conic"]), _p(out["depth"]), _p(out["opacity"]),
                      _p(out["rgb"]), _p(out["clamped"]), _p(out["box"]), _p(out["rect"]),
                      _p(out["tiles"]))
    return out


def render(proj, cam, bg=(0.0, 0.0, 0.0), cfg: Config = Config(), pixels=None):
    """Front-to-back compositing per pixel (Eq. 1) with the dominant map (Eq. 5).

    pixels=None renders the whole image (candidate scan pruned by a cell grid);
    otherwise the given linear pixel indices are rendered by brute force.
    """
    W, H = int(cam["width"]), int(cam["height"])
    n = proj["depth"].shape[0]
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = _c(pixels, np.int64)
        npix = pix.shape[0]
    bg = _c(bg, np.float64)
    out = dict(rgb=np.zeros((npix, 3)), T=np.zeros(npix), n_contrib=np.zeros(npix, np.int32),
               dominant=np.zeros(npix, np.int32), second=np.zeros(npix, np.int32),
               dist=np.zeros((npix, 4)), tie=np.zeros(npix, np.int32))
    cf = cfg.c()
    lib().orc_render(n, _p(proj["mean2d"]), _p(proj["conic"]), _p(proj["depth"]),
                     _p(proj["opacity"]), _p(proj["rgb"]), _p(proj["box"]), _p(proj["tiles"]),
                     W, H, _p(bg), C.byref(cf), npix, _p(pix), _p(out["rgb"]), _p(out["T"]),
                     _p(out["n_contrib"]), _p(out["dominant"]), _p(out["second"]),
                     _p(out["dist"]), _p(out["tie"]))
    out["margin"] = out["dist"][:, 3].copy()
    return out


def tile_lists(depth_f32, rect, tiles, tiles_x, tiles_y):
    """Per-tile instance lists by definition, ordered by (float32 depth, id)."""
    depth_f32 = _c(depth_f32, np.float32)
    rect = _c(rect, np.int32)
    tiles = _c(tiles, np.int32)
    n = depth_f32.shape[0]
    nt = tiles_x * tiles_y
    start = np.zeros(nt + 1, np.int64)
    total = lib().orc_tile_lists(n, _p(depth_f32), _p(rect), _p(tiles), tiles_x, tiles_y,
                                 _p(start), 0, None)
    inst = np.zeros(max(total, 1), np.int32)
    lib().orc_tile_lists(n, _p(depth_f32), _p(rect), _p(tiles), tiles_x, tiles_y, _p(start),
                         total, _p(inst))
    return start, inst[:total]


# --------------------------------------------------------------------------- error stage

def error_map(img_f32, tgt_f32, tau=0.1, L=3):
    """Min-max normalised L1 error (Eq. 6), mask M and bands B, decided in float32."""
    img = _c(img_f32, np.float32)
    tgt = _c(tgt_f32, np.float32)
    H, W = img.shape[0], img.shape[1]
    P = W * H
    out = dict(raw=np.zeros(P, np.float32), E=np.zeros(P, np.float32), M=np.zeros(P, np.uint8),
               B=np.zeros(P, np.uint8), minmax=np.zeros(2, np.float32))
    lib().orc_error_map(W, H, _p(img), _p(tgt), C.c_float(tau), L, _p(out["raw"]), _p(out["E"]),
                        _p(out["M"]), _p(out["B"]), _p(out["minmax"]))
    return out


def erode(M, W, H, r):
    M = _c(M, np.uint8)
    out = np.zeros(W * H, np.uint8)
    lib().orc_erode(W, H, _p(M), r, _p(out))
    return out


def gauss_stats(M, D, E, n, count=None, mass=None):
    """Error pixels attributed to each Gaussian (pre-erosion M, dominant D)."""
    M, D, E = _c(M, np.uint8), _c(D, np.int32), _c(E, np.float32)
    count = np.zeros(n, np.int32) if count is None else count
    mass = np.zeros(n, np.float64) if mass is None else mass
    lib().orc_gauss_stats(M.shape[0], _p(M), _p(D), _p(E), n, _p(count), _p(mass))
    return count, mass


def topk_mass(mass, k):
    mass = _c(mass, np.float64)
    k = min(int(k), mass.shape[0])
    out = np.zeros(k, np.int32)
    lib().orc_topk_mass(mass.shape[0], _p(mass), k, _p(out))
    return out


def regions(view, W, H, Mero, B, D, n, cand_flag, tgt_f32, m_min=5):
    """Error regions of one view (Eqs. 7-8) and their statistics."""
    Mero, B, D = _c(Mero, np.uint8), _c(B, np.uint8), _c(D, np.int32)
    cand_flag = _c(cand_flag, np.uint8)
    tgt = _c(tgt_f32, np.float32)
    labels = np.zeros(W * H, np.int32)
    args = lambda cap, o: [view, W, H, _p(Mero), _p(B), _p(D), n, _p(cand_flag), _p(tgt), m_min,
                           _p(labels), cap] + [_p(x) for x in o]
    empty = [None] * 6
    cnt = lib().orc_regions(*args(0, empty))
    o = dict(view=np.zeros(cnt, np.int32), parent=np.zeros(cnt, np.int32),
             label=np.zeros(cnt, np.int32), band=np.zeros(cnt, np.int32),
             moments=np.zeros((cnt, 6), np.int64), stats=np.zeros((cnt, 12)))
    lib().orc_regions(*args(cnt, [o["view"], o["parent"], o["label"], o["band"], o["moments"],
                                  o["stats"]]))
    o["labels"] = labels
    return o


def concat_regions(parts):
    keys = ["view", "parent", "label", "band", "moments", "stats"]
    if not parts:
        return dict(view=np.zeros(0, np.int32), parent=np.zeros(0, np.int32),
                    label=np.zeros(0, np.int32), band=np.zeros(0, np.int32),
                    moments=np.zeros((0, 6), np.int64), stats=np.zeros((0, 12)))
    return {k: np.ascontiguousarray(np.concatenate([p[k] for p in parts])) for k in keys}


# --------------------------------------------------------------------------- split

def child_proposal(theta_parent, cam, stats, eps_t=1e-8, scale_floor=1e-7):
    """One child from one region (Eqs. 9-10, Appendix A)."""
    th = _c(theta_parent, np.float64)
    st = _c(stats, np.float64)
    mu, R, s, rgb, ts = np.zeros(3), np.zeros(9), np.zeros(3), np.zeros(3), np.zeros(1)
    cc = camera(cam)
    lib().orc_child_proposal(_p(th), C.byref(cc), _p(st), eps_t, scale_floor, _p(mu), _p(R),
                             _p(s), _p(rgb), _p(ts))
    return dict(mu=mu, R=R.reshape(3, 3), s=s, rgb=rgb, tstar=float(ts[0]))


def merge(mu, R, s, rgb, gamma_d=2.0, gamma_c=0.15, scale_floor=1e-7):
    """Cross-view merge of one parent's proposals (Eqs. 11-12)."""
    mu, R, s, rgb = (_c(a, np.float64) for a in (mu, R, s, rgb))
    M = mu.shape[0]
    gof = np.zeros(M, np.int32)
    g_mu, g_rgb, g_R = np.zeros((M, 3)), np.zeros((M, 3)), np.zeros((M, 9))
    g_s, g_Sig = np.zeros((M, 3)), np.zeros((M, 9))
    ng = lib().orc_merge(M, _p(mu), _p(R), _p(s), _p(rgb), gamma_d, gamma_c, scale_floor,
                         _p(gof), _p(g_mu), _p(g_rgb), _p(g_R), _p(g_s), _p(g_Sig))
    return dict(group_of=gof, n_groups=ng, mu=g_mu[:ng], rgb=g_rgb[:ng],
                R=g_R[:ng].reshape(-1, 3, 3), s=g_s[:ng], Sigma=g_Sig[:ng].reshape(-1, 3, 3))


def split(theta, deg, cams, regs, cand, count, noise, sp: SplitParams = SplitParams(),
          adam_m=None, adam_v=None):
    """The AdpSplit operator and the compaction of the new population."""
    theta = _c(theta, np.float64)
    n, P = theta.shape
    cand = _c(cand, np.int32)
    count = _c(count, np.int32)
    noise = _c(noise, np.float64).reshape(-1)
    ncand = cand.shape[0]
    CamArr = OrcCamera * max(1, len(cams))
    ca = CamArr(*[camera(c) for c in cams])
    status = np.zeros(ncand, np.uint8)
    nchild = np.zeros(ncand, np.int32)
    sc = sp.c()
    am = None if adam_m is None else _c(adam_m, np.float64)
    av = None if adam_v is None else _c(adam_v, np.float64)
    base = [n, deg, _p(theta), _p(am), _p(av), ca, len(cams), regs["view"].shape[0],
            _p(regs["view"]), _p(regs["parent"]), _p(regs["label"]), _p(regs["stats"]), ncand,
            _p(cand), _p(count), _p(noise), C.byref(sc), _p(status), _p(nchild)]
    new_n = lib().orc_split(*base, 0, None, None, None)
    o_theta = np.zeros((new_n, P))
    o_m = np.zeros((new_n, P))
    o_v = np.zeros((new_n, P))
    lib().orc_split(*base, new_n, _p(o_theta), _p(o_m), _p(o_v))
    return dict(new_n=int(new_n), status=status, n_children=nchild, theta=o_theta, m=o_m, v=o_v)


# --------------------------------------------------------------------------- backward, Adam

def grad(theta, deg, cam, tgt_f32, sel=None, bg=(0.0, 0.0, 0.0), cfg: Config = Config(),
         loss_scale=None, return_mean2d=False):
    """dL/dtheta of the per-view mean L1 loss (complex-step derivative of the forward).
    With return_mean2d, also dL with respect to each selected Gaussian's projected 2D
    mean in pixel units, [n_sel][2]."""
    theta = _c(theta, np.float64)
    n, P = theta.shape
    W, H = int(cam["width"]), int(cam["height"])
    if loss_scale is None:
        loss_scale = 1.0 / (3.0 * W * H)
    sel = np.arange(n, dtype=np.int32) if sel is None else _c(sel, np.int32)
    out = np.zeros((sel.shape[0], P))
    tgt = _c(tgt_f32, np.float32)
    bg = _c(bg, np.float64)
    cc, cf = camera(cam), cfg.c()
    m2 = np.zeros((sel.shape[0], 2)) if return_mean2d else None
    lib().orc_grad(n, deg, _p(theta), C.byref(cc), C.byref(cf), _p(bg), _p(tgt), loss_scale,
                   sel.shape[0], _p(sel), _p(out), _p(m2) if return_mean2d else None)
    return (out, m2) if return_mean2d else out


def l1_loss(theta, deg, cam, tgt_f32, bg=(0.0, 0.0, 0.0), cfg: Config = Config()):
    """Mean L1 loss of one view, rendered in FP64."""
    pr = project(theta, deg, cam, cfg)
    r = render(pr, cam, bg, cfg)
    tgt = np.asarray(tgt_f32, np.float64).reshape(-1, 3)
    return float(np.abs(r["rgb"] - tgt).sum() / tgt.size)


ADAM_LR = (1.6e-4, 0.05, 0.005, 0.001, 0.0025, 0.0025 / 20.0)


def adam(theta, g, m, v, step, lr=ADAM_LR, b1=0.9, b2=0.999, eps=1e-15):
    """One bias-corrected Adam step, in place; one learning rate per parameter group."""
    n, P = theta.shape
    lr = _c(lr, np.float64)
    for a in (theta, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().orc_adam(n, P, _p(theta), _p(g), _p(m), _p(v), step, _p(lr), b1, b2, eps)


# --------------------------------------------------------------------------- pipeline

def plain_step(scene, cams, targets, k_cand=None, cand=None, sp: SplitParams = SplitParams(),
               cfg: Config = Config(), noise=None, bg=(0.0, 0.0, 0.0)):
    """The whole hot path on the CPU for a list of views, in the paper's order:
    project, render with the dominant map, error map, per-Gaussian statistics,
    candidate choice (top-k error mass), erosion, regions, split."""
    theta = theta_of(scene)
    deg = scene["sh_degree"]
    n = theta.shape[0]
    views = []
    count = np.zeros(n, np.int32)
    mass = np.zeros(n, np.float64)
    for v, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        pr = project(theta, deg, cam, cfg)
        rd = render(pr, cam, bg, cfg)
        img32 = rd["rgb"].astype(np.float32).reshape(H, W, 3)
        em = error_map(img32, targets[v], sp.tau_l1, sp.n_levels)
        gauss_stats(em["M"], rd["dominant"], em["E"], n, count, mass)
        views.append(dict(proj=pr, render=rd, img32=img32, err=em))
    if cand is None:
        cand = topk_mass(mass, k_cand)
    cand = np.ascontiguousarray(cand, np.int32)
    flag = np.zeros(n, np.uint8)
    flag[cand] = 1
    parts = []
    for v, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        em = views[v]["err"]
        Mero = erode(em["M"], W, H, sp.r_erode)
        rg = regions(v, W, H, Mero, em["B"], views[v]["render"]["dominant"], n, flag, targets[v],
                     sp.m_min)
        views[v]["Mero"] = Mero
        views[v]["labels"] = rg["labels"]
        parts.append(rg)
    regs = concat_regions(parts)
    if noise is None:
        noise = np.zeros((cand.shape[0], 2, 3))
    sp_out = split(theta, deg, cams, regs, cand, count, noise, sp)
    return dict(theta=theta, views=views, count=count, mass=mass, cand=cand, regions=regs,
                split=sp_out)


# --------------------------------------------------------------------------- densification (Eq. 2)

def densify_stat_ndc(mean2d_grad, width, height):
    """One view's contribution to the densification statistic of Sec. 3: the norm of
    dL/d(projected 2D mean) in normalised device coordinates (the pixel-space
    gradient times W/2 and H/2, the scaling the baselines' statistic is kept in)."""
    g = np.asarray(mean2d_grad, np.float64)
    return np.hypot(g[:, 0] * (0.5 * width), g[:, 1] * (0.5 * height))


def densify_select(accum_f32, visits_i32, logscale_f32, tau_g, tau_s):
    """Eq. 2 and the clone rule of Sec. 3, decided in float32 on the stored values:
    g_i = accum_i / visits_i (0 if never visited); split iff g_i >= tau_g and
    max(s_i) > tau_s, clone iff g_i >= tau_g and max(s_i) <= tau_s. The scale test
    compares max log s_i with ln(tau_s) rounded to float32 (exp is increasing).
    Returns (split ids, clone ids), ascending."""
    acc = np.asarray(accum_f32, np.float32)
    vis = np.asarray(visits_i32, np.int32)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(vis > 0, acc / vis.astype(np.float32), np.float32(0.0)).astype(np.float32)
    high = g >= np.float32(tau_g)
    large = np.asarray(logscale_f32, np.float32)[:, :3].max(1) > np.float32(math.log(tau_s))
    return (np.nonzero(high & large)[0].astype(np.int32),
            np.nonzero(high & ~large)[0].astype(np.int32))


def clone_rows(theta_new, n, split_status, cand, clone_ids):
    """Appends to the post-split population theta_new a copy of each clone id's kept
    row (kept rows are the non-candidates and RESET candidates, in id order)."""
    keep = np.ones(n, bool)
    keep[np.asarray(cand)] = np.asarray(split_status) == RESET
    new_row = np.cumsum(keep) - 1
    rows = new_row[np.asarray(clone_ids, np.int64)]
    return np.concatenate([theta_new, theta_new[rows]], 0)


# --------------------------------------------------------------------------- D-SSIM loss term

def ssim_window(radius=5, sigma=1.5):
    """The normalised 1-D Gaussian of the SSIM window (11 taps, sigma 1.5)."""
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    return w / w.sum()


def _window_sum(a, w):
    """Zero-padded 'same' sum of a [H, W] map under the separable window w."""
    from scipy.ndimage import correlate1d

    t = correlate1d(a, w, axis=1, mode="constant", cval=0.0)
    return correlate1d(t, w, axis=0, mode="constant", cval=0.0)


def ssim_channel(xc, yc, c1=0.01 ** 2, c2=0.03 ** 2):
    """SSIM map of one channel ([H, W] arrays) under the 11x11 Gaussian window with
    zero padding, and its partial derivatives with respect to the window sums of x,
    x^2 and xy: (S, dS/dm1, dS/dq11, dS/dq12)."""
    w = ssim_window()
    m1, m2 = _window_sum(xc, w), _window_sum(yc, w)
    q11, q22, q12 = _window_sum(xc * xc, w), _window_sum(yc * yc, w), _window_sum(xc * yc, w)
    A1 = 2 * m1 * m2 + c1
    A2 = 2 * (q12 - m1 * m2) + c2
    B1 = m1 * m1 + m2 * m2 + c1
    B2 = (q11 - m1 * m1) + (q22 - m2 * m2) + c2
    S = A1 * A2 / (B1 * B2)
    dS_dm1 = (2 * m2 * A2 - 2 * m2 * A1) / (B1 * B2) - S * (2 * m1 / B1 - 2 * m1 / B2)
    return S, dS_dm1, -S / B2, 2 * A1 / (B1 * B2)


def dssim_loss_grad(img, tgt, width, height, lam=0.2, return_scale=False):
    """The baselines' loss (1 - lam) mean|x - y| + lam (1 - SSIM) of one view in FP64:
    SSIM of each channel (ssim_channel), averaged over pixels and channels; its
    gradient with respect to the render x through the window sums (the window is
    symmetric, so the adjoint of a window sum is the same sum). Returns
    (mean L1, mean SSIM, dL/dx [P][3]); with return_scale also the sum of the
    magnitudes of the three window-sum terms of each gradient entry, which nearly
    cancel in smooth regions (the scale of a float32 computation's rounding)."""
    x = np.asarray(img, np.float64).reshape(height, width, 3)
    y = np.asarray(tgt, np.float64).reshape(height, width, 3)
    w = ssim_window()
    N = 3.0 * width * height
    grad = np.zeros_like(x)
    scale = np.zeros_like(x)
    s_total = 0.0
    for c in range(3):
        xc, yc = x[..., c], y[..., c]
        S, d_m1, d_q11, d_q12 = ssim_channel(xc, yc)
        s_total += S.sum()
        t1, t2, t3 = _window_sum(d_m1, w), 2 * xc * _window_sum(d_q11, w), yc * _window_sum(d_q12, w)
        grad[..., c] = -lam * (t1 + t2 + t3) / N + (1 - lam) * np.sign(xc - yc) / N
        scale[..., c] = lam * (np.abs(t1) + np.abs(t2) + np.abs(t3)) / N
    l1 = np.abs(x - y).sum() / N
    if return_scale:
        return l1, s_total / N, grad.reshape(-1, 3), scale.reshape(-1, 3)
    return l1, s_total / N, grad.reshape(-1, 3)
