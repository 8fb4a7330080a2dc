"""ctypes mirror of include/adpsplit.h: struct layouts, prototypes, status check.

Argument marshalling only; all computation happens in libadpsplit.so. Loading
fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadpsplit.so")

ADP_MAX_VIEWS = 32
ADP_KEEP, ADP_ADAPTIVE, ADP_FALLBACK, ADP_RESET = 0, 1, 2, 3
STATUS_NAMES = {0: "ADP_OK", 1: "ADP_ERR_INVALID_ARG", 2: "ADP_ERR_CAPACITY", 3: "ADP_ERR_CUDA",
                4: "ADP_ERR_TIMEOUT", 5: "ADP_ERR_NUMERIC"}

_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32


class AdpCamera(C.Structure):
    _fields_ = [("width", _i32), ("height", _i32), ("fx", C.c_float), ("fy", C.c_float),
                ("px", C.c_float), ("py", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3)]


class AdpParams(C.Structure):
    _fields_ = [("tau_l1", C.c_float), ("r_erode", _i32), ("m_min", _i32), ("n_levels", _i32),
                ("n_max", _i32), ("gamma_d", C.c_float), ("gamma_c", C.c_float),
                ("eps_t", C.c_float), ("eta", C.c_float), ("scale_floor", C.c_float),
                ("near_plane", C.c_float), ("low_pass", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("t_min", C.c_float), ("tile_w", _i32),
                ("tile_h", _i32), ("batch", _i32)]


class AdpGaussians(C.Structure):
    _fields_ = [("n", _i64), ("sh_degree", _i32), ("reserved", _i32), ("mean_logit", _vp),
                ("logscale", _vp), ("quat", _vp), ("sh", _vp), ("rows", _vp)]


class AdpProjected(C.Structure):
    _fields_ = [("xy_opacity_depth", _vp), ("conic", _vp), ("rgb", _vp), ("rect", _vp),
                ("tiles_touched", _vp)]


class AdpBins(C.Structure):
    _fields_ = [("capacity", _i64), ("inst_gauss", _vp), ("tile_range", _vp),
                ("n_instances", _vp)]


class AdpImage(C.Structure):
    _fields_ = [("rgb", _vp), ("T_final", _vp), ("n_contrib", _vp), ("last", _vp),
                ("dominant", _vp)]


class AdpErrorMaps(C.Structure):
    _fields_ = [("E", _vp), ("mask", _vp), ("minmax", _vp)]


class AdpRegions(C.Structure):
    _fields_ = [("capacity", _i64), ("view", _vp), ("parent", _vp), ("label", _vp),
                ("band", _vp), ("moments", _vp), ("stats", _vp), ("count", _vp),
                ("labels", _vp)]


class AdpConstants(C.Structure):
    _fields_ = [("version", _i32), ("max_views", _i32), ("tile_pixels", _i32),
                ("max_sh_degree", _i32), ("fov_clamp", C.c_float), ("sh_coef", C.c_float * 16),
                ("gram_schmidt_eps", C.c_double), ("topk_noalloc_max_n", _i64),
                ("default_spin_limit", _i64), ("defaults", AdpParams)]


P = C.POINTER
_PROTOS = {
    "adp_version": (_i32, []),
    "adp_default_params": (None, [P(AdpParams)]),
    "adp_get_constants": (None, [P(AdpConstants)]),
    "adp_set_spin_limit": (None, [_i64]),
    "adp_last_error_string": (C.c_char_p, []),
    "adp_project": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32, P(AdpParams),
                              P(AdpProjected), _vp]),
    "adp_bin_sort_workspace_size": (C.c_size_t, [_i64, _i32, _i64]),
    "adp_bin_sort": (C.c_int, [_i64, P(AdpProjected), P(AdpCamera), _i32, P(AdpParams),
                               P(AdpBins), _vp, C.c_size_t, _vp, _vp]),
    "adp_render": (C.c_int, [_i64, P(AdpProjected), P(AdpBins), P(AdpCamera), _i32,
                             P(C.c_float), P(AdpParams), P(AdpImage), _vp]),
    "adp_error_stats_workspace_size": (C.c_size_t, [_i32, P(AdpCamera)]),
    "adp_error_stats": (C.c_int, [_vp, _vp, _vp, _i64, P(AdpCamera), _i32, P(AdpParams),
                                  P(AdpErrorMaps), _vp, _vp, _vp]),
    "adp_select_topk_workspace_size": (C.c_size_t, [_i64]),
    "adp_select_topk": (C.c_int, [_vp, _i64, _i64, _vp, _vp, C.c_size_t, _vp, _vp]),
    "adp_select_topk_noalloc": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp]),
    "adp_error_regions_workspace_size": (C.c_size_t, [_i64, _i32, P(AdpCamera)]),
    "adp_error_regions": (C.c_int, [P(AdpErrorMaps), _vp, _vp, _i64, P(AdpCamera), _i32, _vp,
                                    _i64, P(AdpParams), P(AdpRegions), _vp, C.c_size_t, _vp,
                                    _vp]),
    "adp_split_workspace_size": (C.c_size_t, [_i64, _i64, _i64]),
    "adp_split_plan": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32, P(AdpRegions), _vp, _i64,
                                 _vp, P(AdpParams), _vp, _vp, _vp, P(_i64), _vp, C.c_size_t,
                                 _vp, _vp]),
    "adp_split_apply": (C.c_int, [P(AdpGaussians), P(AdpGaussians), P(AdpGaussians),
                                  P(AdpRegions), _vp, _i64, _vp, _vp, _vp, P(AdpParams),
                                  P(AdpGaussians), P(AdpGaussians), P(AdpGaussians), _vp,
                                  C.c_size_t, _vp]),
    "adp_split_apply_adam": (C.c_int, [P(AdpGaussians), P(AdpGaussians), P(AdpGaussians),
                                       P(AdpGaussians), P(AdpRegions), _vp, _i64, _vp, _vp, _vp,
                                       P(AdpParams), _i32, _vp, P(C.c_float), C.c_float,
                                       C.c_float, C.c_float, P(AdpGaussians), P(AdpGaussians),
                                       P(AdpGaussians), _vp, C.c_size_t, _vp]),
    "adp_split_plan_overlapped": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32, P(AdpRegions),
                                            _vp, _i64, _vp, P(AdpParams), _vp, _vp, _vp, _vp,
                                            C.c_size_t, _vp, _vp]),
    "adp_split_plan_statuses": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32, P(AdpRegions),
                                          _vp, _i64, _vp, P(AdpParams), _vp, _vp, _vp, _vp,
                                          C.c_size_t, _vp, _vp]),
    "adp_split_plan_proposals_overlapped": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32,
                                                      P(AdpRegions), _vp, _i64, _vp,
                                                      P(AdpParams), _vp, _vp, _vp, _vp,
                                                      C.c_size_t, _vp, _vp]),
    "adp_split_keep_overlapped": (C.c_int, [P(AdpGaussians), P(AdpGaussians),
                                                  P(AdpGaussians), P(AdpGaussians), P(AdpRegions),
                                                  _vp, _i64, _vp, _vp, _vp, P(AdpParams), _i32,
                                                  _vp, P(C.c_float), C.c_float, C.c_float,
                                                  C.c_float, P(AdpGaussians), P(AdpGaussians),
                                                  P(AdpGaussians), _vp, C.c_size_t, _vp]),
    "adp_split_append_overlapped": (C.c_int, [P(AdpGaussians), P(AdpGaussians),
                                                  P(AdpGaussians), P(AdpGaussians), P(AdpRegions),
                                                  _vp, _i64, _vp, _vp, _vp, P(AdpParams), _i32,
                                                  _vp, P(C.c_float), C.c_float, C.c_float,
                                                  C.c_float, P(AdpGaussians), P(AdpGaussians),
                                                  P(AdpGaussians), _vp, C.c_size_t, _vp]),
    "adp_render_backward_workspace_size": (C.c_size_t, [_i64, _i32]),
    "adp_render_backward": (C.c_int, [P(AdpGaussians), P(AdpProjected), P(AdpBins), P(AdpImage),
                                      _vp, _vp, P(AdpCamera), _i32, P(C.c_float), P(AdpParams),
                                      P(AdpGaussians), _vp, _vp, _vp, C.c_size_t, _vp]),
    "adp_train_step_batched_workspace_size": (C.c_size_t, [_i64, _i32, P(AdpCamera),
                                                           P(AdpParams), _i64]),
    "adp_train_step_batched": (C.c_int, [P(AdpGaussians), P(AdpCamera), _i32, _vp, P(C.c_float),
                                         P(AdpParams), P(AdpProjected), P(AdpBins), P(AdpImage),
                                         P(AdpErrorMaps), _vp, _vp, P(AdpGaussians), _vp, _vp,
                                         _vp, C.c_size_t, _vp, _vp]),
    "adp_densify_select_workspace_size": (C.c_size_t, [_i64]),
    "adp_densify_select": (C.c_int, [_vp, _vp, P(AdpGaussians), C.c_float, C.c_float, _vp, _vp,
                                     _vp, _vp, C.c_size_t, _vp, _vp]),
    "adp_split_clone": (C.c_int, [_i64, _i64, _i64, _vp, _vp, _i64, P(AdpGaussians),
                                  P(AdpGaussians), P(AdpGaussians), _vp, C.c_size_t, _vp, _vp]),
    "adp_dssim_workspace_size": (C.c_size_t, [_i32, P(AdpCamera)]),
    "adp_dssim_loss_grad": (C.c_int, [_vp, _vp, P(AdpCamera), _i32, C.c_float, P(AdpParams),
                                      _vp, _vp, _vp, C.c_size_t, _vp]),
    "adp_adam_step": (C.c_int, [P(AdpGaussians), P(AdpGaussians), P(AdpGaussians),
                                P(AdpGaussians), _i32, _vp, P(C.c_float), C.c_float, C.c_float,
                                C.c_float, _vp]),
    "adp_adam_step_rows": (C.c_int, [P(AdpGaussians), P(AdpGaussians), P(AdpGaussians),
                                     P(AdpGaussians), _vp, _i64, _i32, _vp, P(C.c_float),
                                     C.c_float, C.c_float, C.c_float, _vp]),
}

_lib = None


def lib():
    """The loaded C-ABI library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA extension first "
                "(python -m paper_2605_06876_b300.build or __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int, what: str):
    if rc != 0:
        msg = lib().adp_last_error_string().decode(errors="replace")
        raise RuntimeError(f"{what}: {STATUS_NAMES.get(rc, rc)}: {msg}")


def constants() -> AdpConstants:
    """The constants fixed inside the library (adp_get_constants)."""
    c = AdpConstants()
    lib().adp_get_constants(C.byref(c))
    return c


def default_params(**overrides) -> AdpParams:
    p = AdpParams()
    lib().adp_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def cameras(cams) -> C.Array:
    """Host array of AdpCamera from camera dicts (width, height, fx, fy, px, py, R, t)."""
    if len(cams) < 1 or len(cams) > ADP_MAX_VIEWS:
        raise ValueError(f"between 1 and {ADP_MAX_VIEWS} views")
    arr = (AdpCamera * len(cams))()
    for a, c in zip(arr, cams):
        a.width, a.height = int(c["width"]), int(c["height"])
        a.fx, a.fy, a.px, a.py = (float(c[k]) for k in ("fx", "fy", "px", "py"))
        for i in range(9):
            a.R[i] = float(c["R"][i])
        for i in range(3):
            a.t[i] = float(c["t"][i])
    return arr
