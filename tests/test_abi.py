"""The C-ABI library loads and exports every symbol include/adpsplit.h declares, the
ctypes mirror matches the header's struct layouts, and host-only queries work.
No GPU work is done here."""
import ctypes as C
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adpsplit.h")


@pytest.fixture(scope="module")
def abi():
    from paper_2605_06876_b300 import build

    build.build()
    from paper_2605_06876_b300 import _abi

    _abi.lib()
    return _abi


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"ADP_API\s+[\w\s\*]+?\b(adp_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(abi):
    names = _declared()
    assert len(names) >= 19
    lib = C.CDLL(abi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(abi._PROTOS), "ctypes prototypes and header disagree"


def test_struct_layouts_match_header(abi, tmp_path):
    structs = ["adp_camera", "adp_params", "adp_gaussians", "adp_projected", "adp_bins",
               "adp_image", "adp_error_maps", "adp_regions", "adp_constants"]
    mirror = {"adp_camera": abi.AdpCamera, "adp_params": abi.AdpParams,
              "adp_gaussians": abi.AdpGaussians, "adp_projected": abi.AdpProjected,
              "adp_bins": abi.AdpBins, "adp_image": abi.AdpImage,
              "adp_error_maps": abi.AdpErrorMaps, "adp_regions": abi.AdpRegions,
              "adp_constants": abi.AdpConstants}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "adpsplit.h"', 'int main(void){']
    for s in structs:
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in mirror[s]._fields_:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        s, f, v = line.split()
        if f == "size":
            assert C.sizeof(mirror[s]) == int(v), s
        else:
            assert getattr(mirror[s], f).offset == int(v), (s, f)


def test_default_params_are_the_papers(abi):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))
    p = abi.default_params()
    for k in ("r_erode", "m_min", "n_levels", "n_max"):
        assert getattr(p, k) == g[k], k
    for k in ("tau_l1", "gamma_d", "gamma_c"):
        assert abs(getattr(p, k) - g[k]) < 1e-7, k
    assert p.tile_w * p.tile_h == 256
    assert abi.lib().adp_version() == 2


def test_workspace_queries_and_argument_errors(abi):
    L = abi.lib()
    a = L.adp_bin_sort_workspace_size(1000, 1, 10000)
    b = L.adp_bin_sort_workspace_size(1000, 2, 10000)
    assert 0 < a < b
    assert L.adp_bin_sort_workspace_size(-1, 1, 10) == 0
    assert L.adp_split_workspace_size(100, 10, 50) > 0
    cams = abi.cameras([{"width": 64, "height": 32, "fx": 50, "fy": 50, "px": 31.5, "py": 15.5,
                         "R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0]}])
    assert L.adp_error_regions_workspace_size(10, 1, cams) > 64 * 32 * 40
    # host-side validation rejects bad arguments before touching the GPU
    p = abi.default_params(tile_w=10)
    g = abi.AdpGaussians(10, 0, 0, None, None, None, None)
    out = abi.AdpProjected()
    rc = L.adp_project(C.byref(g), cams, 1, C.byref(p), C.byref(out), None)
    assert rc == 1 and b"256" in L.adp_last_error_string()
    p2 = abi.default_params()
    rc = L.adp_project(C.byref(g), cams, 0, C.byref(p2), C.byref(out), None)
    assert rc == 1 and b"n_views" in L.adp_last_error_string()


def test_overlapped_split_rejects_bad_arguments_before_any_launch(abi):
    """The overlapped plan (whole or in its two parts) and both compaction calls
    validate on the host first (no device, no auxiliary stream is touched): missing
    arrays, candidates without their status arrays, and an unaligned workspace."""
    L = abi.lib()
    cams = abi.cameras([{"width": 64, "height": 32, "fx": 50, "fy": 50, "px": 31.5, "py": 15.5,
                         "R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0]}])
    p = abi.default_params()
    g = abi.AdpGaussians(0, 0, 0, None, None, None, None)
    regs = abi.AdpRegions()
    for name in ("adp_split_plan_overlapped", "adp_split_plan_statuses",
                 "adp_split_plan_proposals_overlapped"):
        rc = getattr(L, name)(C.byref(g), cams, 1, C.byref(regs), None, 0, None, C.byref(p),
                              None, None, None, None, 0, None, None)
        assert rc == 1 and b"NULL" in L.adp_last_error_string(), name
    lr = (C.c_float * 6)(*([1e-3] * 6))
    for name in ("adp_split_keep_overlapped", "adp_split_append_overlapped"):
        fn = getattr(L, name)
        rc = fn(C.byref(g), C.byref(g), C.byref(g), C.byref(g), C.byref(regs), None, 5, None,
                None, None, C.byref(p), 1, None, lr, 0.9, 0.999, 1e-15, None, None, None,
                None, 0, None)
        assert rc == 1, name
    ws = C.create_string_buffer(4096)
    unaligned = C.c_void_p(((C.addressof(ws) + 255) & ~255) + 8)  # 8 past a 256-byte boundary
    cnt = C.c_int64(0)
    regs2 = abi.AdpRegions()
    regs2.count = C.cast(C.pointer(cnt), C.c_void_p)
    rc = L.adp_split_plan_overlapped(C.byref(g), cams, 1, C.byref(regs2), None, 0,
                                     C.cast(C.pointer(cnt), C.c_void_p), C.byref(p), None, None,
                                     C.cast(C.pointer(cnt), C.c_void_p), unaligned, 4000, None,
                                     None)
    assert rc == 1 and b"aligned" in L.adp_last_error_string()


def test_constants_match_the_oracles(abi):
    """The constants the kernels hard-code (adp_get_constants) against the oracle's
    own: the forward conventions and split defaults of its Config and SplitParams,
    and the real SH basis, whose coefficients are read off the oracle's basis
    values at a random direction (Y_k / m_k for the header's monomials m_k)."""
    import numpy as np

    import oracle as O

    c = abi.constants()
    assert c.version == abi.lib().adp_version() == 2
    assert c.max_views == abi.ADP_MAX_VIEWS and c.tile_pixels == 256 and c.max_sh_degree == 3
    assert c.topk_noalloc_max_n == 1 << 22 and c.default_spin_limit > 0
    cfg, sp = O.Config(), O.SplitParams()
    d = c.defaults
    for k in ("near_plane", "low_pass", "alpha_min", "alpha_max", "t_min"):
        assert abs(getattr(d, k) - getattr(cfg, k)) <= 1e-7 * abs(getattr(cfg, k)), k
    for k in ("tau_l1", "gamma_d", "gamma_c", "eps_t", "eta", "scale_floor"):
        assert abs(getattr(d, k) - getattr(sp, k)) <= 1e-7 * abs(getattr(sp, k)), k
    for k in ("r_erode", "m_min", "n_levels", "n_max"):
        assert getattr(d, k) == getattr(sp, k), k
    assert (d.tile_w, d.tile_h) == (cfg.tile_w, cfg.tile_h)
    rng = np.random.default_rng(5)
    v = rng.normal(size=3)
    x, y, z = v / np.linalg.norm(v)
    mono = [1, y, z, x, x * y, y * z, 2 * z * z - x * x - y * y, x * z, x * x - y * y,
            y * (3 * x * x - y * y), x * y * z, y * (4 * z * z - x * x - y * y),
            z * (2 * z * z - 3 * x * x - 3 * y * y), x * (4 * z * z - x * x - y * y),
            z * (x * x - y * y), x * (x * x - 3 * y * y)]
    Y = O.sh_basis(3, np.array([[x, y, z]]))[0]
    want = Y / np.array(mono)
    got = np.array(list(c.sh_coef), np.float64)
    np.testing.assert_allclose(got, want, rtol=1e-7)
    assert abs(c.fov_clamp - 1.3) < 1e-7
    assert c.gram_schmidt_eps == 1e-12
