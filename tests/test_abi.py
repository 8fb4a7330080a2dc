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
               "adp_image", "adp_error_maps", "adp_regions"]
    mirror = {"adp_camera": abi.AdpCamera, "adp_params": abi.AdpParams,
              "adp_gaussians": abi.AdpGaussians, "adp_projected": abi.AdpProjected,
              "adp_bins": abi.AdpBins, "adp_image": abi.AdpImage,
              "adp_error_maps": abi.AdpErrorMaps, "adp_regions": abi.AdpRegions}
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
    assert abi.lib().adp_version() == 1


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
    """The overlapped plan and both compaction calls validate on the host first (no
    device, no auxiliary stream is touched): missing arrays, candidates without
    their status arrays, and an unaligned workspace."""
    L = abi.lib()
    cams = abi.cameras([{"width": 64, "height": 32, "fx": 50, "fy": 50, "px": 31.5, "py": 15.5,
                         "R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0]}])
    p = abi.default_params()
    g = abi.AdpGaussians(0, 0, 0, None, None, None, None)
    regs = abi.AdpRegions()
    rc = L.adp_split_plan_overlapped(C.byref(g), cams, 1, C.byref(regs), None, 0, None,
                                     C.byref(p), None, None, None, None, 0, None)
    assert rc == 1 and b"NULL" in L.adp_last_error_string()
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
                                     C.cast(C.pointer(cnt), C.c_void_p), unaligned, 4000, None)
    assert rc == 1 and b"aligned" in L.adp_last_error_string()
