"""The densification loop on a synthetic scene (Sec. 3 with AdpSplit as the split
operator, against the vanilla split): both fit the scene, both densify, and the
vanilla run splits every candidate in two while AdpSplit initialises children from
error regions."""
import pytest

import scenes
from gpu_util import DEV
from paper_2605_06876_b300 import ops, train

pytestmark = pytest.mark.gpu


def test_densification_loop_vanilla_and_adpsplit():
    gt_sc = scenes.scene_clusters(80, 40000, 3)
    gt = ops.Gaussians.from_scene(gt_sc, DEV)
    init = ops.Gaussians.from_scene(scenes.scene_initial_points(gt_sc, 0.05, 81), DEV)
    tr = scenes.ring_cameras(82, 16, 14.0, 320, 208)
    te = scenes.ring_cameras(83, 3, 14.0, 320, 208)
    res = train.compare(gt, init, tr, te, iters=800, densify_until=400)
    for mode in ("vanilla", "adpsplit"):
        st = res[mode]
        assert st["test_psnr"] > res["initial_psnr"] + 5.0, (mode, st, res["initial_psnr"])
        assert st["final_gaussians"] > init.n
        assert st["split_candidates"] > 0
        counts = st["population_after_each_densification"]
        assert len(counts) == 4 and all(b >= a for a, b in zip(counts, counts[1:]))
    ss = res["vanilla"]["split_status"]
    assert ss["adaptive"] == 0 and ss["reset"] == 0 and ss["fallback"] == res["vanilla"]["split_candidates"]
    sa = res["adpsplit"]["split_status"]
    assert sa["adaptive"] > 0 and sa["children"] >= sa["adaptive"]
