"""B300-native (sm_103a) implementation of the AdpSplit hot path.

The compute lives in libadpsplit.so (hand-written CUDA behind a C ABI declared in
include/adpsplit.h); this package only marshals torch tensors into its calls.
"""
from . import _abi  # noqa: F401
from .ops import (  # noqa: F401
    Bins,
    ErrorMaps,
    Gaussians,
    Image,
    Projected,
    Regions,
    adam_step,
    bin_sort,
    error_regions,
    error_stats,
    n_pixels,
    n_tiles,
    project,
    render,
    render_backward,
    select_topk,
    split_apply,
    split_plan,
)

__version__ = "0.1.0"
