"""The allocation-free top-k entry point, for callers that cannot allocate device
memory where they run (inside an allocator or memory-pool callback, under a host
framework that forbids allocation mid-step, or in a layer without an allocator).

It is checked through the C ABI against adp_select_topk, which takes a caller
workspace: the selected ids must be identical, on two consecutive calls that share
the static scratch (the second reuses what the first left behind). This file is
collected last so a run that stops at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_06876_b300 import _abi


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    L = _abi.lib()
    n = (1 << 22) + 1
    rc = L.adp_select_topk_noalloc(None, n, 5, None, None, None)
    assert rc == 1
    assert b"exceeds" in L.adp_last_error_string()


@pytest.mark.gpu
def test_noalloc_topk_matches_workspace_topk_on_two_calls():
    import torch

    L = _abi.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(17)
    cases = []
    for n, k in ((300_000, 12_345), (1 << 22, 200_000)):  # second call: the maximum size
        mass = np.floor(rng.exponential(2.0, n) * 16) / 16  # many exact ties
        mass[rng.uniform(size=n) < 0.4] = 0.0
        cases.append((n, k, mass))
    for n, k, mass in cases:
        m = torch.as_tensor(mass, device="cuda")
        ws_bytes = L.adp_select_topk_workspace_size(n)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        ref = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        got = torch.full((k,), -2, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert L.adp_select_topk(_ptr(m), n, k, _ptr(ref), _ptr(ws), ws_bytes, _ptr(status),
                                 stream) == 0
        assert L.adp_select_topk_noalloc(_ptr(m), n, k, _ptr(got), _ptr(status), stream) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0  # no bounded wait gave up
        assert torch.equal(got, ref)
        # the ids are the k largest masses, ties to the lower id, ascending
        order = np.lexsort((np.arange(n), -mass))[:k]
        assert np.array_equal(got.cpu().numpy(), np.sort(order).astype(np.int32))
