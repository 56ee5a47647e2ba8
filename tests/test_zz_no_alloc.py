"""The allocation-free IdentifyFrequent entry point, called through the C ABI,
gives the same L_max as the allocating entry point, on two calls in a row
(the shared scratch keeps the previous call's counts, so the second call
shows that each call clears what it uses).  This file is collected last so
that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2008_03909_gb300 as cc

pytestmark = pytest.mark.gpu


def _noalloc(labels: torch.Tensor, out: torch.Tensor) -> int:
    L = cc.lib()
    st = L.cc_identify_frequent_noalloc(ctypes.c_void_p(labels.data_ptr()), labels.numel(),
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return int(out.item()) & 0xFFFFFFFF


def _alloc(labels: torch.Tensor) -> int:
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    L = cc.lib()
    st = L.cc_identify_frequent(ctypes.c_void_p(labels.data_ptr()), labels.numel(), 0, 0,
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return int(out.item()) & 0xFFFFFFFF


def test_noalloc_matches_allocating_entry_point_twice():
    rng = np.random.default_rng(11)
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    # first call: a large frequent label; second call: fewer, different labels,
    # so counts left over from the first call would change the answer
    n1 = 3_000_000
    a = rng.integers(0, n1, size=n1).astype(np.uint32)
    a[: n1 // 4] = 777_777
    n2 = 1_000_003
    b = rng.integers(0, 5000, size=n2).astype(np.uint32)
    b[:40_000] = 123
    for arr in (a, b):
        t = torch.from_numpy(arr.view(np.int32)).cuda()
        got = _noalloc(t, out)
        want = _alloc(t)
        assert got == want
        assert got == int(np.argmax(np.bincount(arr, minlength=arr.size)))
    assert cc.device_error() == 0


def test_noalloc_edges_of_the_range():
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    # n == 0: nothing to count, the documented "none" result
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    L = cc.lib()
    st = L.cc_identify_frequent_noalloc(None, 0, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(out.item()) & 0xFFFFFFFF == 0xFFFFFFFF
    del empty
    # n == the maximum: the whole scratch array in use, twice in a row with
    # different frequent labels at opposite ends of the id range
    n = cc.NOALLOC_MAX_LABELS
    rng = np.random.default_rng(5)
    for hot in (n - 1, 0):
        arr = rng.integers(0, n, size=n).astype(np.uint32)
        arr[: 1000] = hot
        t = torch.from_numpy(arr.view(np.int32)).cuda()
        got = _noalloc(t, out)
        assert got == _alloc(t) == int(np.argmax(np.bincount(arr, minlength=n))) == hot
    assert cc.device_error() == 0


def test_noalloc_rejects_sizes_over_the_limit():
    L = cc.lib()
    # n above the maximum is refused before any device work (no pointer is read)
    st = L.cc_identify_frequent_noalloc(ctypes.c_void_p(16), cc.NOALLOC_MAX_LABELS + 1, ctypes.c_void_p(16), None)
    assert st == 1
