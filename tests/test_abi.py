"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/connectit_gb.h declares; argument validation rejects bad
calls before anything reaches the device; the build is sm_103a-only."""
import ctypes
import os
import re

import pytest

import paper_2008_03909_gb300 as cc
from paper_2008_03909_gb300 import build as ccbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cc_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = ccbuild.build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(L, nm), nm
    # the Python binding wraps every declared function
    assert set(names) <= set(cc.exported_symbols())


def test_built_for_sm103a_only():
    # every translation unit and the link step name the one sm_103a target
    flags = ccbuild._flags()
    gens = [f for f in flags if f.startswith("-gencode")]
    assert gens == ["-gencode=arch=compute_103a,code=sm_103a"]
    assert ccbuild.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert not any(f.startswith(("-arch", "--gpu-architecture")) for f in flags)


@pytest.mark.gpu
def test_loaded_image_is_sm103():
    # the runtime reports which image it loaded for the library's kernels
    v = ctypes.c_int(0)
    assert cc.lib().cc_binary_version(ctypes.byref(v)) == 0
    assert v.value == 103


def test_status_strings_and_version():
    L = cc.lib()
    assert L.cc_status_str(0) == b"ok"
    assert b"sm_103a" in L.cc_version()


def _call_static(offsets, u64, edges, n, m, so=None, fo=None, labels=None):
    L = cc.lib()
    return L.cc_static(ctypes.c_void_p(offsets), u64, ctypes.c_void_p(edges), n, m,
                       ctypes.byref(so) if so is not None else None, ctypes.byref(fo) if fo is not None else None,
                       ctypes.c_void_p(labels), None)


def test_validation_rejects_before_any_device_work():
    # None of these reach a CUDA call, so they run without a GPU.
    assert _call_static(0, 0, 0, 10, 5, labels=1) == 1           # null offsets
    assert _call_static(8, 0, 0, 10, 5, labels=1) == 1           # null edges with m > 0
    assert _call_static(8, 0, 8, 10, 2**32, labels=1) == 1       # 32-bit offsets, m >= 2^32
    assert _call_static(8, 0, 8, 0xFFFFFFFF, 5, labels=1) == 1   # reserved n
    assert _call_static(8, 0, 8, 10, 5, labels=0) == 1           # null labels
    bad_k = cc.sample_opt("kout", k=0)
    assert _call_static(8, 0, 8, 10, 5, so=bad_k, labels=1) == 1
    bad_beta = cc.sample_opt("ldd", ldd_beta=0.0)
    assert _call_static(8, 0, 8, 10, 5, so=bad_beta, labels=1) == 1
    bad_freq = cc.sample_opt("kout", freq_samples=5000)
    assert _call_static(8, 0, 8, 10, 5, so=bad_freq, labels=1) == 1
    bad_fin = cc.finish_opt("uf_rem_cas")
    bad_fin.find = 7
    assert _call_static(8, 0, 8, 10, 5, fo=bad_fin, labels=1) == 1
    assert _call_static(6, 1, 8, 10, 5, labels=16) == 1           # uint64 offsets not 8-aligned
    assert _call_static(8, 0, 6, 10, 5, labels=16) == 1           # edges not 4-aligned
    assert _call_static(8, 0, 8, 10, 5, labels=18) == 1           # labels not 4-aligned
    res = cc.sample_opt()
    res.kout_rule = 3                                              # no such k-out rule
    assert _call_static(8, 0, 8, 10, 5, so=res, labels=1) == 1
    rem_compress = cc.finish_opt("uf_rem_cas", "compress")          # Rem's Compress excludes FindCompress
    assert _call_static(8, 0, 8, 10, 5, fo=rem_compress, labels=1) == 1
    for bad in (cc.FinishOpt(9, 0, 0, 0), cc.FinishOpt(0, 4, 0, 0), cc.FinishOpt(0, 0, 3, 0),
                cc.FinishOpt(0, 0, 0, 1),                      # Liu-Tarjan rules on a union-find kind
                cc.finish_opt("liu_tarjan", lt_rules=0),       # Connect without Alter
                cc.finish_opt("liu_tarjan", lt_rules=2 | 4),   # ExtendedConnect with RootUpdate
                cc.finish_opt("liu_tarjan", lt_rules=3),       # no such connect rule
                cc.finish_opt("liu_tarjan", lt_rules=32)):     # unknown bit
        assert _call_static(8, 0, 8, 10, 5, fo=bad, labels=1) == 1
    for name in cc.LT_VARIANTS:                               # the sixteen variants pass validation
        assert _call_static(8, 0, 8, 0, 0, fo=cc.finish_opt(name), labels=1) == 0


def test_empty_graph_is_a_no_op():
    assert _call_static(0, 0, 0, 0, 0) == 0


def test_incremental_rejects_non_root_based():
    L = cc.lib()
    h = ctypes.c_void_p(0)
    fo = cc.finish_opt("PUS")
    so = cc.sample_opt()
    # n = 0 keeps this off the device: the finish kind is checked first
    assert L.cc_incr_create(None, 0, None, 0, 0, ctypes.byref(so), ctypes.byref(fo), None, ctypes.byref(h)) == 6
    assert L.cc_incr_create(None, 0, None, 0, 0, ctypes.byref(so), None, None, None) == 1


def test_no_cpu_fallback():
    import torch
    off = torch.zeros(3, dtype=torch.int64)
    edg = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(TypeError):
        cc.cc_static(off, edg)
