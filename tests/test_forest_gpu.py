"""Spanning forest on the GPU: every sampling x root-based finish
combination returns a valid spanning forest of G (checked by the oracle's
checker: every pair an edge of G, no cycle, n - #components pairs, so the
trees span exactly G's components) and the canonical labels.  Which forest
comes back depends on thread timing, so the pairs themselves are not
compared with the oracle's forest; their count and span are unique."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

SAMPLES = ("none", "kout", "bfs", "ldd")
FINISHES = (("uf_rem_cas", "naive", "split_one"), ("uf_rem_cas", "split", "halve_one"),
            ("uf_async", "naive", "split_one"), ("uf_async", "halve", "split_one"),
            ("uf_async", "compress", "split_one"), ("uf_hooks", "naive", "split_one"),
            ("uf_hooks", "split", "split_one"), ("uf_early", "naive", "split_one"),
            ("uf_early", "compress", "split_one"))


def graphs():
    return [synth.rmat(13, 8, seed=3), synth.grid2d(90, 70, 0.35, seed=2), synth.erdos_renyi(30011, 1.2, seed=4),
            synth.cliques([1, 5, 40, 3, 300, 2]), synth.star(5000, centre=4321), synth.path(3001),
            synth.counterexample(), synth.empty(1), synth.empty(77), synth.rmat(16, 16, seed=11)]


def run_forest(g, s, fin, u64=True, **kw):
    off = g.offsets.cuda() if u64 else g.offsets_u32().cuda()
    edg = g.edges.cuda()
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pairs, _ = cc.cc_spanning_forest(off, edg, cc.sample_opt(s, **kw), cc.finish_opt(*fin), labels_out=lab)
    return pairs.cpu().numpy().view(np.uint32), lab.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("s", SAMPLES)
def test_every_combination_gives_a_spanning_forest(s):
    for g in graphs():
        off, edg = g.numpy()
        want, links = oracle.cc_uf(off, edg)
        for fin in FINISHES:
            F, lab = run_forest(g, s, fin)
            assert np.array_equal(lab, want), (g.name, s, fin)
            assert len(F) == links == g.n - int((want == np.arange(g.n)).sum())
            code = oracle.check_forest(off, edg, F, want)
            assert code == 0, (g.name, s, fin, oracle.FOREST_CHECK[code])
    assert cc.device_error() == 0


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("rule", ["hybrid", "afforest", "pure"])
def test_kout_forest_u32_offsets_and_seeds(k, rule):
    g = synth.rmat(15, 8, seed=2)
    off, edg = g.numpy()
    want, links = oracle.cc_uf(off, edg)
    for seed in (1, 7, 99):
        F, lab = run_forest(g, "kout", FINISHES[0], u64=False, k=k, seed=seed, kout_rule=rule)
        assert np.array_equal(lab, want) and len(F) == links
        assert oracle.check_forest(off, edg, F, want) == 0


def test_ldd_and_bfs_forest_high_diameter():
    # BFS levels in the persistent launch, LDD with many search steps
    for g in (synth.grid2d(400, 300, 0.0), synth.grid2d(300, 300, 0.45, seed=8), synth.path(70001)):
        off, edg = g.numpy()
        want, links = oracle.cc_uf(off, edg)
        for s, kw in (("bfs", {}), ("ldd", {"ldd_beta": 0.05}), ("ldd", {"ldd_beta": 2.0})):
            F, lab = run_forest(g, s, FINISHES[0], **kw)
            assert np.array_equal(lab, want) and len(F) == links, (g.name, s, kw)
            assert oracle.check_forest(off, edg, F, want) == 0


def test_forest_without_labels_and_rejections():
    g = synth.rmat(12, 8, seed=5)
    off, edg = g.offsets.cuda(), g.edges.cuda()
    pairs, lab = cc.cc_spanning_forest(off, edg)
    assert lab is None
    assert oracle.check_forest(*g.numpy(), pairs.cpu().numpy().view(np.uint32)) == 0
    for fo in (cc.finish_opt("sv"), cc.finish_opt("lt_prf"), cc.finish_opt("uf_rem_cas", "naive", "atomic")):
        with pytest.raises(cc.CCError) as e:
            cc.cc_spanning_forest(off, edg, finish=fo)
        assert e.value.status == 6
    L = cc.lib()
    cnt = ctypes.c_uint64(5)
    so, fo = cc.sample_opt(), cc.finish_opt()
    # null forest, unaligned forest: rejected before device work
    assert L.cc_spanning_forest(ctypes.c_void_p(off.data_ptr()), 1, ctypes.c_void_p(edg.data_ptr()), g.n, g.m,
                                ctypes.byref(so), ctypes.byref(fo), ctypes.c_void_p(0), ctypes.byref(cnt), None,
                                None) == 1
    buf = torch.empty(2 * g.n + 1, dtype=torch.int32, device="cuda")
    assert L.cc_spanning_forest(ctypes.c_void_p(off.data_ptr()), 1, ctypes.c_void_p(edg.data_ptr()), g.n, g.m,
                                ctypes.byref(so), ctypes.byref(fo), ctypes.c_void_p(buf.data_ptr() + 2),
                                ctypes.byref(cnt), None, None) == 1
    # empty graph: nothing to do, count 0
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.cc_spanning_forest(ctypes.c_void_p(z.data_ptr()), 1, None, 0, 0, None, None, None, ctypes.byref(cnt),
                                None, None) == 0 and cnt.value == 0
