"""Approximate minimum spanning forest on the GPU (Section 5.1): every mode
(NF, NF-S, COO) returns a spanning forest of G (the oracle's checker), the
oracle's labels, and a weight between the exact minimum (the oracle's
Kruskal) and (1 + eps) times it.  Which forest comes back depends on
thread timing; its size, span and weight bound do not."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

MODES = ("nf", "nf_s", "coo")
# float32 bucket bounds: the (1 + eps) ratio holds to about 1e-7 relative
SLACK = 1e-6


def graphs():
    return [synth.rmat(13, 8, seed=3), synth.grid2d(90, 70, 0.35, seed=2), synth.erdos_renyi(30011, 1.2, seed=4),
            synth.cliques([1, 5, 40, 3, 300, 2]), synth.star(5000, centre=4321), synth.path(3001),
            synth.empty(1), synth.empty(77), synth.rmat(16, 16, seed=11)]


def run(g, w, eps, mode, u64=True):
    off = (g.offsets if u64 else g.offsets_u32()).cuda()
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pairs, wt, _ = cc.cc_amsf(off, g.edges.cuda(), w.cuda(), eps, mode, labels_out=lab)
    return pairs.cpu().numpy().view(np.uint32), wt, lab.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("eps", [0.25, 0.05, 2.0])
def test_forest_weight_within_bound(mode, eps):
    for i, g in enumerate(graphs()):
        off, edg = g.numpy()
        w = synth.edge_weights(g, 100 + i)
        want, links = oracle.cc_uf(off, edg)
        _, opt = oracle.msf_kruskal(off, edg, w.numpy())
        F, wt, lab = run(g, w, eps, mode, u64=i % 2 == 0)
        assert np.array_equal(lab, want), (g.name, mode)
        assert len(F) == links
        assert oracle.check_forest(off, edg, F, want) == 0, (g.name, mode)
        # the reported weight is the sum over the returned pairs
        ws = {(int(a), int(b)): float(x) for a, b, x in zip(np.repeat(np.arange(g.n), np.diff(off)), edg, w.numpy())}
        assert abs(sum(ws[(int(a), int(b))] for a, b in F) - wt) <= 1e-6 * max(wt, 1.0)
        assert opt * (1 - 1e-9) <= wt <= (1 + eps) * opt * (1 + SLACK), (g.name, mode, wt / max(opt, 1e-30))
    assert cc.device_error() == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("eps", [0.05, 0.5, 2.0])
def test_forest_edges_per_bucket(mode, eps):
    # Section 5.1's buckets are processed lightest first, so after bucket i
    # the forest spans the subgraph of buckets <= i: the returned forest's
    # edges in buckets <= i number exactly n - #components of that subgraph,
    # and the oracle's forest has the same counts
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle import forest_bucket_counts
    for i, g in enumerate((synth.rmat(12, 8, seed=3), synth.grid2d(60, 50, 0.35, seed=2),
                           synth.erdos_renyi(9001, 1.5, seed=4))):
        off, edg = g.numpy()
        w = synth.edge_weights(g, 200 + i)
        F, _, _ = run(g, w, eps, mode)
        got, rank = forest_bucket_counts(off, edg, w.numpy(), F, eps)
        Fo, _ = oracle.amsf(off, edg, w.numpy(), eps)
        want, _ = forest_bucket_counts(off, edg, w.numpy(), Fo, eps)
        assert np.array_equal(got, rank), (g.name, mode)
        assert np.array_equal(got, want), (g.name, mode)


def test_equal_weights_and_one_bucket():
    g = synth.rmat(14, 8, seed=5)
    off, edg = g.numpy()
    ones = torch.ones(g.m, dtype=torch.float32)
    for mode in MODES:
        F, wt, lab = run(g, ones, 0.25, mode)
        assert wt == len(F) == oracle.cc_uf(off, edg)[1]


def test_rejections():
    g = synth.rmat(10, 8, seed=1)
    off, edg = g.offsets.cuda(), g.edges.cuda()
    w = synth.edge_weights(g, 1).cuda()
    for eps in (0.0, 1e-4, 100.0):
        with pytest.raises(cc.CCError):
            cc.cc_amsf(off, edg, w, eps)
    with pytest.raises(cc.CCError):
        cc.cc_amsf(off, edg, w, 0.25, mode=3)
    # weights spanning more than 65536 buckets of ratio 1.001
    wide = w.clone()
    wide[0] = 1e-30
    wide[1] = 1e30
    with pytest.raises(cc.CCError):
        cc.cc_amsf(off, edg, wide, 1e-3)
    # a non-positive weight is skipped and flagged, not faulted
    bad = w.clone()
    bad[5] = -1.0
    cnt, wt = ctypes.c_uint64(0), ctypes.c_double(0)
    out = torch.empty(2 * g.n, dtype=torch.int32, device="cuda")
    st = cc.lib().cc_amsf(ctypes.c_void_p(off.data_ptr()), 1, ctypes.c_void_p(edg.data_ptr()),
                          ctypes.c_void_p(bad.data_ptr()), g.n, g.m, 0.25, 1, ctypes.c_void_p(out.data_ptr()),
                          ctypes.byref(cnt), ctypes.byref(wt), None, None)
    assert st == 5   # CC_ERR_BAD_INPUT from the device error word
    cc.device_error()
