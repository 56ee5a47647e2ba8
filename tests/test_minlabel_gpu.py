"""Parity of the min-label finishes that need not be monotone (the sixteen
Liu-Tarjan variants, Stergiou et al.'s algorithm, label propagation) with
the oracle's union-find labels, bit for bit, alone and composed with every
sampling method (the frequent cluster ranked first, Section 3.3), plus the
calls that refuse them."""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

SAMPLES = ["none", "kout", "bfs", "ldd"]
KINDS = sorted(cc.LT_VARIANTS) + ["stergiou", "label_prop"]


def graphs():
    return [synth.rmat(12, 8, seed=3), synth.grid2d(61, 47, 0.3, seed=2), synth.erdos_renyi(20011, 1.2, seed=4),
            synth.cliques([1, 5, 40, 3, 300, 2]), synth.star(5000, centre=4321), synth.path(3001),
            synth.counterexample(), synth.empty(1), synth.empty(77)]


@pytest.fixture(scope="module")
def small():
    return [(g, oracle.cc_uf(*g.numpy())[0]) for g in graphs()]


def labels(g, sample, kind, u64=True, **kw):
    off = (g.offsets if u64 else g.offsets_u32()).cuda()
    lab, st = cc.cc_static(off, g.edges.cuda(), cc.sample_opt(sample, **kw), cc.finish_opt(kind), stats=True)
    return lab.cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sample", SAMPLES)
def test_small_graphs(small, sample, kind):
    for g, want in small:
        got, st = labels(g, sample, kind, seed=5)
        assert np.array_equal(got, want), (g.name, sample, kind)
        # the round loop ran (label propagation's first frontier is empty
        # when sampling already covered every vertex with edges)
        if g.m and (kind != "label_prop" or sample == "none"):
            assert st["rounds"] >= 1, "the min-label rounds did not run"
    assert cc.device_error() == 0


@pytest.mark.parametrize("kind", ["PUS", "PRS", "CUSA", "CRFA", "EUS", "EUFA", "stergiou", "label_prop"])
@pytest.mark.parametrize("sample", ["none", "kout", "ldd"])
def test_medium_graphs(sample, kind):
    """RMAT-17 / a 500x400 grid / ER-2^18: many tiles, hubs split into warp
    chunks, a frequent cluster that is not vertex 0's (R-MAT relabelled)."""
    rng = np.random.default_rng(3)
    base = synth.rmat(17, 16, seed=2)
    perm = torch.from_numpy(rng.permutation(base.n).astype(np.int64))
    for g in (synth.relabel(base, perm), synth.grid2d(500, 400, 0.3, seed=1), synth.erdos_renyi(1 << 18, 1.3, seed=6)):
        want, _ = oracle.cc_uf(*g.numpy())
        got, st = labels(g, sample, kind, u64=False, seed=9)
        assert np.array_equal(got, want), (g.name, sample, kind)
        if sample != "none":
            assert st["lmax"] != 0xFFFFFFFF
    assert cc.device_error() == 0


def test_label_propagation_on_long_paths():
    # label 0 must cross the whole path; a round moves it at least one hop
    # (more when a neighbour is processed later in the same round)
    for n in (2000, 100001):
        g = synth.path(n)
        got, st = labels(g, "none", "label_prop")
        assert (got == 0).all()
        assert 1 <= st["rounds"] <= n


def test_refused_where_not_root_based():
    g = synth.rmat(10, 8, seed=1)
    off, edg = g.offsets.cuda(), g.edges.cuda()
    for kind in ("PUS", "stergiou", "label_prop"):
        with pytest.raises(cc.CCError) as e:
            cc.cc_spanning_forest(off, edg, finish=cc.finish_opt(kind))
        assert e.value.status == 6
        with pytest.raises(cc.CCError) as e:
            cc.Incremental(g.n, off, edg, finish=cc.finish_opt(kind))
        assert e.value.status == 6
