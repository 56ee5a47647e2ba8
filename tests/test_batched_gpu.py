"""Parity of the batched launch (many packed graphs in one persistent
kernel) with the oracle, graph by graph and bit for bit, for every schedule
the autotuner may pick, including empty, single-vertex and large graphs
that do not fit the shared-memory threshold."""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu


def batch_with_edge_cases(count, seed):
    gs = synth.batch_config3(count, seed=seed, lo=4, hi=14)
    gs.insert(3, synth.empty(0))
    gs.insert(5, synth.empty(1))
    gs.insert(7, synth.counterexample())
    gs.append(synth.rmat(15, 4, seed=seed))          # larger than every shared-memory threshold but two
    gs.append(synth.grid2d(256, 256, 0.1, seed=seed))  # exactly 65536 vertices: the largest 16-bit local id
    gs.append(synth.rmat(17, 2, seed=seed))          # above 65536: global parents under every schedule
    gs.append(synth.grid2d(260, 240, 0.3, seed=seed))
    return gs


def expected(gs):
    return np.concatenate([oracle.cc_uf(*g.numpy())[0] if g.n else np.zeros(0, np.uint32) for g in gs])


@pytest.fixture(scope="module")
def batch():
    gs = batch_with_edge_cases(120, seed=4)
    gv, off, edg = synth.pack(gs)
    return gs, gv.cuda(), off.cuda(), edg.cuda(), expected(gs)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("threads", [128, 256, 1024])
@pytest.mark.parametrize("smem", [0, 4096, 57344, 65536])
def test_batched_schedules(batch, mode, threads, smem):
    gs, gv, off, edg, want = batch
    lab = cc.cc_batched(gv, off, edg, cc.batch_opt(threads, smem, mode))
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
    assert cc.device_error() == 0


@pytest.mark.parametrize("smem", [0, 28672, 57344])
def test_batched_two_ctas_per_sm(batch, smem):
    # mode 3: the tile walk at two 1024-thread CTAs per SM (1024 threads only)
    gs, gv, off, edg, want = batch
    lab = cc.cc_batched(gv, off, edg, cc.batch_opt(1024, smem, 3))
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
    with pytest.raises(cc.CCError):
        cc.cc_batched(gv, off, edg, cc.batch_opt(512, smem, 3))
    assert cc.device_error() == 0


def test_batched_u32_offsets_and_autotune(batch):
    gs, gv, off, edg, want = batch
    lab, best, ms = cc.cc_batched_autotune(gv, off.to(torch.int32), edg)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
    assert best.threads in (128, 256, 512, 1024) and ms > 0
    lab2 = cc.cc_batched(gv, off.to(torch.int32), edg, best)
    assert torch.equal(lab, lab2)


def test_batched_equals_per_graph_static(batch):
    gs, gv, off, edg, want = batch
    for i in (0, 7, len(gs) - 1):
        g = gs[i]
        if g.n == 0:
            continue
        b, e = int(gv[i]), int(gv[i + 1])
        lab = cc.cc_static(off[b:e + 1].contiguous(), edg, cc.sample_opt("none"))
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want[b:e])


def test_batched_bad_local_ids_flagged():
    gs = [synth.path(10), synth.path(5)]
    gv, off, edg = synth.pack(gs)
    edg = edg.clone()
    edg[3] = 50  # graph 0 has only 10 vertices
    cc.cc_batched(gv.cuda(), off.cuda(), edg.cuda())
    assert cc.device_error() & 1
