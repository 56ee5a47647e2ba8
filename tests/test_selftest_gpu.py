"""The bounded grid barrier (used by the persistent BFS levels) ends a wait
that cannot complete: a block that never arrives makes the others give up
after the limit, the call reports CC_ERR_NONCONVERGED, and the context
keeps working.  No fault, trap or endless loop is involved."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu


def test_all_blocks_pass():
    st, passed = cc.selftest_grid_barrier(-1, 200)
    assert st == 0
    assert passed == torch.cuda.get_device_properties(0).multi_processor_count


def test_missing_block_times_out_and_context_survives():
    t0 = time.perf_counter()
    st, passed = cc.selftest_grid_barrier(0, 200)
    elapsed = time.perf_counter() - t0
    assert st == 4 and passed == 0          # CC_ERR_NONCONVERGED, nobody got through
    assert elapsed < 3.0
    assert cc.device_error() == 0           # the call already read and cleared the word
    g = synth.rmat(12, 8, seed=1)
    lab = cc.cc_static(g.offsets.cuda(), g.edges.cuda(), cc.sample_opt("bfs"))
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.cc_uf(*g.numpy())[0])


def test_rejects_bad_limits():
    assert cc.selftest_grid_barrier(-1, 0)[0] == 1
    assert cc.selftest_grid_barrier(-1, 5000)[0] == 1
