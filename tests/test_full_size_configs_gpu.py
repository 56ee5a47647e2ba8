"""Parity at the full sizes of the batched and served workloads, against the
oracle graph by graph and answer by answer.

* Batched: the 10,000 packed graphs of the batched workload (vertex counts
  log-uniform in [2^6, 2^16], half G(n, M) with average degree in [0.5, 4],
  half grids with edge drop in [0, 0.5]), labelled in one launch with the
  autotuned schedule and with the default one; every graph's labels equal
  the oracle's sequential union-find (O1) on that graph.
* Served: an R-MAT scale-24 edge-factor-16 base graph loaded into a
  resident union-find, then 24 batches whose sizes run from 10^3 to 10^7
  operations at 10 / 50 / 90 % queries (inserts R-MAT distributed, queries
  uniform).  Every answer of every batch, and the labels after the last,
  equal the batch-incremental oracle (Section 3.5, Algorithm 3: a batch's
  inserts, then its queries), both through the plain handle and through the
  continuous-batching request loop.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch10k():
    gs = synth.batch_config3(10000, seed=1)
    gv, off, edg = synth.pack(gs)
    want = np.concatenate([oracle.cc_uf(*g.numpy())[0] for g in gs])
    return gs, gv, off, edg, want


def _first_bad(gv, got, want):
    bad = np.flatnonzero(got != want)
    if bad.size == 0:
        return None
    g = int(np.searchsorted(gv, bad[0], side="right") - 1)
    return g, int(bad[0]), int(got[bad[0]]), int(want[bad[0]])


@pytest.mark.parametrize("offsets", ["u32", "u64"])
def test_batched_10000_graphs_equal_oracle(batch10k, offsets):
    gs, gv, off, edg, want = batch10k
    assert len(gs) == 10000 and int(gv[-1]) == want.size
    o = off.to(torch.int32) if offsets == "u32" else off
    gvd, od, ed = gv.cuda(), o.cuda(), edg.cuda()
    lab, best, ms = cc.cc_batched_autotune(gvd, od, ed)
    got = lab.cpu().numpy().view(np.uint32)
    assert _first_bad(gv.numpy(), got, want) is None
    for opt in (best, None):
        lab2 = cc.cc_batched(gvd, od, ed, opt)
        assert _first_bad(gv.numpy(), lab2.cpu().numpy().view(np.uint32), want) is None
    assert cc.device_error() == 0


SERVE_SCALE = 24


def serve_batches(n):
    """24 batches, sizes log-spaced over [1e3, 1e7], query fractions cycling
    0.1 / 0.5 / 0.9; returns host int32 (inserts, queries) pairs."""
    sizes = np.round(np.logspace(3, 7, 24)).astype(np.int64)
    out = []
    for b, sz in enumerate(sizes):
        qf = (0.1, 0.5, 0.9)[b % 3]
        nq = int(round(int(sz) * qf))
        ni = int(sz) - nq
        ins = synth.rmat_pairs(SERVE_SCALE, ni, seed=900 + b, stream=60, device="cuda").reshape(-1).cpu()
        qs = synth.random_pairs(n, nq, seed=900 + b, stream=70, device="cuda").reshape(-1).cpu()
        out.append((ins.contiguous(), qs.contiguous()))
    return out


@pytest.fixture(scope="module")
def served():
    base = synth.rmat(SERVE_SCALE, 16, seed=2, device="cuda")
    n = base.n
    batches = serve_batches(n)
    assert batches[0][0].numel() // 2 + batches[0][1].numel() // 2 == 1000
    assert batches[-1][0].numel() // 2 + batches[-1][1].numel() // 2 == 10_000_000
    ref = oracle.Incremental(base.offsets.cpu().numpy(), base.edges.cpu().numpy())
    want = []
    for ins, qs in batches:
        ref.insert(ins.numpy())
        want.append(ref.query(qs.numpy()))
    return base, batches, want, ref.labels()


def test_served_workload_plain_handle_equals_oracle(served):
    base, batches, want, want_labels = served
    inc = cc.Incremental(base.n, base.offsets, base.edges)
    for b, ((ins, qs), w) in enumerate(zip(batches, want)):
        inc.insert(ins.cuda())
        ans = inc.query(qs.cuda()).cpu().numpy()
        assert np.array_equal(ans, w), b
    assert np.array_equal(inc.labels().cpu().numpy().view(np.uint32), want_labels)
    inc.close()
    assert cc.device_error() == 0


@pytest.mark.parametrize("pinned,stage", [(True, False), (True, True), (False, False)])
def test_served_workload_request_loop_equals_oracle(served, pinned, stage):
    base, batches, want, want_labels = served
    inc = cc.Incremental(base.n, base.offsets, base.edges)
    srv = cc.Server(inc, slots=4, slot_pairs=1 << 22, stage=stage)
    reqs = [(i.pin_memory(), q.pin_memory()) if pinned else (i, q) for i, q in batches]
    outs = [torch.empty(max(1, q.numel() // 2), dtype=torch.uint8) for _, q in reqs]
    if pinned:
        outs = [o.pin_memory() for o in outs]
    tickets = [srv.submit(i, q, a) for (i, q), a in zip(reqs, outs)]
    for b, (t, w, a) in enumerate(zip(tickets, want, outs)):
        srv.wait(t)
        assert np.array_equal(a[: w.size].numpy(), w), b
    srv.close()
    assert np.array_equal(inc.labels().cpu().numpy().view(np.uint32), want_labels)
    inc.close()
    assert cc.device_error() == 0
