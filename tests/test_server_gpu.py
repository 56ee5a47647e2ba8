"""The continuous-batching request loop: every request's answers equal the
oracle replaying the requests one by one in ticket order, whether requests
are submitted one at a time, all at once, or from several threads, and with
slots small enough that large requests are split into chunks."""
import threading

import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

SCALE = 14


def make_requests(n, count, seed):
    reqs = []
    sizes = synth.log_uniform_sizes(count, 1, 30000, seed, 600)
    for i, sz in enumerate(sizes):
        qf = (0.1, 0.5, 0.9, 0.0, 1.0)[i % 5]
        nq = int(sz * qf)
        ni = sz - nq
        ins = (synth.rmat_pairs(SCALE, ni, seed=seed * 1000 + i, stream=610) % n).reshape(-1).contiguous()
        qs = synth.random_pairs(n, nq, seed=seed * 1000 + i, stream=620).reshape(-1).contiguous()
        reqs.append((ins.pin_memory(), qs.pin_memory()))
    return reqs


def oracle_replay(base, reqs):
    inc = oracle.Incremental(*base.numpy())
    out = []
    for ins, qs in reqs:
        inc.insert(ins.numpy())
        out.append(inc.query(qs.numpy()))
    return out, inc.labels()


def new_server(base, slots, slot_pairs, stage=False):
    inc = cc.Incremental(base.n, base.offsets.cuda(), base.edges.cuda())
    return inc, cc.Server(inc, slots=slots, slot_pairs=slot_pairs, stage=stage)


@pytest.fixture(scope="module")
def setup():
    base = synth.rmat(SCALE, 4, seed=5)
    reqs = make_requests(base.n, 40, seed=3)
    want, want_labels = oracle_replay(base, reqs)
    return base, reqs, want, want_labels


@pytest.mark.parametrize("stage", [False, True])
@pytest.mark.parametrize("slots,slot_pairs", [(1, 1 << 20), (3, 4096), (8, 777)])
def test_all_at_once_matches_oracle(setup, slots, slot_pairs, stage):
    base, reqs, want, want_labels = setup
    inc, srv = new_server(base, slots, slot_pairs, stage)
    tickets = [srv.submit(i, q) for i, q in reqs]
    for t, w in zip(tickets, want):
        ans, lat = srv.wait(t)
        assert np.array_equal(ans.numpy(), w) and lat >= 0
    srv.close()
    assert np.array_equal(inc.labels().cpu().numpy().view(np.uint32), want_labels)
    inc.close()
    assert cc.device_error() == 0


@pytest.mark.parametrize("slots,slot_pairs", [(2, 3000), (4, 1 << 20)])
def test_pageable_requests_are_staged(setup, slots, slot_pairs):
    """Pageable host buffers take the staged path (copies through device
    slots, large requests split into chunks); answers are the same."""
    base, reqs, want, want_labels = setup
    inc, srv = new_server(base, slots, slot_pairs)
    pageable = [(i.clone(), q.clone()) for i, q in reqs]
    outs = [torch.empty(max(1, q.numel() // 2), dtype=torch.uint8) for _, q in pageable]
    tickets = [srv.submit(i, q, a) for (i, q), a in zip(pageable, outs)]
    for t, w, a in zip(tickets, want, outs):
        srv.wait(t)
        assert np.array_equal(a[: w.size].numpy(), w)
    srv.close()
    assert np.array_equal(inc.labels().cpu().numpy().view(np.uint32), want_labels)
    inc.close()


def test_alone_equals_in_the_mix(setup):
    base, reqs, want, _ = setup
    inc, srv = new_server(base, 2, 5000)
    alone = []
    for i, q in reqs:
        ans, _ = srv.wait(srv.submit(i, q))
        alone.append(ans.clone())
    srv.close()
    inc.close()
    inc, srv = new_server(base, 4, 5000)
    tickets = [srv.submit(i, q) for i, q in reqs]
    mixed = [srv.wait(t)[0] for t in tickets]
    srv.close()
    inc.close()
    for a, b, w in zip(alone, mixed, want):
        assert torch.equal(a, b) and np.array_equal(a.numpy(), w)


def test_concurrent_submitters_follow_ticket_order(setup):
    base, reqs, _, _ = setup
    inc, srv = new_server(base, 4, 8192)
    got = {}
    lock = threading.Lock()

    def client(part):
        for idx in part:
            t = srv.submit(*reqs[idx])
            with lock:
                got[t] = idx

    parts = [list(range(k, len(reqs), 3)) for k in range(3)]
    th = [threading.Thread(target=client, args=(p,)) for p in parts]
    for x in th:
        x.start()
    for x in th:
        x.join()
    order = [got[t] for t in sorted(got)]
    want, _ = oracle_replay(base, [reqs[i] for i in order])
    for t, w in zip(sorted(got), want):
        ans, _ = srv.wait(t)
        assert np.array_equal(ans.numpy(), w)
    srv.close()
    inc.close()
