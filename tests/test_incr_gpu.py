"""Parity of the batch-incremental path (resident union-find) with the
oracle: every query answer and the canonical labels after every batch, bit
for bit, for every union-find variant, from an empty and from a non-empty
base graph; bad ids are flagged, not faulted."""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

VARIANTS = [("uf_rem_cas", "naive", "split_one"), ("uf_rem_cas", "split", "halve_one"),
            ("uf_rem_cas", "halve", "split_one"), ("uf_async", "naive", "split_one"),
            ("uf_async", "split", "split_one"), ("uf_async", "halve", "split_one"),
            ("uf_rem_cas", "naive", "atomic"), ("uf_rem_cas", "halve", "atomic"),
            ("uf_async", "compress", "split_one"), ("uf_hooks", "naive", "split_one"),
            ("uf_hooks", "compress", "split_one"), ("uf_early", "naive", "split_one"),
            ("uf_early", "split", "split_one"), ("uf_early", "compress", "split_one"),
            ("sv", "naive", "split_one"), ("lt_prf", "naive", "split_one")]


def run_batches(base, n, fin, nbatches, seed, sizes, qfrac, sample="kout"):
    if base is not None:
        inc = cc.Incremental(n, base.offsets.cuda(), base.edges.cuda(), sample=cc.sample_opt(sample),
                             finish=cc.finish_opt(*fin))
        ref = oracle.Incremental(*base.numpy())
    else:
        inc = cc.Incremental(n, finish=cc.finish_opt(*fin))
        ref = oracle.Incremental(np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32))
    scale = max(1, (n - 1).bit_length())
    for b in range(nbatches):
        k = sizes[b % len(sizes)]
        nq = int(k * qfrac / (1 - qfrac)) if qfrac < 1 else k
        ins = synth.rmat_pairs(scale, k, seed=seed + b, stream=300) % n if k else torch.zeros(0, 2, dtype=torch.int32)
        qs = synth.random_pairs(n, nq, seed=seed + b, stream=400)
        inc.insert(ins.reshape(-1).cuda())
        ans = inc.query(qs.reshape(-1).cuda())
        ref.insert(ins.numpy())
        want = ref.query(qs.numpy())
        assert np.array_equal(ans.cpu().numpy(), want), (fin, b)
        lab = inc.labels().cpu().numpy().view(np.uint32)
        assert np.array_equal(lab, ref.labels()), (fin, b)
    inc.close()


@pytest.mark.parametrize("fin", VARIANTS, ids=lambda f: "-".join(f))
def test_incremental_from_empty(fin):
    run_batches(None, 1 << 14, fin, 8, seed=1, sizes=[1, 10, 1000, 20000], qfrac=0.5)


@pytest.mark.parametrize("fin", VARIANTS[:2] + VARIANTS[3:4] + VARIANTS[6:7] + VARIANTS[9:10] + VARIANTS[11:12] +
                         VARIANTS[14:16], ids=lambda f: "-".join(f))
@pytest.mark.parametrize("sample", ["none", "kout", "ldd"])
def test_incremental_on_base_graph(fin, sample):
    base = synth.rmat(15, 4, seed=3)
    run_batches(base, base.n, fin, 6, seed=7, sizes=[5000, 50000, 300], qfrac=0.9, sample=sample)


def test_query_only_and_insert_only_batches():
    base = synth.erdos_renyi(50000, 0.8, seed=2)
    inc = cc.Incremental(base.n, base.offsets.cuda(), base.edges.cuda())
    ref = oracle.Incremental(*base.numpy())
    qs = synth.random_pairs(base.n, 100000, seed=5, stream=9)
    assert np.array_equal(inc.query(qs.reshape(-1).cuda()).cpu().numpy(), ref.query(qs.numpy()))
    ins = synth.random_pairs(base.n, 30000, seed=6, stream=10)
    inc.insert(ins.reshape(-1).cuda())
    ref.insert(ins.numpy())
    assert np.array_equal(inc.labels().cpu().numpy().view(np.uint32), ref.labels())
    # empty batches are no-ops
    inc.insert(torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert inc.query(torch.zeros(0, dtype=torch.int32, device="cuda")).numel() == 0
    inc.close()


def test_bad_pair_ids_flagged():
    inc = cc.Incremental(100)
    pairs = torch.tensor([1, 2, 3, 500, 7, 8], dtype=torch.int32, device="cuda")
    inc.insert(pairs)
    assert cc.device_error() & 1
    ans = inc.query(torch.tensor([1, 2, 500, 3, 7, 8], dtype=torch.int32, device="cuda"))
    assert ans.cpu().tolist() == [1, 0, 1]
    assert cc.device_error() & 1
    lab = inc.labels().cpu().numpy()
    assert lab[2] == 1 and lab[8] == 7 and lab[3] == 3 and lab[0] == 0
    inc.close()
