"""Parity of the CUDA static-connectivity path with the CPU oracle: labels,
sampled labels, L_max and finish work counts, element by element and bit for
bit, through the C ABI, on graphs that span many warps, chunks and a ragged
tail; plus the edge cases the method has."""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_03909_gb300 as cc
import synth

pytestmark = pytest.mark.gpu

SAMPLES = ["none", "kout", "bfs", "ldd"]
UF_VARIANTS = [("uf_rem_cas", "naive", "split_one"), ("uf_rem_cas", "naive", "halve_one"),
               ("uf_rem_cas", "split", "split_one"), ("uf_rem_cas", "halve", "halve_one"),
               ("uf_rem_cas", "naive", "atomic"), ("uf_rem_cas", "split", "atomic"),
               ("uf_rem_cas", "halve", "atomic"),
               ("uf_async", "naive", "split_one"), ("uf_async", "split", "split_one"),
               ("uf_async", "halve", "split_one"), ("uf_async", "compress", "split_one"),
               ("uf_hooks", "naive", "split_one"), ("uf_hooks", "split", "split_one"),
               ("uf_hooks", "halve", "split_one"), ("uf_hooks", "compress", "split_one"),
               ("uf_early", "naive", "split_one"), ("uf_early", "split", "split_one"),
               ("uf_early", "halve", "split_one"), ("uf_early", "compress", "split_one")]
FINISHES = UF_VARIANTS + [("sv", "naive", "split_one"), ("lt_prf", "naive", "split_one")]


def on_gpu(g, u64=True):
    off = g.offsets if u64 else g.offsets_u32()
    return off.cuda(), g.edges.cuda()


def gpu_labels(g, sample="none", fin=("uf_rem_cas", "naive", "split_one"), u64=True, **kw):
    off, edg = on_gpu(g, u64)
    so = cc.sample_opt(sample, **kw)
    fo = cc.finish_opt(*fin)
    lab, st = cc.cc_static(off, edg, so, fo, stats=True)
    torch.cuda.synchronize()
    return lab.cpu().numpy().view(np.uint32), st


def graphs_small():
    return [synth.rmat(12, 8, seed=3), synth.grid2d(61, 47, 0.3, seed=2), synth.erdos_renyi(20011, 1.2, seed=4),
            synth.cliques([1, 5, 40, 3, 300, 2]), synth.star(5000, centre=4321), synth.path(3001),
            synth.counterexample(), synth.empty(1), synth.empty(77)]


@pytest.fixture(scope="module")
def small():
    gs = graphs_small()
    return [(g, oracle.cc_uf(*g.numpy())[0]) for g in gs]


@pytest.mark.parametrize("fin", FINISHES, ids=lambda f: "-".join(f))
@pytest.mark.parametrize("sample", SAMPLES)
def test_labels_match_oracle_small(small, sample, fin):
    for g, want in small:
        got, _ = gpu_labels(g, sample, fin, seed=5)
        assert np.array_equal(got, want), (g.name, sample, fin)
    assert cc.device_error() == 0


@pytest.mark.parametrize("sample", SAMPLES)
def test_u32_offsets_match(sample):
    g = synth.rmat(14, 8, seed=9)
    want, _ = oracle.cc_uf(*g.numpy())
    got, _ = gpu_labels(g, sample, u64=False, seed=3)
    assert np.array_equal(got, want)


def test_rmat16_config1():
    """RMAT scale 16, edge factor 8, (0.57, 0.19, 0.19, 0.05), seed 1, uint32
    offsets, no sampling, union-find finish."""
    g = synth.rmat(16, 8, seed=1)
    want, _ = oracle.cc_uf(*g.numpy())
    got, st = gpu_labels(g, "none", ("uf_rem_cas", "naive", "split_one"), u64=False)
    assert np.array_equal(got, want)
    assert st["lmax"] == 0xFFFFFFFF and st["edges_finish"] == g.m


@pytest.mark.parametrize("sample", ["kout", "bfs", "ldd"])
@pytest.mark.parametrize("fin", [("uf_rem_cas", "naive", "split_one"), ("uf_async", "halve", "split_one"),
                                 ("sv", "naive", "split_one"), ("lt_prf", "naive", "split_one")],
                         ids=lambda f: f[0])
def test_medium_graphs_and_work_counts(sample, fin):
    """RMAT-18 / grid / ER: labels bit-exact; with exact IdentifyFrequent the
    GPU picks the oracle's L_max and reads exactly the oracle's finish edges."""
    for g in (synth.rmat(18, 16, seed=1), synth.grid2d(700, 650, 0.3, seed=1),
              synth.erdos_renyi(1 << 19, 1.2, seed=1)):
        off, edg = g.numpy()
        want, ost = oracle.connectivity(off, edg, sample, fin[0], seed=11, tries=3, beta=0.2)
        got, st = gpu_labels(g, sample, fin, seed=11)
        assert np.array_equal(got, want), (g.name, sample, fin)
        assert st["lmax"] == ost["lmax"]
        deg = np.diff(off)
        sampled = {"kout": lambda: oracle.kout_sample(off, edg, 2, 11),
                   "bfs": lambda: oracle.bfs_sample(off, edg, 3, 11)[0],
                   "ldd": lambda: oracle.ldd_sample(off, edg, 0.2)[0]}[sample]()
        assert st["edges_finish"] == int(deg[sampled != ost["lmax"]].sum())
        if sample == "bfs":
            assert st["sample_info"] == ost["sample_info"]
        if sample == "ldd":
            assert st["sample_info"] == ost["sample_info"]


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("rule", ["hybrid", "afforest", "pure"])
def test_kout_sampled_labels_bit_exact(k, rule):
    for g in (synth.rmat(15, 8, seed=2), synth.grid2d(300, 200, 0.3, seed=3)):
        off, edg = on_gpu(g)
        lab, info = cc.cc_sample(off, edg, cc.sample_opt("kout", k=k, seed=77, kout_rule=rule))
        want = oracle.kout_sample(*g.numpy(), k=k, seed=77, rule=rule)
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("rule", ["afforest", "pure"])
@pytest.mark.parametrize("fin", [("uf_rem_cas", "naive", "split_one"), ("uf_hooks", "compress", "split_one"),
                                 ("uf_early", "halve", "split_one"), ("sv", "naive", "split_one")],
                         ids=lambda f: f[0])
def test_kout_rules_full_pipeline(rule, fin):
    """Each rule through sampling, IdentifyFrequent and the finish: the
    oracle's L_max, finish edge count and labels."""
    for g in (synth.rmat(17, 16, seed=4), synth.grid2d(500, 400, 0.3, seed=2)):
        off, edg = g.numpy()
        want, ost = oracle.connectivity(off, edg, "kout", fin[0], k=2, seed=13, kout_rule=rule)
        got, st = gpu_labels(g, "kout", fin, seed=13, kout_rule=rule)
        assert np.array_equal(got, want), (g.name, rule, fin)
        assert st["lmax"] == ost["lmax"]
        sampled = oracle.kout_sample(off, edg, 2, 13, rule=rule)
        assert st["edges_finish"] == int(np.diff(off)[sampled != ost["lmax"]].sum())


@pytest.mark.parametrize("tries,seed", [(3, 1), (1, 2), (3, 7)])
def test_bfs_sampled_labels_bit_exact(tries, seed):
    for g in (synth.rmat(16, 8, seed=5), synth.grid2d(400, 300, 0.3, seed=1), synth.erdos_renyi(1 << 17, 1.1)):
        off, edg = on_gpu(g)
        lab, info = cc.cc_sample(off, edg, cc.sample_opt("bfs", bfs_tries=tries, seed=seed))
        want, t = oracle.bfs_sample(*g.numpy(), tries=tries, seed=seed)
        assert info == t
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)


def test_bfs_long_paths_run_many_persistent_launches():
    """High-diameter inputs keep the top-down levels in the persistent launch;
    a path longer than its per-launch level cap (65536) continues across
    launches.  Labels and the successful try match the oracle."""
    for g in (synth.path(150001), synth.grid2d(700, 650, 0.0), synth.grid2d(900, 800, 0.4, seed=7)):
        off, edg = on_gpu(g)
        lab, info = cc.cc_sample(off, edg, cc.sample_opt("bfs", bfs_tries=3, seed=2))
        want, t = oracle.bfs_sample(*g.numpy(), tries=3, seed=2)
        assert info == t
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
        full, _ = gpu_labels(g, "bfs", seed=2)
        assert np.array_equal(full, oracle.cc_uf(*g.numpy())[0])
    assert cc.device_error() == 0


def test_bfs_sample_retries_and_fallback():
    # 40% in one clique, 60% isolated: tries succeed or fall back per the draws
    n = 1000
    g = synth.from_edge_list(n, [(i, j) for i in range(600, 1000, 3) for j in range(i + 1, min(i + 40, 1000))])
    off, edg = on_gpu(g)
    for seed in range(12):
        lab, info = cc.cc_sample(off, edg, cc.sample_opt("bfs", bfs_tries=2, seed=seed))
        want, t = oracle.bfs_sample(*g.numpy(), tries=2, seed=seed)
        assert info == t and np.array_equal(lab.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("beta", [0.05, 0.2, 1.0, 50.0])
def test_ldd_sampled_labels_bit_exact(beta):
    for g in (synth.rmat(15, 8, seed=4), synth.grid2d(250, 250, 0.3, seed=2), synth.path(500)):
        off, edg = on_gpu(g)
        lab, rounds = cc.cc_sample(off, edg, cc.sample_opt("ldd", ldd_beta=beta))
        want, r = oracle.ldd_sample(*g.numpy(), beta=beta)
        assert rounds == r
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)


def ldd_pull_graph():
    """A graph whose second and third LDD rounds (beta 0.05: one new centre
    per round) run bottom-up and need every branch of the bottom-up scan.
    Round 0 claims F = 10000..10099 (a clique) for centre 0; round 1 starts
    centre 1, whose neighbours are the two heavy vertices h1 = 6000 and
    h2 = 6001.  Each heavy vertex lists vertex 1 first, then 3000 fillers
    (2000..4999), then (h1 only) all of F: h1's first edges reach only
    centre 1, its probe misses the smallest centre 0, its chunks are listed
    and the second one meets 0; h2 never meets 0 and keeps 1.  In round 2
    the fillers (light, neighbours h1 < h2) stop at h1's centre 0."""
    F = range(10000, 10100)
    fill = range(2000, 5000)
    e = [(0, f) for f in F] + [(a, b) for a in F for b in F if a < b] + [(1, 6000), (1, 6001)]
    e += [(h, x) for h in (6000, 6001) for x in fill] + [(6000, f) for f in F]
    return synth.from_edge_list(10100, e)


def test_ldd_bottom_up_scan_paths():
    g = ldd_pull_graph()
    off, edg = g.numpy()
    deg = np.diff(off)
    m = int(off[-1])
    # the direction rule (bottom-up when the uncovered vertices' edges are
    # fewer than twice the frontier's) picks bottom-up in rounds 1 and 2
    mf1 = int(deg[10000:10100].sum() + deg[1])
    assert m - deg[0] - mf1 < 2 * mf1
    mf2 = int(deg[6000] + deg[6001] + deg[2])
    assert m - deg[0] - mf1 - mf2 < 2 * mf2
    assert deg[6000] > 2048 and deg[6001] > 2048   # two chunks each
    want, r = oracle.ldd_sample(off, edg, beta=0.05)
    assert want[6000] == want[10000] and want[6001] == want[1] != want[0]
    d_off, d_edg = on_gpu(g)
    for _ in range(5):
        lab, rounds = cc.cc_sample(d_off, d_edg, cc.sample_opt("ldd", ldd_beta=0.05))
        assert rounds == r
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
    assert cc.device_error() == 0


@pytest.mark.parametrize("sizes", [[30] * 20 + [31], [30] * 20, [2] * 500 + [40, 40]])
def test_lmax_without_a_majority_cluster(sizes):
    # disjoint cliques: after k-out every clique is one cluster and none holds
    # a majority of the non-root vertices, so the sampled L_max guess cannot
    # be confirmed by its share and the labels are counted in full; L_max
    # (ties to the smallest label) and the finish's edges match the oracle
    g = synth.cliques(sizes)
    off, edg = g.numpy()
    for fin in (("uf_rem_cas", "naive", "split_one"), ("sv", "naive", "split_one")):
        want, ost = oracle.connectivity(off, edg, "kout", fin[0], seed=5, tries=3, beta=0.2)
        got, st = gpu_labels(g, "kout", fin, seed=5)
        assert np.array_equal(got, want)
        assert st["lmax"] == ost["lmax"]
        lab = oracle.kout_sample(off, edg, 2, 5)
        deg = np.diff(off)
        assert st["edges_finish"] == int(deg[lab != ost["lmax"]].sum())


def test_ldd_tie_golden():
    # the hand-worked graph where vertex 19 is claimed by two clusters in the
    # same round: the smaller centre must win on every run (the kernel's
    # claims race, the rule does not)
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle import load_ldd_tie
    beta, g, want, rounds = load_ldd_tie()
    off, edg = on_gpu(g)
    for _ in range(20):
        lab, r = cc.cc_sample(off, edg, cc.sample_opt("ldd", ldd_beta=beta))
        assert r == rounds
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("samples", [0, 1, 100, 4096])
def test_identify_frequent_bit_exact(samples):
    rng = np.random.default_rng(3)
    for n in (1, 31, 1000, 200_003):
        lab = rng.integers(0, max(1, n // 7), size=n).astype(np.uint32)
        lab[: n // 3] = n // 11  # a frequent label
        got = cc.cc_identify_frequent(torch.from_numpy(lab.view(np.int32)).cuda(), samples, seed=9)
        want, _ = oracle.identify_frequent(lab, samples, 9)
        assert int(got.item()) & 0xFFFFFFFF == want


@pytest.mark.parametrize("fin", FINISHES, ids=lambda f: "-".join(f))
def test_finish_from_oracle_sampled_labels(fin):
    """cc_finish on the oracle's sampled labels and L_max (phase parity)."""
    g = synth.rmat(16, 8, seed=6)
    off, edg = g.numpy()
    lab = oracle.kout_sample(off, edg, 2, 3)
    lm, _ = oracle.identify_frequent(lab)
    want, _ = oracle.finish(off, edg, lab, lm, fin[0])
    t = torch.from_numpy(lab.astype(np.uint32).view(np.int32)).cuda()
    o, e = on_gpu(g)
    cc.cc_finish(o, e, t, lm, cc.finish_opt(*fin))
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want)
    # and with nothing to skip
    t = torch.arange(g.n, dtype=torch.int32, device="cuda")
    cc.cc_finish(o, e, t, 0xFFFFFFFF, cc.finish_opt(*fin))
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want)


def test_rmat22_all_combinations_agree_with_oracle():
    g = synth.rmat(22, 16, seed=1, device="cuda").to("cpu")
    want, _ = oracle.cc_uf(*g.numpy())
    for sample in SAMPLES:
        for fin in [("uf_rem_cas", "naive", "split_one"), ("uf_async", "split", "split_one"),
                    ("sv", "naive", "split_one"), ("lt_prf", "naive", "split_one")]:
            got, _ = gpu_labels(g, sample, fin)
            assert np.array_equal(got, want), (sample, fin)
    assert cc.device_error() == 0


def test_repeat_runs_identical():
    """Nondeterministic atomics, deterministic output."""
    g = synth.rmat(17, 16, seed=8)
    first, _ = gpu_labels(g, "kout")
    for _ in range(5):
        again, _ = gpu_labels(g, "kout")
        assert np.array_equal(first, again)


def test_host_buffer_zero_copy_and_fallback_copy():
    """k-out on pinned host buffers reads them in place; a graph whose
    frequent cluster is small copies the CSR before the finish.  Both give
    the oracle's labels."""
    for g in (synth.rmat(16, 16, seed=4), synth.erdos_renyi(1 << 17, 0.6, seed=2), synth.grid2d(300, 280, 0.45)):
        want, _ = oracle.cc_uf(*g.numpy())
        for u64 in (True, False):
            off = (g.offsets if u64 else g.offsets_u32()).pin_memory()
            lab = cc.cc_static_host(off, g.edges.pin_memory(), cc.sample_opt("kout"))
            assert np.array_equal(lab.numpy().view(np.uint32), want), (g.name, u64)
    assert cc.device_error() == 0


def test_host_buffer_entry_point():
    g = synth.rmat(15, 8, seed=2)
    want, _ = oracle.cc_uf(*g.numpy())
    lab = cc.cc_static_host(g.offsets.pin_memory(), g.edges.pin_memory())
    assert np.array_equal(lab.numpy().view(np.uint32), want)
    lab = cc.cc_static_host(g.offsets_u32(), g.edges, sample=cc.sample_opt("ldd"))  # pageable host memory
    assert np.array_equal(lab.numpy().view(np.uint32), want)


def test_bad_edge_ids_are_flagged_not_faulted():
    g = synth.path(100)
    off, edg = on_gpu(g)
    edg = edg.clone()
    edg[7] = 100 + 12345  # out of range
    lab = cc.cc_static(off, edg, cc.sample_opt("none"))
    bits = cc.device_error()
    assert bits & 1
    lab = cc.cc_static(off, edg, cc.sample_opt("kout"))
    assert cc.device_error() & 1
    # offsets past m
    off2 = off.clone()
    off2[50] = 10**6
    cc.cc_static(off2, edg, cc.sample_opt("none"))
    assert cc.device_error() & 2
    assert cc.device_error() == 0


def test_iteration_cap_reports_nonconvergence():
    g = synth.path(4000)
    off, edg = on_gpu(g)
    try:
        cc.set_iteration_cap(2)
        with pytest.raises(cc.CCError) as ei:
            cc.cc_static(off, edg, cc.sample_opt("none"), cc.finish_opt("sv"), stats=True)
        assert ei.value.status == 4
    finally:
        cc.set_iteration_cap(0)
    cc.device_error()
    got, _ = gpu_labels(g, "none", ("sv", "naive", "split_one"))
    assert np.all(got == 0)


def test_unaligned_label_slices():
    """Label buffers that are 4-byte- but not 16-byte-aligned slices work
    (vector accesses only where the address allows them)."""
    g = synth.rmat(14, 8, seed=3)
    want, _ = oracle.cc_uf(*g.numpy())
    off, edg = on_gpu(g)
    buf = torch.full((g.n + 7,), -1, dtype=torch.int32, device="cuda")
    for shift in (1, 2, 3):
        out = buf[shift:shift + g.n]
        for s in ("none", "kout", "bfs", "ldd"):
            cc.cc_static(off, edg, cc.sample_opt(s), labels_out=out)
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want), (shift, s)
        lab, _ = cc.cc_sample(off, edg, cc.sample_opt("kout"), labels_out=out)
        lm = cc.cc_identify_frequent(out)
        wl, _ = oracle.identify_frequent(oracle.kout_sample(*g.numpy(), 2, 1))
        assert int(lm.item()) == wl
    assert cc.device_error() == 0


@pytest.mark.parametrize("u64", [True, False])
def test_map_and_gather_edges_bit_exact(u64):
    """Table 8's primitives against their definitions (numpy reductions)."""
    for g in (synth.rmat(16, 8, seed=2), synth.star(70000, centre=3), synth.empty(9)):
        off, edg = on_gpu(g, u64)
        o, e = g.numpy()
        deg = np.diff(o).astype(np.uint32)
        assert np.array_equal(cc.cc_map_edges(off, edg).cpu().numpy().view(np.uint32), deg)
        x = np.random.default_rng(1).integers(0, 2**32, size=g.n, dtype=np.uint64).astype(np.uint32)
        got = cc.cc_gather_edges(off, edg, torch.from_numpy(x.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
        want = np.zeros(g.n, np.uint64)
        src = np.repeat(np.arange(g.n), np.diff(o))
        np.add.at(want, src, x[e.astype(np.int64)].astype(np.uint64))
        assert np.array_equal(got, (want % 2**32).astype(np.uint32))


def _splitmix64(seed, ctr):
    """SplitMix64 (Steele, Lea and Flood, 2014) at counter ctr, in Python integers."""
    M = (1 << 64) - 1
    z = (seed + (ctr + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


@pytest.mark.parametrize("words,count", [(1, 5), (1000, 3), (123457, 10001), (1 << 20, 1 << 16)])
def test_random_sectors_sum(words, count):
    """The random-sector probe reads exactly the words its definition names."""
    x = np.random.default_rng(words).integers(0, 2**32, size=words, dtype=np.uint64).astype(np.uint32)
    got = cc.cc_random_sectors(torch.from_numpy(x.view(np.int32)).cuda(), count, seed=77)
    idx = [(_splitmix64(77, i) * words) >> 64 for i in range(count)]
    want = int(x[np.array(idx, dtype=np.int64)].astype(np.uint64).sum()) % 2**32
    assert int(got.cpu().numpy().view(np.uint32)[0]) == want
    empty = cc.cc_random_sectors(torch.from_numpy(x.view(np.int32)).cuda(), 0)
    assert int(empty.item()) == 0
