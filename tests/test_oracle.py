"""Pins for the CPU oracle (no GPU): each check ties the oracle to something
other than itself -- brute force, closed forms, library routines, published
test vectors, invariants that follow from the paper's definitions."""
import itertools
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1
COMBOS = [(s, f) for s in ("none", "kout", "bfs", "ldd") for f in ("uf_rem_cas", "uf_async", "sv", "lt_prf")]


# ---------------------------------------------------------------- helpers
def closure_labels(n, pairs):
    """Min-id labels from the boolean transitive closure (Warshall)."""
    R = np.eye(n, dtype=bool)
    for u, v in pairs:
        R[u, v] = R[v, u] = True
    for k in range(n):
        R |= R[:, k:k + 1] & R[k:k + 1, :]
    return np.array([int(np.argmax(R[v])) for v in range(n)], dtype=np.uint32)


def scipy_labels(n, u, v):
    """Min-id labels via scipy's connected_components (a library routine)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    g = coo_matrix((np.ones(len(u)), (np.asarray(u), np.asarray(v))), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    cmin = np.full(comp.max() + 1 if n else 0, n, dtype=np.int64)
    np.minimum.at(cmin, comp, np.arange(n))
    return cmin[comp].astype(np.uint32)


def csr_pairs(g):
    off, edg = g.numpy()
    src = np.repeat(np.arange(g.n), np.diff(off))
    return src, edg.astype(np.int64)


def splitmix_out(seed, ctr):
    """The ctr-th output of SplitMix64 from state ``seed``, from its definition."""
    z = (seed + (ctr + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def check_invariants(g, lab):
    off, edg = g.numpy()
    src, dst = csr_pairs(g)
    assert np.all(lab[src] == lab[dst]), "an edge's endpoints differ"
    assert np.all(lab <= np.arange(g.n)), "label above its vertex"
    assert np.all(lab[lab] == lab), "label is not a fixed point"


# ---------------------------------------------------------------- the draw
def test_splitmix_published_vector():
    vals = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    assert [oracle.draw(1234567, i) for i in range(5)] == vals


def test_splitmix_counter_form():
    for s in (0, 1, 99, 2**63 + 5):
        for i in (0, 1, 7, 1000):
            assert oracle.draw(s, i) == splitmix_out(s, i)


# ---------------------------------------------------------------- O1 / O2
def test_bruteforce_all_graphs_n5():
    """All 1,024 graphs on 5 vertices: O1, O2 and every sampling x finish
    combination equal the transitive-closure minimum."""
    n = 5
    allpairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(allpairs)):
        pairs = [allpairs[i] for i in range(len(allpairs)) if mask >> i & 1]
        want = closure_labels(n, pairs)
        g = synth.from_edge_list(n, pairs)
        off, edg = g.numpy()
        lab, links = oracle.cc_uf(off, edg)
        assert np.array_equal(lab, want), (pairs, lab, want)
        assert links == n - len(np.unique(want))
        assert np.array_equal(oracle.cc_bfs(off, edg), want)
        if mask % 7 == 0:  # the combination matrix on a seventh of the graphs
            for s, f in COMBOS:
                got, _ = oracle.connectivity(off, edg, s, f, seed=mask, tries=2, beta=0.7)
                assert np.array_equal(got, want), (pairs, s, f)


def test_bruteforce_random_n8():
    rng = np.random.default_rng(5)
    for t in range(300):
        n = int(rng.integers(1, 9))
        allpairs = list(itertools.combinations(range(n), 2))
        pairs = [p for p in allpairs if rng.random() < 0.25]
        want = closure_labels(n, pairs)
        g = synth.from_edge_list(n, pairs)
        off, edg = g.numpy()
        for s, f in COMBOS:
            got, _ = oracle.connectivity(off, edg, s, f, seed=t, k=int(rng.integers(1, 4)))
            assert np.array_equal(got, want), (n, pairs, s, f)


def test_o1_equals_o2_and_scipy_on_workload_shapes():
    for g in (synth.rmat(12, 8, seed=3), synth.grid2d(40, 37, 0.45, seed=2),
              synth.erdos_renyi(5000, 1.2, seed=4)):
        off, edg = g.numpy()
        a, links = oracle.cc_uf(off, edg)
        b = oracle.cc_bfs(off, edg)
        src, dst = csr_pairs(g)
        c = scipy_labels(g.n, src, dst)
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert links == g.n - len(np.unique(a))
        check_invariants(g, a)


def test_uf_prefix_is_o1_slice():
    g = synth.rmat(12, 8, seed=4)
    off, edg = g.numpy()
    full, _ = oracle.cc_uf(off, edg)
    P, cnt = oracle.uf_prefix(off, edg, g.n)
    assert cnt == g.m
    roots = np.array([P[v] for v in range(g.n)])
    for _ in range(20):
        roots = P[roots]
    assert np.array_equal(roots, full)
    P, cnt = oracle.uf_prefix(off, edg, 100)
    assert cnt == int(off[100])


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("s,f", COMBOS)
def test_closed_forms(s, f):
    cases = []
    cases.append((synth.empty(17), np.arange(17)))
    cases.append((synth.path(50), np.zeros(50)))
    cases.append((synth.grid2d(13, 11, 0.0), np.zeros(143)))
    sizes = [3, 1, 7, 2, 5]
    starts = np.repeat(np.cumsum([0] + sizes[:-1]), sizes)
    cases.append((synth.cliques(sizes), starts))
    cases.append((synth.star(30, centre=17), np.zeros(30)))
    ce = synth.counterexample()
    gold = [ln for ln in open(os.path.join(GOLDEN, "rem_counterexample.txt"))
            if ln.startswith("labels")][0].split()[1:]
    cases.append((ce, np.array([int(x) for x in gold])))
    for g, want in cases:
        off, edg = g.numpy()
        got, _ = oracle.connectivity(off, edg, s, f, seed=7)
        assert np.array_equal(got, np.asarray(want, dtype=np.uint32)), (g.name, s, f)


def test_permuted_graphs():
    """Relabelling vertices by pi maps each component C to label min pi(C)."""
    for g in (synth.cliques([4, 9, 2, 6]), synth.grid2d(9, 8, 0.4, seed=5), synth.path(20)):
        base, _ = oracle.cc_uf(*g.numpy())
        perm = synth.random_perm(g.n, 3).numpy()
        gp = synth.relabel(g, torch.from_numpy(perm))
        got, _ = oracle.cc_uf(*gp.numpy())
        want = np.empty(g.n, np.uint32)
        for c in np.unique(base):
            members = np.nonzero(base == c)[0]
            want[perm[members]] = perm[members].min()
        assert np.array_equal(got, want)


def test_er_component_statistics():
    """G(n, M) at average degree 1.2: giant fraction S solves S = 1 - exp(-1.2 S)
    (S ~= 0.3137) and #components ~= n (1 - S)(1 - 1.2 (1 - S) / 2) (~0.404 n)."""
    n = 1 << 17
    g = synth.erdos_renyi(n, 1.2, seed=9)
    lab, _ = oracle.cc_uf(*g.numpy())
    S = 0.5
    for _ in range(200):
        S = 1 - np.exp(-1.2 * S)
    counts = np.bincount(lab, minlength=n)
    assert abs(counts.max() / n - S) < 0.03
    ncomp = len(np.unique(lab))
    assert abs(ncomp / n - (1 - S) * (1 - 1.2 * (1 - S) / 2)) < 0.01


# ---------------------------------------------------------------- IdentifyFrequent
def test_identify_frequent_exact_matches_bincount():
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(1, 300))
        lab = rng.integers(0, n, size=n).astype(np.uint32)
        lm, c = oracle.identify_frequent(lab)
        bc = np.bincount(lab, minlength=n)
        assert lm == int(np.argmax(bc)) and c == int(bc.max())  # argmax: first (smallest) of ties


def test_identify_frequent_sampled_positions():
    rng = np.random.default_rng(2)
    n = 1000
    lab = rng.integers(0, 37, size=n).astype(np.uint32)
    S, seed = 257, 12345
    pos = [splitmix_out(seed ^ 0x66726571, i) % n for i in range(S)]
    bc = np.bincount(lab[pos], minlength=n)
    lm, c = oracle.identify_frequent(lab, S, seed)
    assert lm == int(np.argmax(bc)) and c == int(bc.max())


# ---------------------------------------------------------------- sampling
def kout_edges_py(g, k, seed, rule="hybrid"):
    off, edg = g.numpy()
    us, vs = [], []
    for v in range(g.n):
        d = int(off[v + 1] - off[v])
        if d == 0:
            continue
        for j in range(k):
            if rule == "afforest":
                if j >= d:
                    continue
                w = edg[off[v] + j]
            elif j == 0 and rule == "hybrid":
                w = edg[off[v]]
            else:
                h = splitmix_out(seed ^ 0x6B6F7574, v * k + j) >> 32
                w = edg[off[v] + ((h * d) >> 32)]
            us.append(v)
            vs.append(int(w))
    return us, vs


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("rule", ["hybrid", "afforest", "pure"])
def test_kout_sample_is_cc_of_picked_edges(k, rule):
    for g in (synth.rmat(10, 8, seed=2), synth.grid2d(30, 30, 0.3, seed=1), synth.erdos_renyi(3000, 2.0)):
        off, edg = g.numpy()
        us, vs = kout_edges_py(g, k, seed=77, rule=rule)
        want = scipy_labels(g.n, us, vs)
        got = oracle.kout_sample(off, edg, k=k, seed=77, rule=rule)
        assert np.array_equal(got, want)


def test_kout_rules_closed_forms():
    g = synth.rmat(11, 8, seed=4)
    off, edg = g.numpy()
    maxdeg = int(np.diff(off).max())
    # afforest with k >= the maximum degree samples every edge: exact labels
    assert np.array_equal(oracle.kout_sample(off, edg, k=maxdeg, rule="afforest"), oracle.cc_uf(off, edg)[0])
    # hybrid and afforest coincide at k = 1 (both take the first edge)
    assert np.array_equal(oracle.kout_sample(off, edg, k=1, rule="afforest"),
                          oracle.kout_sample(off, edg, k=1, seed=5, rule="hybrid"))
    # afforest pick j is the j-th neighbour, none past the degree
    v = int(np.argmax(np.diff(off) == 3))
    assert [oracle.kout_pick(off, edg, v, 5, j, 1, "afforest") for j in range(5)] == \
        [int(x) for x in edg[off[v]:off[v] + 3]] + [oracle.NONE] * 2
    # every rule is exact on a perfect matching (each vertex has one edge)
    mt = synth.from_edge_list(40, [(2 * i, 2 * i + 1) for i in range(20)])
    for rule in ("hybrid", "afforest", "pure"):
        lab = oracle.kout_sample(*mt.numpy(), k=1, seed=3, rule=rule)
        assert np.array_equal(lab, np.repeat(np.arange(0, 40, 2), 2))


def test_kout_pure_picks_are_uniform():
    """Pure sampling draws every slot uniformly: positions of the picks in
    the adjacency lists of K_50 (degree 49) pass a chi-square test."""
    from scipy.stats import chisquare
    g = synth.cliques([50])
    off, edg = g.numpy()
    counts = np.zeros(49)
    for v in range(50):
        for j in range(40):
            w = oracle.kout_pick(off, edg, v, 40, j, 11, "pure")
            counts[int(np.flatnonzero(edg[off[v]:off[v + 1]] == w)[0])] += 1
    assert chisquare(counts).pvalue > 1e-3


def test_kout_on_matching_is_exact():
    """Every vertex of a perfect matching has degree 1: the sample is the graph."""
    g = synth.from_edge_list(20, [(2 * i, 2 * i + 1) for i in range(10)])
    lab = oracle.kout_sample(*g.numpy(), k=2, seed=3)
    assert np.array_equal(lab, np.repeat(np.arange(0, 20, 2), 2))


def reach_labels(g, s):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    off, edg = g.numpy()
    A = csr_matrix((np.ones(g.m), edg, off), shape=(g.n, g.n))
    return breadth_first_order(A, s, directed=True, return_predecessors=False)


def test_bfs_sample_tries_and_threshold():
    # 40% of vertices in one clique, the rest isolated: a try succeeds iff the
    # source lands in the clique (40% > 10%); the outcome follows the draws.
    n = 100
    g = synth.from_edge_list(n, [(i, j) for i in range(60, 100) for j in range(i + 1, 100)])
    for seed in range(40):
        got, t = oracle.bfs_sample(*g.numpy(), tries=3, seed=seed)
        srcs = [splitmix_out(seed ^ 0x62667373, i) % n for i in range(3)]
        ok = [i for i, s in enumerate(srcs) if s >= 60]
        want = np.arange(n, dtype=np.uint32)
        if ok:
            assert t == ok[0]
            want[60:] = 60
        else:
            assert t == -1
        assert np.array_equal(got, want)


def test_bfs_sample_is_reachability():
    g = synth.rmat(11, 8, seed=5)
    for seed in range(5):
        got, t = oracle.bfs_sample(*g.numpy(), tries=3, seed=seed)
        s = splitmix_out(seed ^ 0x62667373, t) % g.n
        reach = reach_labels(g, s)
        want = np.arange(g.n, dtype=np.uint32)
        want[reach] = reach.min()
        assert t >= 0 and np.array_equal(got, want)


def test_ten_percent_is_strict():
    # exactly 10% reachable is not "more than 10%"; 11% is
    for size, ok in ((10, False), (11, True)):
        g = synth.from_edge_list(100, [(i, i + 1) for i in range(size - 1)])
        # find a seed whose first source is vertex < size
        seed = next(s for s in range(10000) if splitmix_out(s ^ 0x62667373, 0) % 100 < size)
        _, t = oracle.bfs_sample(*g.numpy(), tries=1, seed=seed)
        assert (t == 0) == ok


def ldd_partition_ok(g, lab):
    """Each cluster is connected inside itself and lies in one component."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    src, dst = csr_pairs(g)
    inside = lab[src] == lab[dst]
    h = coo_matrix((np.ones(inside.sum()), (src[inside], dst[inside])), shape=(g.n, g.n))
    _, comp = connected_components(h, directed=False)
    for c in np.unique(lab):
        assert len(np.unique(comp[lab == c])) == 1
    assert np.all(lab <= np.arange(g.n)) and np.all(lab[lab] == lab)


def test_ldd_closed_forms():
    # beta large: round 0 starts vertex 0 alone, round 1 starts everything else
    g = synth.rmat(9, 4, seed=1)
    off, edg = g.numpy()
    lab, r = oracle.ldd_sample(off, edg, beta=50.0)
    want = np.arange(g.n, dtype=np.uint32)
    want[edg[off[0]:off[1]]] = 0
    assert np.array_equal(lab, want)
    # beta tiny: one new id per round; each clique / path becomes one cluster
    sizes = [4, 1, 6, 3]
    lab, _ = oracle.ldd_sample(*synth.cliques(sizes).numpy(), beta=1e-9)
    assert np.array_equal(lab, np.repeat(np.cumsum([0] + sizes[:-1]), sizes))
    lab, r = oracle.ldd_sample(*synth.path(30).numpy(), beta=1e-9)
    assert np.all(lab == 0) and r == 29  # vertex r+1 is claimed in round r


def load_ldd_tie():
    """The hand-worked tie fixture: (beta, graph, expected labels, rounds)."""
    beta, n, pairs, want, rounds = None, None, [], None, None
    with open(os.path.join(GOLDEN, "ldd_tie.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            if ln.startswith("beta"):
                beta = float(ln.split()[1])
            elif ln.startswith("labels"):
                want = np.array([int(x) for x in ln.split()[1:]], dtype=np.uint32)
            elif ln.startswith("rounds"):
                rounds = int(ln.split()[1])
            elif n is None:
                n = int(ln)
            else:
                a, b = ln.split()
                pairs.append((int(a), int(b)))
    return beta, synth.from_edge_list(n, pairs), want, rounds


def test_ldd_tie_takes_the_smallest_centre():
    # a vertex claimed by two clusters in one round joins the smaller centre's
    beta, g, want, rounds = load_ldd_tie()
    lab, r = oracle.ldd_sample(*g.numpy(), beta=beta)
    assert np.array_equal(lab, want) and r == rounds
    # the schedule the hand derivation used
    assert [oracle.ldd_schedule(g.n, beta, i) for i in range(5)] == [1, 2, 4, 11, 24]


def test_ldd_schedule_counts():
    for beta in (0.2, 0.5, 1.0):
        for r in range(30):
            want = max(1, int(np.floor(np.exp(beta * r))))
            assert oracle.ldd_schedule(1 << 20, beta, r) == min(want, 2**32 - 1)


@pytest.mark.parametrize("beta", [0.05, 0.2, 0.8])
def test_ldd_is_partial_labelling(beta):
    for g in (synth.rmat(11, 8, seed=6), synth.grid2d(40, 40, 0.3, seed=3)):
        lab, _ = oracle.ldd_sample(*g.numpy(), beta=beta)
        ldd_partition_ok(g, lab)
        full, _ = oracle.cc_uf(*g.numpy())
        # same cluster => same component
        assert np.all(full[lab] == full)


# ---------------------------------------------------------------- finish methods
@pytest.mark.parametrize("f", ["uf_rem_cas", "sv", "lt_prf"])
@pytest.mark.parametrize("s", ["kout", "bfs", "ldd"])
def test_finish_from_sampled_labels(s, f):
    for g in (synth.rmat(12, 8, seed=8), synth.grid2d(50, 40, 0.35, seed=4), synth.erdos_renyi(4000, 1.2)):
        off, edg = g.numpy()
        if s == "kout":
            lab = oracle.kout_sample(off, edg, 2, 5)
        elif s == "bfs":
            lab, _ = oracle.bfs_sample(off, edg, 3, 5)
        else:
            lab, _ = oracle.ldd_sample(off, edg, 0.2)
        for samples in (0, 64):
            lm, _ = oracle.identify_frequent(lab, samples, 5)
            got, _ = oracle.finish(off, edg, lab, lm, f)
            want, _ = oracle.cc_uf(off, edg)
            assert np.array_equal(got, want)


def test_uf_finish_skips_lmax_edges():
    """The sampled-work model m - X + Y: the finish applies exactly the edges
    out of vertices whose sampled label is not L_max."""
    g = synth.rmat(12, 8, seed=2)
    off, edg = g.numpy()
    lab = oracle.kout_sample(off, edg, 2, 1)
    lm, _ = oracle.identify_frequent(lab)
    _, applied = oracle.finish(off, edg, lab, lm, "uf_rem_cas")
    deg = np.diff(off)
    assert applied == int(deg[lab != lm].sum())


def test_dropping_skip_side_breaks_cc():
    """A planted mistake (skipping BOTH endpoints' edges of L_max, i.e. also
    from the other side) must change the result: edges into L_max matter."""
    g = synth.from_edge_list(6, [(0, 1), (1, 2), (2, 3), (4, 5)])
    off, edg = g.numpy()
    lab = np.array([0, 0, 0, 3, 4, 4], np.uint32)  # sampled: {0,1,2}, {3}, {4,5}
    good, _ = oracle.finish(off, edg, lab, 0, "uf_rem_cas")
    assert np.array_equal(good, [0, 0, 0, 0, 4, 4])
    # planted: drop edge (2,3) from vertex 3's list as well
    bad_edges = [(0, 1), (1, 2), (4, 5)]
    gb = synth.from_edge_list(6, bad_edges)
    bad, _ = oracle.finish(*gb.numpy(), lab, 0, "uf_rem_cas")
    assert not np.array_equal(bad, good)


# ---------------------------------------------------------------- incremental
def test_incremental_matches_recompute():
    n = 3000
    base = synth.erdos_renyi(n, 0.6, seed=2)
    inc = oracle.Incremental(*base.numpy())
    src, dst = csr_pairs(base)
    us, vs = list(src), list(dst)
    for b in range(6):
        ins = synth.random_pairs(n, 150, seed=b, stream=100).numpy()
        qs = synth.random_pairs(n, 400, seed=b, stream=200).numpy()
        inc.insert(ins)
        ans = inc.query(qs)
        us += list(ins[:, 0]); vs += list(ins[:, 1])
        want = scipy_labels(n, us, vs)
        assert np.array_equal(ans, (want[qs[:, 0]] == want[qs[:, 1]]).astype(np.uint8))
        assert np.array_equal(inc.labels(), want)


# ---------------------------------------------------------------- selector network
def _mlp_case(seed, B=7):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.NPARAM)
    d = mlp.unpack(p)
    d["mu"][:] = rng.normal(0, 1, mlp.IN)
    d["sigma"][:] = rng.uniform(0.5, 2.0, mlp.IN)
    p = mlp.pack(d)
    X = rng.normal(0, 1, (B, mlp.IN))
    Q = mlp.soft_targets(rng.uniform(1, 3, (B, mlp.OUT)), 0.3)
    return p, X, Q


def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp
    p, X, Q = _mlp_case(1)
    g, _ = mlp.backward(p, X, Q)
    rng = np.random.default_rng(2)
    idx = rng.choice(np.arange(2 * mlp.IN, mlp.NPARAM), 60, replace=False)
    h = 1e-6
    for j in idx:
        e = np.zeros_like(p)
        e[j] = h
        num = (mlp.loss(p + e, X, Q) - mlp.loss(p - e, X, Q)) / (2 * h)
        assert abs(num - g[j]) <= 1e-6 + 1e-5 * abs(num), (j, num, g[j])
    assert np.all(g[:2 * mlp.IN] == 0)


def test_mlp_closed_forms():
    from oracle import mlp
    p, X, Q = _mlp_case(3)
    d = mlp.unpack(p)
    d["W3"][:] = 0
    d["b3"][:] = 0
    uniform = np.full_like(Q, 1.0 / mlp.OUT)
    assert abs(mlp.loss(mlp.pack(d), X, uniform) - np.log(mlp.OUT)) < 1e-12   # zero logits
    T = np.random.default_rng(4).uniform(1, 2, (5, mlp.OUT))
    S = mlp.soft_targets(T, 0.1)
    assert np.allclose(S.sum(axis=1), 1) and np.all(S.argmax(axis=1) == T.argmin(axis=1))
    # first Adam step: bias-corrected moments give p - lr * g / (|g| + eps)
    g = np.random.default_rng(5).normal(0, 1, mlp.NPARAM)
    p2, m2, v2 = mlp.adam(p, g, np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM), 1, 0.01)
    want = p - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p2[2 * mlp.IN:], want[2 * mlp.IN:]) and np.array_equal(p2[:2 * mlp.IN], p[:2 * mlp.IN])


# ---------------------------------------------------------------- spanning forest
def forest_is_valid_bruteforce(n, pairs, forest):
    """Independent of the oracle's union-find: every forest pair is an edge,
    the forest has no cycle (DFS over an adjacency dict), and its
    transitive-closure components equal those of the graph."""
    edges = {frozenset(p) for p in pairs}
    if any(frozenset((int(u), int(v))) not in edges or u == v for u, v in forest):
        return False
    adj = {v: [] for v in range(n)}
    for i, (u, v) in enumerate(forest):
        adj[int(u)].append((int(v), i))
        adj[int(v)].append((int(u), i))
    seen = [False] * n
    for s in range(n):
        if seen[s]:
            continue
        stack = [(s, -1)]
        seen[s] = True
        while stack:
            x, via = stack.pop()
            for y, i in adj[x]:
                if i == via:
                    continue
                if seen[y]:
                    return False          # a second path to y: a cycle
                seen[y] = True
                stack.append((y, i))
    return np.array_equal(closure_labels(n, [tuple(map(int, p)) for p in forest]), closure_labels(n, pairs))


def test_spanning_forest_bruteforce_all_graphs_n5():
    n = 5
    allpairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(allpairs)):
        pairs = [allpairs[i] for i in range(len(allpairs)) if mask >> i & 1]
        g = synth.from_edge_list(n, pairs)
        off, edg = g.numpy()
        F = oracle.spanning_forest(off, edg)
        assert forest_is_valid_bruteforce(n, pairs, F), (pairs, F)
        assert oracle.check_forest(off, edg, F) == 0


def test_spanning_forest_closed_forms():
    # a path, a star and a random tree are their own spanning trees
    rng = np.random.default_rng(3)
    parent = [int(rng.integers(0, v)) for v in range(1, 500)]
    tree = synth.from_edge_list(500, [(v, p) for v, p in zip(range(1, 500), parent)])
    for g in (synth.path(300), synth.star(200, centre=17), tree):
        off, edg = g.numpy()
        F = oracle.spanning_forest(off, edg)
        src, dst = csr_pairs(g)
        want = {frozenset((int(a), int(b))) for a, b in zip(src, dst)}
        assert {frozenset(map(int, p)) for p in F} == want
    # a cycle keeps n - 1 of its n edges; disjoint cliques sum(s - 1); an
    # empty graph none
    cyc = synth.from_edge_list(64, [(i, (i + 1) % 64) for i in range(64)])
    assert oracle.spanning_forest(*cyc.numpy()).shape == (63, 2)
    sizes = [4, 9, 1, 30, 2]
    assert oracle.spanning_forest(*synth.cliques(sizes).numpy()).shape == (sum(s - 1 for s in sizes), 2)
    assert oracle.spanning_forest(*synth.empty(10).numpy()).shape == (0, 2)


def test_check_forest_rejects_planted_mistakes():
    g = synth.grid2d(30, 20, 0.3, seed=4)
    off, edg = g.numpy()
    lab, _ = oracle.cc_uf(off, edg)
    F = oracle.spanning_forest(off, edg)
    assert oracle.check_forest(off, edg, F, lab) == 0
    # a pair that is not an edge (two far-apart grid vertices)
    bad = F.copy()
    bad[0] = (0, 599)
    assert oracle.check_forest(off, edg, bad, lab) in (2,)
    # a repeated pair closes a cycle
    assert oracle.check_forest(off, edg, np.vstack([F, F[:1]]), lab) == 3
    # a dropped pair leaves a component unspanned
    assert oracle.check_forest(off, edg, F[1:], lab) == 5
    # an endpoint out of range
    bad = F.copy()
    bad[3, 1] = g.n
    assert oracle.check_forest(off, edg, bad, lab) == 1
    # wrong labels: a forest pair across two claimed components
    lab2 = lab.copy()
    u = int(F[0, 0])
    lab2[lab2 == lab[u]] = np.arange(g.n, dtype=np.uint32)[lab2 == lab[u]]
    assert oracle.check_forest(off, edg, F, lab2) == 4


def test_spanning_forest_workload_shapes():
    for g in (synth.rmat(12, 8, seed=9), synth.grid2d(60, 40, 0.45, seed=1), synth.erdos_renyi(6000, 1.2, seed=2)):
        off, edg = g.numpy()
        lab, links = oracle.cc_uf(off, edg)
        F = oracle.spanning_forest(off, edg)
        assert len(F) == links == g.n - int((lab == np.arange(g.n)).sum())
        assert oracle.check_forest(off, edg, F, lab) == 0


# ---------------------------------------------------------------- minimum spanning forests
def scipy_msf_weight(g, w):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    off, edg = g.numpy()
    A = csr_matrix((np.asarray(w, dtype=np.float64), edg, off), shape=(g.n, g.n))
    return float(minimum_spanning_tree(A).sum())


def test_kruskal_matches_scipy_and_brute_force():
    for g in (synth.rmat(11, 8, seed=2), synth.grid2d(40, 30, 0.2, seed=1), synth.erdos_renyi(3000, 1.5, seed=3)):
        w = synth.edge_weights(g, 5).numpy()
        F, W = oracle.msf_kruskal(*g.numpy(), w)
        assert abs(W - scipy_msf_weight(g, w)) <= 1e-9 * max(W, 1.0)
        assert oracle.check_forest(*g.numpy(), F) == 0
    # brute force: the lightest acyclic edge set of size n - #components
    rng = np.random.default_rng(11)
    for t in range(60):
        n = int(rng.integers(2, 7))
        allp = list(itertools.combinations(range(n), 2))
        pairs = [p for p in allp if rng.random() < 0.6]
        if not pairs:
            continue
        g = synth.from_edge_list(n, pairs)
        wd = {frozenset(p): float(np.float32(rng.random() + 0.01)) for p in pairs}
        off, edg = g.numpy()
        src = np.repeat(np.arange(n), np.diff(off))
        w = np.array([wd[frozenset((int(a), int(b)))] for a, b in zip(src, edg)], dtype=np.float32)
        k = n - len(np.unique(closure_labels(n, pairs)))
        best = min(sum(wd[frozenset(p)] for p in sub) for sub in itertools.combinations(pairs, k)
                   if len(np.unique(closure_labels(n, list(sub)))) == n - k)
        _, W = oracle.msf_kruskal(off, edg, w)
        assert abs(W - best) <= 1e-6


@pytest.mark.parametrize("eps", [0.01, 0.25, 1.0, 4.0])
def test_amsf_within_its_bound(eps):
    for g in (synth.rmat(11, 8, seed=4), synth.grid2d(50, 40, 0.3, seed=2)):
        off, edg = g.numpy()
        w = synth.edge_weights(g, 9).numpy()
        _, opt = oracle.msf_kruskal(off, edg, w)
        F, W = oracle.amsf(off, edg, w, eps)
        assert oracle.check_forest(off, edg, F) == 0
        assert opt * (1 - 1e-9) <= W <= (1 + eps) * opt * (1 + 1e-9)


def amsf_bucket(w, eps):
    """Bucket index of each weight: floor(log(w / Wmin) / log(1 + eps)) in
    double, the index of the interval [Wmin(1+eps)^i, Wmin(1+eps)^(i+1))
    holding w (Section 5.1)."""
    w = np.asarray(w, dtype=np.float64)
    return np.maximum(0, np.floor(np.log(w / w.min()) / np.log1p(eps))).astype(np.int64)


def forest_bucket_counts(off, edg, w, F, eps):
    """Forest edges per bucket (cumulative), with each pair's weight looked up
    in the graph, against the rank of the subgraph of buckets <= i."""
    src = np.repeat(np.arange(len(off) - 1), np.diff(off))
    b = amsf_bucket(w, eps)
    key = {(int(a), int(c)): int(x) for a, c, x in zip(src, edg, b)}
    fb = np.array([key[(int(a), int(c))] for a, c in F], dtype=np.int64)
    nb = int(b.max()) + 1 if b.size else 0
    got = np.cumsum(np.bincount(fb, minlength=nb)) if nb else np.zeros(0, np.int64)
    rank = np.zeros(nb, dtype=np.int64)
    n = len(off) - 1
    for i in range(nb):
        keep = b <= i
        lab = scipy_labels(n, src[keep], edg[keep].astype(np.int64))
        rank[i] = n - len(np.unique(lab))
    return got, rank


@pytest.mark.parametrize("eps", [0.05, 0.5, 2.0])
def test_amsf_per_bucket_ranks(eps):
    # after bucket i the forest spans the subgraph of buckets <= i, so the
    # forest edges of buckets <= i number n - #components of that subgraph
    for g in (synth.rmat(10, 8, seed=4), synth.grid2d(30, 20, 0.3, seed=2), synth.cliques([3, 7, 1, 12])):
        off, edg = g.numpy()
        w = synth.edge_weights(g, 5).numpy()
        F, _ = oracle.amsf(off, edg, w, eps)
        got, rank = forest_bucket_counts(off, edg, w, F, eps)
        assert np.array_equal(got, rank)


def test_amsf_per_bucket_counts_catch_a_wrong_order():
    # visiting the heaviest bucket first (a planted mistake, applied here to
    # the oracle's inputs by reversing the weight order) breaks the counts
    g = synth.rmat(9, 8, seed=3)
    off, edg = g.numpy()
    w = synth.edge_weights(g, 6).numpy()
    F, _ = oracle.amsf(off, edg, (1.0 / w).astype(np.float32), 0.25)
    got, rank = forest_bucket_counts(off, edg, w, F, 0.25)
    assert not np.array_equal(got, rank)


def test_amsf_closed_forms():
    g = synth.rmat(10, 8, seed=7)
    off, edg = g.numpy()
    w = synth.edge_weights(g, 2).numpy()
    # buckets thinner than any weight gap: Kruskal's order, the exact weight
    _, opt = oracle.msf_kruskal(off, edg, w)
    _, W = oracle.amsf(off, edg, w, 1e-9)
    assert abs(W - opt) <= 1e-9 * opt
    # equal weights: every spanning forest is minimum, one bucket
    ones = np.ones(g.m, np.float32)
    F, W = oracle.amsf(off, edg, ones, 0.25)
    assert W == len(F) == oracle.cc_uf(off, edg)[1]
