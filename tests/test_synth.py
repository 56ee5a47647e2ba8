"""The seeded input generators shared by the oracle and the CUDA path
(no GPU): every graph is a symmetric CSR with sorted adjacency, no
self-loops and no duplicates; the shapes follow the recipe the inputs
stand in for (R-MAT skew, the dropped grid's edge count, G(n, M)'s edge
count, log-uniform batch sizes), and a seed fixes the graph."""
import math

import numpy as np
import pytest

import synth


def _check_csr(g):
    off, edg = g.numpy()
    assert off[0] == 0 and off[-1] == len(edg) == g.m
    assert np.all(np.diff(off) >= 0)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(off))
    dst = edg.astype(np.int64)
    assert np.all(dst < g.n)
    assert not np.any(src == dst), "self-loop"
    for v in range(0, g.n, max(1, g.n // 200)):   # sorted, duplicate-free adjacency
        a = edg[off[v]:off[v + 1]].astype(np.int64)
        assert np.all(np.diff(a) > 0)
    fwd = set(zip(src.tolist(), dst.tolist()))
    assert all((b, a) in fwd for a, b in fwd), "not symmetric"
    return off, edg


@pytest.mark.parametrize("make", [lambda: synth.rmat(12, 8, seed=3), lambda: synth.grid2d(40, 30, 0.3, seed=2),
                                  lambda: synth.erdos_renyi(5000, 1.2, seed=4), lambda: synth.cliques([3, 1, 7]),
                                  lambda: synth.star(50, centre=7), lambda: synth.path(33)])
def test_graphs_are_symmetric_simple_sorted(make):
    _check_csr(make())


def test_seed_fixes_the_graph():
    a, b, c = synth.rmat(11, 8, seed=5), synth.rmat(11, 8, seed=5), synth.rmat(11, 8, seed=6)
    assert np.array_equal(a.numpy()[1], b.numpy()[1])
    assert not np.array_equal(a.numpy()[1], c.numpy()[1])


def test_grid_edge_counts():
    w, h = 50, 40
    full = synth.grid2d(w, h, 0.0, seed=1)
    assert full.m == 2 * (w * (h - 1) + h * (w - 1))
    dropped = synth.grid2d(w, h, 0.3, seed=1)
    und = w * (h - 1) + h * (w - 1)
    kept = dropped.m // 2
    # each undirected edge kept with probability 0.7: within 5 standard deviations
    assert abs(kept - 0.7 * und) <= 5 * math.sqrt(und * 0.21)


def test_erdos_renyi_edge_count():
    n, d = 20000, 1.2
    g = synth.erdos_renyi(n, d, seed=2)
    M = round(d * n / 2)
    # G(n, M) pairs after dropping loops and duplicates: at most M undirected edges, few lost
    assert 0.99 * M <= g.m // 2 <= M


def test_rmat_is_skewed():
    g = synth.rmat(14, 8, seed=1)
    deg = np.diff(g.numpy()[0])
    # (0.57, 0.19, 0.19, 0.05): low ids collect the edges; many vertices are isolated
    assert deg[: g.n // 16].sum() > deg[g.n // 2:].sum()
    assert deg.max() > 50 * max(1.0, deg.mean())
    assert (deg == 0).sum() > g.n // 10


def test_log_uniform_batch_sizes():
    s = np.array(synth.log_uniform_sizes(2000, 1e3, 1e7, seed=3, stream=50), dtype=np.float64)
    assert s.min() >= 1e3 and s.max() <= 1e7
    # log10 of a log-uniform draw on [3, 7] has mean 5
    assert abs(np.log10(s).mean() - 5.0) < 0.15


def test_edge_weights_are_symmetric_and_positive():
    g = synth.grid2d(20, 20, 0.2, seed=1)
    off, edg = g.numpy()
    w = synth.edge_weights(g, 1).numpy()
    assert np.all(w > 0)
    src = np.repeat(np.arange(g.n), np.diff(off))
    wt = {(int(a), int(b)): float(x) for a, b, x in zip(src, edg, w)}
    assert all(wt[(b, a)] == x for (a, b), x in wt.items())
