"""Seeded synthetic graph generators (test and benchmark inputs).

This module is shared by the oracle's tests and by the CUDA path's tests and
benchmark.  It holds none of the connectivity method's arithmetic: it only
draws graphs and lays them out as a symmetric CSR (offsets ``I``, edges ``A``;
the incident edges of ``v`` are ``A[I[v]:I[v+1]]`` and ``I[n] = m``, the
layout of the paper's Section 2), with self-loops and duplicate edges removed
and every adjacency list sorted ascending.

Every generator is a pure function of its arguments and seed.  Randomness
comes from a 32-bit integer mixing hash evaluated on (seed, stream, index)
counters with torch integer ops, so the same call gives the same graph on the
CPU and on a CUDA device (generation of the large workloads runs on the GPU,
where it takes seconds; the small ones run on the CPU).

Workload shapes (the paper's datasets are not available; these stand in for
them, shaped like its power-law social/web graphs, its high-diameter road
network and a sparse near-percolation graph):

* ``rmat``   -- R-MAT (Chakrabarti et al.), ``scale`` quadrant draws per edge
  with probabilities (a, b, c, d), no noise, no vertex permutation; the
  generator of the paper's streaming RMAT inputs (Section 4.5).
* ``grid2d`` -- w x h 4-neighbour grid, each undirected edge dropped
  independently with probability ``p_drop`` (road-network stand-in).
* ``erdos_renyi`` -- G(n, M) with M = round(avg_deg * n / 2) uniform pairs.
* small closed-form families used as pins: paths, stars, disjoint cliques,
  the Appendix B.2 counter-example graph, and vertex relabelling.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

M32 = 0xFFFFFFFF
_GOLDEN = 0x9E3779B9


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for x in [0, 2^32) without int64 overflow."""
    lo = x & 0xFFFF
    hi = x >> 16
    return (lo * c + (((hi * c) & 0xFFFF) << 16)) & M32


def mix32(x: torch.Tensor) -> torch.Tensor:
    """A 32-bit avalanche mixer (xorshift-multiply, 'lowbias32' constants)."""
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def hash3(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform 32-bit value for counter ``idx`` (int64 >= 0) of ``stream``."""
    k0 = ((seed & M32) ^ (((seed >> 32) * 3) & M32) ^ ((stream * _GOLDEN) & M32)) & M32
    key = mix32(torch.tensor(k0, dtype=torch.int64, device=idx.device))
    lo = idx & M32
    hi = idx >> 32
    return mix32(mix32(lo ^ key) ^ mix32(hi + 0x632BE5AB))


@dataclass
class CSR:
    """Symmetric CSR graph: ``offsets`` int64[n+1], ``edges`` int32[m]."""
    n: int
    offsets: torch.Tensor
    edges: torch.Tensor
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.edges.numel())

    def to(self, device) -> "CSR":
        return CSR(self.n, self.offsets.to(device), self.edges.to(device), self.name)

    def offsets_u32(self) -> torch.Tensor:
        assert self.m < 2**31, "graph too large for 32-bit offsets"
        return self.offsets.to(torch.int32)

    def numpy(self):
        return self.offsets.cpu().numpy(), self.edges.cpu().numpy()


def _csr_from_keys(n: int, keys: torch.Tensor, device) -> tuple[torch.Tensor, torch.Tensor]:
    """keys = u * 2^32 + v, sorted and unique -> (offsets int64[n+1], edges int32[m])."""
    src = keys >> 32
    edges = (keys & M32).to(torch.int32)
    counts = torch.bincount(src, minlength=n) if keys.numel() else torch.zeros(n, dtype=torch.int64, device=device)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=offsets[1:])
    return offsets, edges


def from_pairs(n: int, u: torch.Tensor, v: torch.Tensor, name: str = "", max_sort: int = 1 << 29) -> CSR:
    """Symmetrise, drop self-loops and duplicates, sort, and build a CSR.

    Large inputs are processed in source-vertex ranges, each sorted on its own,
    so that no single sort holds more than ``max_sort`` keys.
    """
    device = u.device
    u = u.to(torch.int64)
    v = v.to(torch.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    if u.numel() == 0:
        return CSR(n, torch.zeros(n + 1, dtype=torch.int64, device=device),
                   torch.zeros(0, dtype=torch.int32, device=device), name)
    total = 2 * u.numel()
    if total <= max_sort:
        keys = torch.cat([u * (1 << 32) + v, v * (1 << 32) + u])
        keys = torch.unique(keys, sorted=True)
        off, edg = _csr_from_keys(n, keys, device)
        return CSR(n, off, edg, name)
    # Range-partitioned build: histogram endpoints by vertex block, then group
    # consecutive blocks into ranges of at most max_sort directed keys.
    nblk = 4096
    bsz = max(1, -(-n // nblk))
    hist = torch.bincount(u // bsz, minlength=nblk) + torch.bincount(v // bsz, minlength=nblk)
    hist = hist.cpu().tolist()
    ranges, lo, acc = [], 0, 0
    for b, c in enumerate(hist):
        if acc + c > max_sort and acc > 0:
            ranges.append((lo * bsz, b * bsz))
            lo, acc = b, 0
        acc += c
    ranges.append((lo * bsz, n))
    edge_parts = []
    counts = torch.zeros(n, dtype=torch.int64, device=device)
    for (r0, r1) in ranges:
        mu = (u >= r0) & (u < r1)
        mv = (v >= r0) & (v < r1)
        keys = torch.cat([u[mu] * (1 << 32) + v[mu], v[mv] * (1 << 32) + u[mv]])
        del mu, mv
        keys = torch.unique(keys, sorted=True)
        src = keys >> 32
        counts[r0:r1] = torch.bincount(src - r0, minlength=r1 - r0)
        edge_parts.append((keys & M32).to(torch.int32))
        del keys, src
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=offsets[1:])
    return CSR(n, offsets, torch.cat(edge_parts), name)


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, device="cpu", chunk: int = 1 << 25) -> CSR:
    """R-MAT graph with n = 2^scale and edge_factor * n generated pairs."""
    n = 1 << scale
    npairs = edge_factor * n
    t_a = int(round(a * 2**32))
    t_ab = int(round((a + b) * 2**32))
    t_abc = int(round((a + b + c) * 2**32))
    us, vs = [], []
    for start in range(0, npairs, chunk):
        cnt = min(chunk, npairs - start)
        idx = torch.arange(start, start + cnt, dtype=torch.int64, device=device)
        state = hash3(seed, 11, idx)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        for lvl in range(scale):
            r = mix32(state ^ ((lvl + 1) * _GOLDEN & M32))
            bu = (r >= t_ab).to(torch.int64)
            bv = (((r >= t_a) & (r < t_ab)) | (r >= t_abc)).to(torch.int64)
            u = (u << 1) | bu
            v = (v << 1) | bv
        us.append(u.to(torch.int32))
        vs.append(v.to(torch.int32))
        del idx, state, u, v
    return from_pairs(n, torch.cat(us), torch.cat(vs), name=f"rmat{scale}_ef{edge_factor}")


def grid2d(w: int, h: int, p_drop: float, seed: int = 1, device="cpu") -> CSR:
    """w x h 4-neighbour grid, row-major ids; each undirected edge kept iff its
    hash is >= p_drop * 2^32."""
    n = w * h
    thr = int(round(p_drop * 2**32))
    nh = (w - 1) * h  # horizontal edges (r, c)-(r, c+1), index r*(w-1)+c
    nv = w * (h - 1)  # vertical edges (r, c)-(r+1, c), index nh + r*w + c
    ih = torch.arange(nh, dtype=torch.int64, device=device)
    keep_h = hash3(seed, 21, ih) >= thr
    ih = ih[keep_h]
    wm = max(w - 1, 1)
    hu = (ih // wm) * w + ih % wm
    hv = hu + 1
    iv = torch.arange(nv, dtype=torch.int64, device=device)
    keep_v = hash3(seed, 21, iv + nh) >= thr
    iv = iv[keep_v]
    vu = iv
    vv = iv + w
    u = torch.cat([hu, vu])
    v = torch.cat([hv, vv])
    return from_pairs(n, u, v, name=f"grid{w}x{h}_p{p_drop}")


def erdos_renyi(n: int, avg_deg: float, seed: int = 1, device="cpu") -> CSR:
    """G(n, M) with M = round(avg_deg * n / 2) uniform vertex pairs."""
    M = int(round(avg_deg * n / 2))
    idx = torch.arange(M, dtype=torch.int64, device=device)
    u = (hash3(seed, 31, idx) * n) >> 32
    v = (hash3(seed, 32, idx) * n) >> 32
    return from_pairs(n, u, v, name=f"er{n}_d{avg_deg}")


def from_edge_list(n: int, pairs, name: str = "", device="cpu") -> CSR:
    """CSR from a Python list of undirected (u, v) pairs."""
    if len(pairs) == 0:
        z = torch.zeros(0, dtype=torch.int64, device=device)
        return from_pairs(n, z, z, name)
    t = torch.tensor(pairs, dtype=torch.int64, device=device).reshape(-1, 2)
    return from_pairs(n, t[:, 0], t[:, 1], name)


def empty(n: int) -> CSR:
    return from_edge_list(n, [], name=f"empty{n}")


def path(n: int) -> CSR:
    return from_edge_list(n, [(i, i + 1) for i in range(n - 1)], name=f"path{n}")


def star(n: int, centre: int = 0) -> CSR:
    return from_edge_list(n, [(centre, i) for i in range(n) if i != centre], name=f"star{n}")


def cliques(sizes) -> CSR:
    """Disjoint cliques laid out consecutively (sizes[0] first)."""
    pairs, base = [], 0
    for s in sizes:
        pairs += [(base + i, base + j) for i in range(s) for j in range(i + 1, s)]
        base += s
    return from_edge_list(base, pairs, name=f"cliques{len(sizes)}")


def counterexample() -> CSR:
    """The six-vertex graph of the Rem's-algorithm counter-example (Appendix
    B.2): one component."""
    return from_edge_list(6, [(0, 2), (1, 3), (2, 5), (3, 4), (4, 5)], name="rem_counterexample")


def relabel(g: CSR, perm: torch.Tensor) -> CSR:
    """Graph with vertex v renamed perm[v]."""
    off, edg = g.offsets.cpu(), g.edges.cpu().to(torch.int64)
    src = torch.repeat_interleave(torch.arange(g.n, dtype=torch.int64), off[1:] - off[:-1])
    p = perm.cpu().to(torch.int64)
    return from_pairs(g.n, p[src], p[edg], name=g.name + "_perm")


def random_perm(n: int, seed: int) -> torch.Tensor:
    keys = hash3(seed, 41, torch.arange(n, dtype=torch.int64)) * (1 << 32) + torch.arange(n)
    return torch.argsort(keys)


def random_pairs(n: int, count: int, seed: int, stream: int, device="cpu") -> torch.Tensor:
    """count uniform vertex pairs as int32[count, 2] (incremental queries)."""
    idx = torch.arange(count, dtype=torch.int64, device=device)
    u = (hash3(seed, stream, idx) * n) >> 32
    v = (hash3(seed, stream + 1, idx) * n) >> 32
    return torch.stack([u, v], 1).to(torch.int32)


def rmat_pairs(scale: int, count: int, seed: int, stream: int, a=0.57, b=0.19, c=0.19,
               device="cpu") -> torch.Tensor:
    """count R-MAT-distributed vertex pairs as int32[count, 2] (incremental inserts)."""
    t_a = int(round(a * 2**32))
    t_ab = int(round((a + b) * 2**32))
    t_abc = int(round((a + b + c) * 2**32))
    idx = torch.arange(count, dtype=torch.int64, device=device)
    state = hash3(seed, stream, idx)
    u = torch.zeros(count, dtype=torch.int64, device=device)
    v = torch.zeros(count, dtype=torch.int64, device=device)
    for lvl in range(scale):
        r = mix32(state ^ ((lvl + 1) * _GOLDEN & M32))
        u = (u << 1) | (r >= t_ab).to(torch.int64)
        v = (v << 1) | (((r >= t_a) & (r < t_ab)) | (r >= t_abc)).to(torch.int64)
    return torch.stack([u, v], 1).to(torch.int32)


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int, stream: int) -> list[int]:
    """count integers log-uniform in [lo, hi] (batch sizes, graph sizes)."""
    h = hash3(seed, stream, torch.arange(count, dtype=torch.int64)).to(torch.float64) / 2**32
    vals = torch.exp(math.log(lo) + h * (math.log(hi) - math.log(lo)))
    return [int(round(x)) for x in vals.tolist()]


def pack(graphs):
    """Pack graphs into one CSR with per-graph vertex offsets: returns
    (gv int64[G+1], offsets int64[V+1] with global edge positions, edges
    int32[M] holding each graph's LOCAL vertex ids)."""
    nv = [g.n for g in graphs]
    gv = torch.zeros(len(graphs) + 1, dtype=torch.int64)
    gv[1:] = torch.cumsum(torch.tensor(nv, dtype=torch.int64), 0)
    offs, edgs, ebase = [torch.zeros(1, dtype=torch.int64)], [], 0
    for g in graphs:
        o = g.offsets.cpu()
        offs.append(o[1:] + ebase)
        edgs.append(g.edges.cpu())
        ebase += g.m
    return gv, torch.cat(offs), (torch.cat(edgs) if edgs else torch.zeros(0, dtype=torch.int32))


def batch_config3(count: int, seed: int = 1, lo: int = 6, hi: int = 16):
    """The batched workload: graph sizes log-uniform in [2^lo, 2^hi]; even
    indices G(n, M) with average degree uniform in [0.5, 4], odd indices
    w x h grids (w = floor(sqrt(n)), h = floor(n / w)) with drop probability
    uniform in [0, 0.5]."""
    sizes = log_uniform_sizes(count, 2.0 ** lo, 2.0 ** hi, seed, 500)
    u = hash3(seed, 501, torch.arange(count, dtype=torch.int64)).to(torch.float64) / 2**32
    graphs = []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            graphs.append(erdos_renyi(n, 0.5 + 3.5 * float(u[i]), seed=seed * 100003 + i))
        else:
            w = max(1, int(math.isqrt(n)))
            h = max(1, n // w)
            graphs.append(grid2d(w, h, 0.5 * float(u[i]), seed=seed * 100003 + i))
    return graphs


def cliques_fast(sizes, device="cpu") -> CSR:
    """Disjoint cliques (vectorised): clique i occupies ids [sum(sizes[:i]), ...)."""
    sizes = [int(s) for s in sizes]
    base = 0
    us, vs = [], []
    by_size = {}
    for s in sizes:
        by_size.setdefault(s, []).append(base)
        base += s
    for s, starts in by_size.items():
        if s < 2:
            continue
        iu = torch.triu_indices(s, s, 1, device=device)
        st = torch.tensor(starts, dtype=torch.int64, device=device)[:, None]
        us.append((st + iu[0][None, :]).reshape(-1))
        vs.append((st + iu[1][None, :]).reshape(-1))
    if not us:
        z = torch.zeros(0, dtype=torch.int64, device=device)
        return from_pairs(base, z, z, name="cliques")
    return from_pairs(base, torch.cat(us), torch.cat(vs), name="cliques")


def selector_graph(i: int, seed: int = 1, scale_lo: int = 14, scale_hi: int = 22, device="cpu") -> CSR:
    """Graph i of the selector's training / held-out families (seeded):
    i % 4 == 0 RMAT with a in [0.45, 0.65], b = c = (1 - a - 0.05) / 2 and
    edge factor 4, 8 or 16; 1 a grid with drop probability in [0, 0.5];
    2 G(n, M) with average degree in [0.5, 8]; 3 disjoint cliques of 4-64
    vertices.  Scales (log2 n) uniform in [scale_lo, scale_hi]."""
    u = hash3(seed, 700 + i % 4, torch.tensor([i, i + 1_000_003, i + 2_000_006], dtype=torch.int64))
    r = (u.to(torch.float64) / 2**32).tolist()
    scale = scale_lo + min(scale_hi - scale_lo, int(r[0] * (scale_hi - scale_lo + 1)))
    gseed = seed * 1_000_003 + i
    fam = i % 4
    if fam == 0:
        a = 0.45 + 0.2 * r[1]
        bc = (1.0 - a - 0.05) / 2
        ef = (4, 8, 16)[int(r[2] * 3) % 3]
        return rmat(scale, ef, a=a, b=bc, c=bc, seed=gseed, device=device)
    n = 1 << scale
    if fam == 1:
        w = max(1, int(math.isqrt(n)))
        return grid2d(w, max(1, n // w), 0.5 * r[1], seed=gseed, device=device)
    if fam == 2:
        return erdos_renyi(n, 0.5 + 7.5 * r[1], seed=gseed, device=device)
    cnt = max(1, n // 34)
    sz = (4 + (hash3(gseed, 710, torch.arange(cnt, dtype=torch.int64)) % 61)).tolist()
    return cliques_fast(sz, device=device)


def edge_weights(g: CSR, seed: int = 1) -> torch.Tensor:
    """float32[m] weights for g's CSR entries, exponential with mean 1 (the
    paper's weighted inputs draw exponential weights with a constant mean),
    equal on both stored copies of an undirected edge: the draw hashes
    (min(u, v), max(u, v))."""
    off = g.offsets
    src = torch.repeat_interleave(torch.arange(g.n, dtype=torch.int64, device=off.device), off[1:] - off[:-1])
    dst = g.edges.to(torch.int64)
    key = torch.minimum(src, dst) * (1 << 32) + torch.maximum(src, dst)
    del src, dst
    h = hash3(seed, 41, key).to(torch.float64)
    u = (h + 0.5) / 2.0**32
    return (-torch.log(u)).to(torch.float32)
