"""CPU oracle for ConnectIt's connectivity path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain sequential C, see
its header for the passage each function follows) through ctypes, on numpy
arrays.  It shares no code with the CUDA path and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF
SAMPLE = {"none": 0, "kout": 1, "bfs": 2, "ldd": 3}
KOUT_RULE = {"hybrid": 0, "afforest": 1, "pure": 2}
# every union-find option of Algorithm 7's meta-algorithm (Union = Async,
# Hooks, Early or Rem-CAS, any find / splice) reaches the same sequential
# union-find result, so they share the oracle's one union-find finish
FINISH = {"uf_rem_cas": 0, "uf_async": 1, "sv": 2, "lt_prf": 3, "uf_hooks": 0, "uf_early": 0}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            c = ctypes
            L.oracle_draw.restype = c.c_uint64
            L.oracle_draw.argtypes = [c.c_uint64, c.c_uint64]
            L.oracle_cc_uf.restype = c.c_uint64
            L.oracle_cc_uf.argtypes = [c.c_uint32, u64p, u32p, u32p]
            L.oracle_uf_prefix.restype = c.c_uint64
            L.oracle_uf_prefix.argtypes = [c.c_uint32, u64p, u32p, c.c_uint32, u32p]
            L.oracle_cc_bfs.restype = c.c_int
            L.oracle_cc_bfs.argtypes = [c.c_uint32, u64p, u32p, u32p]
            L.oracle_identify_frequent.restype = c.c_uint32
            L.oracle_identify_frequent.argtypes = [c.c_uint32, u32p, c.c_uint32, c.c_uint64, u64p]
            L.oracle_kout_pick.restype = c.c_uint32
            L.oracle_kout_pick.argtypes = [u64p, u32p, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64, c.c_int]
            L.oracle_kout_sample.restype = None
            L.oracle_kout_sample.argtypes = [c.c_uint32, u64p, u32p, c.c_uint32, c.c_uint64, c.c_int, u32p]
            L.oracle_bfs_sample.restype = c.c_int
            L.oracle_bfs_sample.argtypes = [c.c_uint32, u64p, u32p, c.c_uint32, c.c_uint64, u32p]
            L.oracle_ldd_schedule.restype = c.c_uint64
            L.oracle_ldd_schedule.argtypes = [c.c_uint32, c.c_double, c.c_uint32]
            L.oracle_ldd_sample.restype = c.c_int
            L.oracle_ldd_sample.argtypes = [c.c_uint32, u64p, u32p, c.c_double, u32p]
            L.oracle_finish_uf.restype = c.c_uint64
            L.oracle_finish_uf.argtypes = [c.c_uint32, u64p, u32p, u32p, c.c_uint32]
            L.oracle_finish_sv.restype = c.c_int
            L.oracle_finish_sv.argtypes = [c.c_uint32, u64p, u32p, u32p, c.c_uint32]
            L.oracle_finish_lt_prf.restype = c.c_int
            L.oracle_finish_lt_prf.argtypes = [c.c_uint32, u64p, u32p, u32p, c.c_uint32]
            L.oracle_connectivity.restype = c.c_int
            L.oracle_connectivity.argtypes = [c.c_uint32, u64p, u32p, c.c_int, c.c_uint32, c.c_int, c.c_uint32,
                                              c.c_double, c.c_uint64, c.c_uint32, c.c_int, u32p, u64p]
            L.oracle_incr_insert.restype = None
            L.oracle_incr_insert.argtypes = [c.c_uint32, u32p, u32p, c.c_uint64]
            L.oracle_incr_query.restype = None
            L.oracle_incr_query.argtypes = [c.c_uint32, u32p, u32p, c.c_uint64, u8p]
            L.oracle_incr_labels.restype = None
            L.oracle_incr_labels.argtypes = [c.c_uint32, u32p, u32p]
            L.oracle_spanning_forest.restype = c.c_uint64
            L.oracle_spanning_forest.argtypes = [c.c_uint32, u64p, u32p, u32p]
            fp = ctypes.POINTER(ctypes.c_float)
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_msf_kruskal.restype = c.c_uint64
            L.oracle_msf_kruskal.argtypes = [c.c_uint32, u64p, u32p, fp, u32p, dp]
            L.oracle_amsf.restype = c.c_uint64
            L.oracle_amsf.argtypes = [c.c_uint32, u64p, u32p, fp, c.c_double, u32p, dp]
            L.oracle_check_forest.restype = c.c_int
            L.oracle_check_forest.argtypes = [c.c_uint32, u64p, u32p, u32p, c.c_uint64, u32p]
            _lib = L
    return _lib


def _u32(a):
    a = np.ascontiguousarray(np.asarray(a).astype(np.uint32, copy=False))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64(a):
    a = np.ascontiguousarray(np.asarray(a).astype(np.uint64, copy=False))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _graph(offsets, edges):
    I, Ip = _u64(offsets)
    A, Ap = _u32(edges)
    n = I.shape[0] - 1
    return n, (I, Ip), (A, Ap)


def _as_np(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return x.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(x)


def draw(seed: int, ctr: int) -> int:
    return int(lib().oracle_draw(seed, ctr))


def cc_uf(offsets, edges):
    """O1: canonical min-id labels by sequential union-find; also #links."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    links = lib().oracle_cc_uf(n, Ip, Ap, lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return lab, int(links)


def uf_prefix(offsets, edges, u_end: int, P=None):
    """O1's union loop over the edges of vertices [0, u_end) (a bounded slice
    for timing).  Returns (forest P, edges processed)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    if P is None:
        P = np.arange(n, dtype=np.uint32)
    cnt = lib().oracle_uf_prefix(n, Ip, Ap, u_end, P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return P, int(cnt)


def cc_bfs(offsets, edges):
    """O2: canonical min-id labels by BFS (independent of O1)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    rc = lib().oracle_cc_bfs(n, Ip, Ap, lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert rc == 0
    return lab


def identify_frequent(labels, samples: int = 0, seed: int = 0):
    L, Lp = _u32(_as_np(labels))
    cnt = ctypes.c_uint64(0)
    lm = lib().oracle_identify_frequent(L.shape[0], Lp, samples, seed, ctypes.byref(cnt))
    return int(lm), int(cnt.value)


def kout_pick(offsets, edges, v: int, k: int, j: int, seed: int, rule: str = "hybrid") -> int:
    """Pick j of vertex v under the selection rule (NONE: no pick)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    return int(lib().oracle_kout_pick(Ip, Ap, v, k, j, seed, KOUT_RULE[rule]))


def kout_sample(offsets, edges, k: int = 2, seed: int = 1, rule: str = "hybrid"):
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    lib().oracle_kout_sample(n, Ip, Ap, k, seed, KOUT_RULE[rule], lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return lab


def bfs_sample(offsets, edges, tries: int = 3, seed: int = 1):
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    t = lib().oracle_bfs_sample(n, Ip, Ap, tries, seed, lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return lab, int(t)


def ldd_schedule(n: int, beta: float, r: int) -> int:
    return int(lib().oracle_ldd_schedule(n, beta, r))


def ldd_sample(offsets, edges, beta: float = 0.2):
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    r = lib().oracle_ldd_sample(n, Ip, Ap, beta, lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return lab, int(r)


def finish(offsets, edges, labels, lmax: int, kind: str = "uf_rem_cas"):
    """Apply one finish method to sampled labels; returns (labels, stat)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.array(_as_np(labels), dtype=np.uint32, copy=True)
    lp = lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    L = lib()
    if kind in ("uf_rem_cas", "uf_async", "uf_hooks", "uf_early"):
        st = L.oracle_finish_uf(n, Ip, Ap, lp, lmax)
    elif kind == "sv":
        st = L.oracle_finish_sv(n, Ip, Ap, lp, lmax)
    elif kind == "lt_prf":
        st = L.oracle_finish_lt_prf(n, Ip, Ap, lp, lmax)
    else:
        raise ValueError(kind)
    return lab, int(st)


def connectivity(offsets, edges, sample: str = "none", finish: str = "uf_rem_cas", k: int = 2,
                 tries: int = 3, beta: float = 0.2, seed: int = 1, freq_samples: int = 0, kout_rule: str = "hybrid"):
    """Algorithm 1: labels and stats dict (lmax, applied, rounds, sample_info)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    lab = np.empty(n, np.uint32)
    st = np.zeros(4, np.uint64)
    rc = lib().oracle_connectivity(n, Ip, Ap, SAMPLE[sample], k, KOUT_RULE[kout_rule], tries, beta, seed, freq_samples,
                                   FINISH[finish], lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    assert rc == 0
    return lab, {"lmax": int(st[0]), "applied": int(st[1]), "rounds": int(st[2]),
                 "sample_info": int(np.int64(st[3].astype(np.int64)))}


class Incremental:
    """O3: union-find forest kept across batches (inserts, then queries)."""

    def __init__(self, offsets, edges):
        self.P, _ = cc_uf(offsets, edges)
        self.n = self.P.shape[0]

    def insert(self, pairs):
        pr, pp = _u32(_as_np(pairs).reshape(-1))
        lib().oracle_incr_insert(self.n, self.P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), pp,
                                 pr.shape[0] // 2)

    def query(self, pairs):
        pr, pp = _u32(_as_np(pairs).reshape(-1))
        ans = np.empty(pr.shape[0] // 2, np.uint8)
        lib().oracle_incr_query(self.n, self.P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), pp,
                                pr.shape[0] // 2, ans.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return ans

    def labels(self):
        lab = np.empty(self.n, np.uint32)
        lib().oracle_incr_labels(self.n, self.P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        return lab


def spanning_forest(offsets, edges):
    """Spanning forest by sequential union-find: uint32[count, 2] pairs."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    out = np.empty(2 * max(n - 1, 1), np.uint32)
    cnt = lib().oracle_spanning_forest(n, Ip, Ap, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out[: 2 * cnt].reshape(-1, 2)


FOREST_CHECK = {0: "ok", 1: "endpoint out of range", 2: "not an edge of G", 3: "closes a cycle",
                4: "joins two components of G", 5: "does not span a component"}


def check_forest(offsets, edges, pairs, labels=None) -> int:
    """0 if `pairs` (uint32[count, 2]) is a spanning forest of G, else the
    code of the first failed property (FOREST_CHECK).  `labels` are G's
    canonical labels (computed by O1 when not given)."""
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    if labels is None:
        labels, _ = cc_uf(I, A)
    L, Lp = _u32(_as_np(labels))
    pr, pp = _u32(_as_np(pairs).reshape(-1))
    return int(lib().oracle_check_forest(n, Ip, Ap, pp, pr.size // 2, Lp))


def _forest_call(fn, offsets, edges, weights, *extra):
    n, (I, Ip), (A, Ap) = _graph(_as_np(offsets), _as_np(edges))
    W = np.ascontiguousarray(np.asarray(_as_np(weights), dtype=np.float32))
    out = np.empty(2 * max(n - 1, 1), np.uint32)
    wt = ctypes.c_double(0.0)
    cnt = fn(n, Ip, Ap, W.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), *extra,
             out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ctypes.byref(wt))
    return out[: 2 * cnt].reshape(-1, 2), wt.value


def msf_kruskal(offsets, edges, weights):
    """Exact minimum spanning forest: (pairs uint32[count, 2], total weight)."""
    return _forest_call(lib().oracle_msf_kruskal, offsets, edges, weights)


def amsf(offsets, edges, weights, eps: float):
    """Approximate MSF by weight buckets of ratio 1 + eps: (pairs, weight)."""
    return _forest_call(lib().oracle_amsf, offsets, edges, weights, ctypes.c_double(eps))
