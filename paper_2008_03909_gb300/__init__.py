"""GB300-native ConnectIt connectivity: Python binding of ``libconnectit_gb``.

Argument marshalling only: every step of the connectivity path runs in the
library's CUDA kernels (``csrc/``).  PyTorch supplies device memory and
streams.  The functions mirror the C ABI of ``include/connectit_gb.h``:

* ``cc_static``            -- Algorithm 1 (sampling, IdentifyFrequent, finish)
* ``cc_static_host``       -- the same on host buffers (copies included)
* ``cc_sample`` / ``cc_identify_frequent`` / ``cc_finish`` -- its phases
* ``Incremental``          -- ``cc_incr_create`` / ``_insert_batch`` /
  ``_query_batch`` / ``_labels`` / ``_destroy``

There is no CPU fallback: if the library cannot be loaded, or a tensor is
not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libconnectit_gb.so")

SAMPLE = {"none": 0, "kout": 1, "bfs": 2, "ldd": 3}
FINISH = {"uf_rem_cas": 0, "uf_async": 1, "sv": 2, "lt_prf": 3, "uf_hooks": 4, "uf_early": 5, "liu_tarjan": 6,
          "stergiou": 7, "label_prop": 8}
# the sixteen Liu-Tarjan variants: connect (C/P/E), update (U/R), shortcut
# (S one step / F full), A = alter
LT_VARIANTS = {name: {"C": 0, "P": 1, "E": 2}[name[0]] | (4 if name[1] == "R" else 0) |
               (8 if name[2] == "F" else 0) | (16 if name.endswith("A") else 0)
               for name in ("CUSA", "CRSA", "PUSA", "PRSA", "PUS", "PRS", "EUSA", "EUS",
                            "CUFA", "CRFA", "PUFA", "PRFA", "PUF", "PRF", "EUFA", "EUF")}
FIND = {"naive": 0, "split": 1, "halve": 2, "compress": 3}
SPLICE = {"split_one": 0, "halve_one": 1, "atomic": 2}
KOUT_RULE = {"hybrid": 0, "afforest": 1, "pure": 2}
NONE = 0xFFFFFFFF

STATUS = {0: "CC_OK", 1: "CC_ERR_INVALID", 2: "CC_ERR_OOM", 3: "CC_ERR_CUDA", 4: "CC_ERR_NONCONVERGED",
          5: "CC_ERR_BAD_INPUT", 6: "CC_ERR_UNSUPPORTED"}


class CCError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class SampleOpt(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_uint32), ("bfs_tries", ctypes.c_uint32),
                ("ldd_beta", ctypes.c_float), ("seed", ctypes.c_uint64), ("freq_samples", ctypes.c_uint32),
                ("kout_rule", ctypes.c_uint32)]


class FinishOpt(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("find", ctypes.c_int32), ("splice", ctypes.c_int32),
                ("lt_rules", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]


class BatchOpt(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("smem_max_vertices", ctypes.c_uint32),
                ("vertex_mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ServerOpt(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("slot_pairs", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_uint32), ("sample_info", ctypes.c_int32), ("rounds", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("edges_finish", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "cc_default_opts": (None, [ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt)]),
    "cc_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt), ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "cc_static_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt),
                                    ctypes.c_void_p, ctypes.POINTER(Stats), ctypes.c_void_p]),
    "cc_spanning_forest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt),
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "cc_amsf": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                               ctypes.c_uint64, ctypes.c_float, ctypes.c_int, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                               ctypes.c_void_p]),
    "cc_selftest_grid_barrier": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                                ctypes.c_void_p]),
    "cc_static_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt),
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "cc_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.POINTER(SampleOpt), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                 ctypes.c_void_p]),
    "cc_identify_frequent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "cc_identify_frequent_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                                    ctypes.c_void_p]),
    "cc_finish": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.POINTER(FinishOpt), ctypes.c_uint32, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p]),
    "cc_batch_default_opt": (None, [ctypes.POINTER(BatchOpt)]),
    "cc_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(BatchOpt), ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "cc_batched_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.POINTER(BatchOpt), ctypes.POINTER(ctypes.c_float),
                                           ctypes.c_void_p]),
    "cc_incr_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.POINTER(SampleOpt), ctypes.POINTER(FinishOpt),
                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "cc_incr_insert_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "cc_incr_query_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "cc_incr_labels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cc_incr_num_vertices": (ctypes.c_uint32, [ctypes.c_void_p]),
    "cc_incr_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "cc_server_default_opt": (None, [ctypes.POINTER(ServerOpt)]),
    "cc_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerOpt), ctypes.POINTER(ctypes.c_void_p)]),
    "cc_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "cc_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "cc_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "cc_map_edges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "cc_gather_edges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cc_random_sectors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "cc_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "cc_select_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.c_void_p]),
    "cc_mlp_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "cc_mlp_set_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "cc_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "cc_mlp_soft_targets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "cc_mlp_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "cc_mlp_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p]),
    "cc_mlp_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "cc_device_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "cc_set_iteration_cap": (None, [ctypes.c_uint64]),
    "cc_profile_enable": (None, [ctypes.c_int]),
    "cc_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "cc_launch_count": (ctypes.c_uint64, []),
    "cc_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "cc_version": (ctypes.c_char_p, []),
    "cc_binary_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
}


def lib():
    """Load (building first if needed) the CUDA library.  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, what: str):
    if status != 0:
        raise CCError(status, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t: torch.Tensor, dtypes, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor (no CPU fallback)")
    if t.dtype not in dtypes:
        raise TypeError(f"{what}: dtype {t.dtype} not in {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t


def sample_opt(kind="kout", k=2, bfs_tries=3, ldd_beta=0.2, seed=1, freq_samples=0, kout_rule="hybrid") -> SampleOpt:
    return SampleOpt(SAMPLE[kind] if isinstance(kind, str) else kind, k, bfs_tries, ldd_beta, seed, freq_samples,
                     KOUT_RULE[kout_rule] if isinstance(kout_rule, str) else kout_rule)


def finish_opt(kind="uf_rem_cas", find="naive", splice="split_one", lt_rules=0) -> FinishOpt:
    """kind may also name a Liu-Tarjan variant ("PRS", "CUFA", ...)."""
    if isinstance(kind, str) and kind in LT_VARIANTS:
        kind, lt_rules = "liu_tarjan", LT_VARIANTS[kind]
    return FinishOpt(FINISH[kind] if isinstance(kind, str) else kind, FIND[find] if isinstance(find, str) else find,
                     SPLICE[splice] if isinstance(splice, str) else splice, lt_rules)


def _graph_args(offsets: torch.Tensor, edges: torch.Tensor):
    _dev(offsets, (torch.int32, torch.int64), "offsets")
    _dev(edges, (torch.int32,), "edges")
    n = offsets.numel() - 1
    return (ctypes.c_void_p(offsets.data_ptr()), 1 if offsets.dtype == torch.int64 else 0,
            ctypes.c_void_p(edges.data_ptr() if edges.numel() else 0), n, edges.numel())


def cc_static(offsets, edges, sample: SampleOpt | None = None, finish: FinishOpt | None = None,
              labels_out: torch.Tensor | None = None, stream=None, stats: bool = False):
    """Canonical min-id labels (int32 view of uint32) on the offsets' device.
    With stats=True also returns a dict of counters (and synchronises)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    _dev(labels_out, (torch.int32,), "labels_out")
    so = sample if sample is not None else sample_opt()
    fo = finish if finish is not None else finish_opt()
    L = lib()
    if stats:
        st = Stats()
        _check(L.cc_static_ex(Ip, u64, Ap, n, m, ctypes.byref(so), ctypes.byref(fo),
                              ctypes.c_void_p(labels_out.data_ptr()), ctypes.byref(st), _stream(stream)),
               "cc_static_ex")
        return labels_out, {"lmax": st.lmax, "sample_info": st.sample_info, "rounds": st.rounds,
                            "edges_finish": st.edges_finish}
    _check(L.cc_static(Ip, u64, Ap, n, m, ctypes.byref(so), ctypes.byref(fo), ctypes.c_void_p(labels_out.data_ptr()),
                       _stream(stream)), "cc_static")
    return labels_out


def cc_spanning_forest(offsets, edges, sample: SampleOpt | None = None, finish: FinishOpt | None = None,
                       forest_out: torch.Tensor | None = None, labels_out: torch.Tensor | None = None,
                       stream=None):
    """Spanning forest: (pairs int32[count, 2] view of forest_out, labels or
    None).  forest_out: int32[2 * n] on the device (allocated if None)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if forest_out is None:
        forest_out = torch.empty(2 * max(n, 1), dtype=torch.int32, device=offsets.device)
    _dev(forest_out, (torch.int32,), "forest_out")
    if forest_out.numel() < 2 * n:
        raise ValueError("forest_out needs room for 2 * n values")
    if labels_out is not None:
        _dev(labels_out, (torch.int32,), "labels_out")
    so = sample if sample is not None else sample_opt()
    fo = finish if finish is not None else finish_opt()
    cnt = ctypes.c_uint64(0)
    _check(lib().cc_spanning_forest(Ip, u64, Ap, n, m, ctypes.byref(so), ctypes.byref(fo),
                                    ctypes.c_void_p(forest_out.data_ptr()), ctypes.byref(cnt),
                                    ctypes.c_void_p(labels_out.data_ptr() if labels_out is not None else 0),
                                    _stream(stream)), "cc_spanning_forest")
    return forest_out[: 2 * cnt.value].view(-1, 2), labels_out


def selftest_grid_barrier(skip_block: int = -1, wait_ms: int = 200, stream=None):
    """(status, blocks that passed) of the bounded grid-barrier self-check."""
    passed = ctypes.c_uint32(0)
    st = lib().cc_selftest_grid_barrier(skip_block, wait_ms, ctypes.byref(passed), _stream(stream))
    return st, passed.value


AMSF_MODE = {"nf": 0, "nf_s": 1, "coo": 2}


def cc_amsf(offsets, edges, weights, epsilon: float = 0.25, mode: str = "nf_s", forest_out=None, labels_out=None,
            stream=None):
    """Approximate minimum spanning forest: (pairs int32[count, 2] view of
    forest_out, total weight, labels or None)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    _dev(weights, (torch.float32,), "weights")
    if weights.numel() != m:
        raise ValueError("weights needs one value per CSR entry")
    if forest_out is None:
        forest_out = torch.empty(2 * max(n, 1), dtype=torch.int32, device=offsets.device)
    _dev(forest_out, (torch.int32,), "forest_out")
    if forest_out.numel() < 2 * n:
        raise ValueError("forest_out needs room for 2 * n values")
    if labels_out is not None:
        _dev(labels_out, (torch.int32,), "labels_out")
    cnt, wt = ctypes.c_uint64(0), ctypes.c_double(0.0)
    _check(lib().cc_amsf(Ip, u64, Ap, ctypes.c_void_p(weights.data_ptr() if m else 0), n, m, epsilon,
                         AMSF_MODE[mode] if isinstance(mode, str) else mode, ctypes.c_void_p(forest_out.data_ptr()),
                         ctypes.byref(cnt), ctypes.byref(wt),
                         ctypes.c_void_p(labels_out.data_ptr() if labels_out is not None else 0), _stream(stream)),
           "cc_amsf")
    return forest_out[: 2 * cnt.value].view(-1, 2), wt.value, labels_out


def cc_static_host(offsets: torch.Tensor, edges: torch.Tensor, sample=None, finish=None,
                   labels_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """cc_static on host (ideally pinned) tensors; copies inside the call."""
    for t, nm in ((offsets, "offsets"), (edges, "edges")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous host tensor")
    n = offsets.numel() - 1
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
    so = sample if sample is not None else sample_opt()
    fo = finish if finish is not None else finish_opt()
    _check(lib().cc_static_host(ctypes.c_void_p(offsets.data_ptr()), 1 if offsets.dtype == torch.int64 else 0,
                                ctypes.c_void_p(edges.data_ptr() if edges.numel() else 0), n, edges.numel(),
                                ctypes.byref(so), ctypes.byref(fo), ctypes.c_void_p(labels_out.data_ptr()),
                                _stream(stream)), "cc_static_host")
    return labels_out


def cc_sample(offsets, edges, sample: SampleOpt | None = None, labels_out=None, stream=None):
    """Sampled labels (min-rooted stars) and the sampling info (BFS try / LDD rounds)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    info = ctypes.c_int32(0)
    so = sample if sample is not None else sample_opt()
    _check(lib().cc_sample(Ip, u64, Ap, n, m, ctypes.byref(so), ctypes.c_void_p(labels_out.data_ptr()),
                           ctypes.byref(info), _stream(stream)), "cc_sample")
    return labels_out, info.value


def cc_identify_frequent(labels: torch.Tensor, freq_samples: int = 0, seed: int = 1, out=None, stream=None):
    _dev(labels, (torch.int32,), "labels")
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=labels.device)
    _check(lib().cc_identify_frequent(ctypes.c_void_p(labels.data_ptr()), labels.numel(), freq_samples, seed,
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)), "cc_identify_frequent")
    return out


NOALLOC_MAX_LABELS = 1 << 22


def cc_identify_frequent_noalloc(labels: torch.Tensor, out=None, stream=None):
    """Exact IdentifyFrequent that allocates nothing on the device (for
    callers that cannot allocate there); at most NOALLOC_MAX_LABELS labels.
    Calls must not overlap on the GPU: they share one scratch array."""
    _dev(labels, (torch.int32,), "labels")
    if out is None:
        raise ValueError("pass a preallocated 1-element int32 CUDA tensor as out")
    _dev(out, (torch.int32,), "out")
    _check(lib().cc_identify_frequent_noalloc(ctypes.c_void_p(labels.data_ptr()), labels.numel(),
                                              ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "cc_identify_frequent_noalloc")
    return out


def cc_finish(offsets, edges, labels_inout: torch.Tensor, lmax: int, finish: FinishOpt | None = None, stream=None):
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    _dev(labels_inout, (torch.int32,), "labels_inout")
    fo = finish if finish is not None else finish_opt()
    rounds = ctypes.c_uint32(0)
    _check(lib().cc_finish(Ip, u64, Ap, n, m, ctypes.byref(fo), lmax & 0xFFFFFFFF,
                           ctypes.c_void_p(labels_inout.data_ptr()), ctypes.byref(rounds), _stream(stream)),
           "cc_finish")
    return labels_inout, rounds.value


def device_error(stream=None) -> int:
    """Synchronise the stream and read-and-clear the sticky device error bits."""
    bits = ctypes.c_uint32(0)
    lib().cc_device_error(_stream(stream), ctypes.byref(bits))
    return bits.value


def set_iteration_cap(cap: int):
    lib().cc_set_iteration_cap(cap)


def launch_count() -> int:
    """Kernel launches the library has made in this process."""
    return int(lib().cc_launch_count())


def profile_enable(on: bool = True):
    lib().cc_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{kernel: (launches, total_ms)} since profiling was enabled."""
    L = lib()
    cnt = L.cc_profile_read(None, 0)
    arr = (KernelTime * max(cnt, 1))()
    cnt = L.cc_profile_read(ctypes.cast(arr, ctypes.c_void_p), cnt)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(cnt)}


def batch_opt(threads=1024, smem_max_vertices=65536, vertex_mode=2) -> BatchOpt:
    return BatchOpt(threads, smem_max_vertices, vertex_mode, 0)


def _batch_args(gv, offsets, edges):
    _dev(gv, (torch.int64,), "gv")
    _dev(offsets, (torch.int32, torch.int64), "offsets")
    _dev(edges, (torch.int32,), "edges")
    return (ctypes.c_void_p(gv.data_ptr()), gv.numel() - 1, ctypes.c_void_p(offsets.data_ptr()),
            1 if offsets.dtype == torch.int64 else 0, ctypes.c_void_p(edges.data_ptr() if edges.numel() else 0),
            offsets.numel() - 1, edges.numel())


def cc_batched(gv, offsets, edges, opt: BatchOpt | None = None, labels_out=None, stream=None):
    """Local min-id labels of every packed graph (see connectit_gb.h)."""
    a = _batch_args(gv, offsets, edges)
    if labels_out is None:
        labels_out = torch.empty(a[5], dtype=torch.int32, device=offsets.device)
    _check(lib().cc_batched(*a, ctypes.byref(opt) if opt is not None else None,
                            ctypes.c_void_p(labels_out.data_ptr()), _stream(stream)), "cc_batched")
    return labels_out


def cc_batched_autotune(gv, offsets, edges, labels_out=None, stream=None):
    """Time every schedule on this batch; returns (labels, best BatchOpt, best ms)."""
    a = _batch_args(gv, offsets, edges)
    if labels_out is None:
        labels_out = torch.empty(a[5], dtype=torch.int32, device=offsets.device)
    best = BatchOpt()
    ms = ctypes.c_float(0)
    _check(lib().cc_batched_autotune(*a, ctypes.c_void_p(labels_out.data_ptr()), ctypes.byref(best),
                                     ctypes.byref(ms), _stream(stream)), "cc_batched_autotune")
    return labels_out, best, ms.value


def cc_map_edges(offsets, edges, out=None, stream=None) -> torch.Tensor:
    """MapEdges: edges read per vertex (int32 view of uint32)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    _check(lib().cc_map_edges(Ip, u64, Ap, n, m, ctypes.c_void_p(out.data_ptr()), _stream(stream)), "cc_map_edges")
    return out


def cc_gather_edges(offsets, edges, x, out=None, stream=None) -> torch.Tensor:
    """GatherEdges: per vertex, the sum mod 2^32 of x over its neighbours."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    _dev(x, (torch.int32,), "x")
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    _check(lib().cc_gather_edges(Ip, u64, Ap, n, m, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 _stream(stream)), "cc_gather_edges")
    return out


def cc_random_sectors(x, count: int, seed: int = 1, out=None, stream=None) -> torch.Tensor:
    """Random-sector reads: the sum mod 2^32 of `count` seeded random words of x
    (int32 CUDA tensor), one device word."""
    _dev(x, (torch.int32,), "x")
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=x.device)
    _check(lib().cc_random_sectors(ctypes.c_void_p(x.data_ptr()), ctypes.c_uint64(x.numel()), ctypes.c_uint64(count),
                                   ctypes.c_uint64(seed), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "cc_random_sectors")
    return out


def cc_features(offsets, edges, seed: int = 1, out=None, stream=None) -> torch.Tensor:
    """The selector's 16 graph features (float32 CUDA tensor)."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if out is None:
        out = torch.empty(16, dtype=torch.float32, device=offsets.device)
    _check(lib().cc_features(Ip, u64, Ap, n, m, seed, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "cc_features")
    return out


def cc_select_static(offsets, edges, params=None, force_class: int = -1, seed: int = 1, labels_out=None,
                     feat_out=None, stream=None):
    """The selected static path: labels (int32 view of uint32) and the class
    run (see connectit_gb.h).  params: the MLP's parameter tensor (CUDA
    float32), or None with force_class >= 0."""
    Ip, u64, Ap, n, m = _graph_args(offsets, edges)
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    cls = ctypes.c_int32(-1)
    pp = ctypes.c_void_p(params.data_ptr()) if params is not None else None
    fp = ctypes.c_void_p(feat_out.data_ptr()) if feat_out is not None else None
    _check(lib().cc_select_static(Ip, u64, Ap, n, m, pp, force_class, seed, ctypes.c_void_p(labels_out.data_ptr()),
                                  fp, ctypes.byref(cls), _stream(stream)), "cc_select_static")
    return labels_out, cls.value


MLP_IN, MLP_HID, MLP_OUT = 16, 64, 12
MLP_NPARAM = 2 * MLP_IN + MLP_IN * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID * MLP_OUT + MLP_OUT


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def mlp_init(params, seed=1, stream=None):
    _check(lib().cc_mlp_init(_p(params), seed, _stream(stream)), "cc_mlp_init")


def mlp_set_norm(params, X, stream=None):
    _check(lib().cc_mlp_set_norm(_p(params), _p(X), X.shape[0], _stream(stream)), "cc_mlp_set_norm")


def mlp_forward(params, X, logits, acts=None, stream=None):
    _check(lib().cc_mlp_forward(_p(params), _p(X), X.shape[0], _p(logits), _p(acts), _stream(stream)),
           "cc_mlp_forward")


def mlp_soft_targets(times, tau, targets, stream=None):
    _check(lib().cc_mlp_soft_targets(_p(times), times.shape[0], tau, _p(targets), _stream(stream)),
           "cc_mlp_soft_targets")


def mlp_backward(params, X, acts, logits, targets, grads, loss=None, stream=None):
    _check(lib().cc_mlp_backward(_p(params), _p(X), _p(acts), _p(logits), _p(targets), X.shape[0], _p(grads),
                                 _p(loss), _stream(stream)), "cc_mlp_backward")


def mlp_adam(params, grads, m, v, step, lr, stream=None):
    _check(lib().cc_mlp_adam(_p(params), _p(grads), _p(m), _p(v), step, lr, _stream(stream)), "cc_mlp_adam")


def mlp_predict(params, X, out, stream=None):
    _check(lib().cc_mlp_predict(_p(params), _p(X), X.shape[0], _p(out), _stream(stream)), "cc_mlp_predict")


class Incremental:
    """Resident union-find for batch-incremental connectivity."""

    def __init__(self, n: int, offsets=None, edges=None, sample=None, finish=None, stream=None, device=None):
        self._h = ctypes.c_void_p(0)
        so = sample if sample is not None else sample_opt()
        fo = finish if finish is not None else finish_opt()
        if offsets is not None:
            Ip, u64, Ap, n2, m = _graph_args(offsets, edges)
            assert n2 == n
            self.device = offsets.device
        else:
            Ip, u64, Ap, m = ctypes.c_void_p(0), 0, ctypes.c_void_p(0), 0
            self.device = torch.device(device or "cuda")
        _check(lib().cc_incr_create(Ip, u64, Ap, n, m, ctypes.byref(so), ctypes.byref(fo), _stream(stream),
                                    ctypes.byref(self._h)), "cc_incr_create")
        self.n = n

    def insert(self, pairs: torch.Tensor, stream=None):
        _dev(pairs, (torch.int32,), "pairs")
        _check(lib().cc_incr_insert_batch(self._h, ctypes.c_void_p(pairs.data_ptr()), pairs.numel() // 2,
                                          _stream(stream)), "cc_incr_insert_batch")

    def query(self, pairs: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _dev(pairs, (torch.int32,), "pairs")
        q = pairs.numel() // 2
        if out is None:
            out = torch.empty(q, dtype=torch.uint8, device=pairs.device)
        _check(lib().cc_incr_query_batch(self._h, ctypes.c_void_p(pairs.data_ptr()), q,
                                         ctypes.c_void_p(out.data_ptr()), _stream(stream)), "cc_incr_query_batch")
        return out

    def labels(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _check(lib().cc_incr_labels(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)), "cc_incr_labels")
        return out

    def close(self):
        if self._h:
            lib().cc_incr_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over an Incremental handle.  Host
    tensors (pinned for overlap) are kept alive until wait()."""

    STAGE = 1

    def __init__(self, inc: "Incremental", slots: int = 4, slot_pairs: int = 1 << 22, stage: bool = False):
        self._s = ctypes.c_void_p(0)
        self._keep = {}
        self.inc = inc
        opt = ServerOpt(slots, self.STAGE if stage else 0, slot_pairs)
        _check(lib().cc_server_create(inc._h, ctypes.byref(opt), ctypes.byref(self._s)), "cc_server_create")

    def submit(self, inserts: torch.Tensor | None, queries: torch.Tensor | None, answers: torch.Tensor | None = None):
        for t, nm in ((inserts, "inserts"), (queries, "queries")):
            if t is not None and (t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous()):
                raise TypeError(f"{nm} must be a contiguous host int32 tensor")
        k = inserts.numel() // 2 if inserts is not None else 0
        q = queries.numel() // 2 if queries is not None else 0
        if answers is None:
            answers = torch.empty(q, dtype=torch.uint8, pin_memory=True)
        t = ctypes.c_uint64(0)
        _check(lib().cc_server_submit(self._s, ctypes.c_void_p(inserts.data_ptr() if k else 0), k,
                                      ctypes.c_void_p(queries.data_ptr() if q else 0), q,
                                      ctypes.c_void_p(answers.data_ptr() if q else 0), ctypes.byref(t)),
               "cc_server_submit")
        self._keep[t.value] = (inserts, queries, answers)
        return t.value

    def wait(self, ticket: int):
        """Returns (answers tensor, latency in ms)."""
        lat = ctypes.c_double(0)
        _check(lib().cc_server_wait(self._s, ticket, ctypes.byref(lat)), "cc_server_wait")
        ins, qs, ans = self._keep.pop(ticket)
        return ans, lat.value

    def close(self):
        if self._s:
            lib().cc_server_destroy(self._s)
            self._s = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
